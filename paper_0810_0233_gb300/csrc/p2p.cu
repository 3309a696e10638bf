// p2p.cu -- near field (Eq. H2 as read: field of dipole j at i,
// [3 (m_j.u) u - m_j] / r^3) over each leaf's nearPartners (Appendix,
// updateField), the final unpermute + energy (E = -1/2 sum m.H), and the
// FP64 direct sum used to measure the error of the fast method.
#include "ccfmm_dev.cuh"

namespace ccfmm {

constexpr int P2P_T = 128;
constexpr int P2P_CH = 1024;  // sources staged in shared memory per batch

template <typename real> __device__ __forceinline__ real rsqrt_or_zero(real r2);
template <> __device__ __forceinline__ float rsqrt_or_zero<float>(float r2)
{
    return r2 > 0.f ? rsqrtf(r2) : 0.f;
}
template <> __device__ __forceinline__ double rsqrt_or_zero<double>(double r2)
{
    return r2 > 0.0 ? 1.0 / sqrt(r2) : 0.0;
}

// One block per target leaf.  Targets are spread over the block's threads
// with S = floor(128 / nt) stripes of sources per target; source dipoles of
// the near leaves are staged in shared memory with positions relative to the
// target leaf centre, s_j = l_j - (c_target - c_source), so every difference
// is formed between numbers of leaf-size magnitude.  A source located at the
// field point (the target itself) gives r = 0 and contributes nothing.
template <typename real>
__global__ void __launch_bounds__(P2P_T) k_p2p(int L, const int *leaf_start,
                                               const int *near_start, const NearEnt *near,
                                               const Geom *g, const typename vec4<real>::t *A,
                                               const typename vec2<real>::t *B,
                                               typename vec4<real>::t *H)
{
    typedef typename vec4<real>::t R4;
    __shared__ R4 sp[P2P_CH];          // (sx, sy, sz, mx)
    __shared__ real sm2[P2P_CH][2];    // (my, mz)
    const long long key = blockIdx.x;
    const int t0 = leaf_start[key], nt = leaf_start[key + 1] - t0;
    if (nt == 0) return;
    const int e0 = near_start[key], e1 = near_start[key + 1];
    const double wx = g->w[L][0], wy = g->w[L][1], wz = g->w[L][2];
    const int tid = threadIdx.x;

    for (int tb = 0; tb < nt; tb += P2P_T) {
        const int ntc = min(nt - tb, P2P_T);
        const int S = max(1, P2P_T / ntc);
        const int ti = tid % ntc, stripe = tid / ntc;
        const bool active = stripe < S;
        real xi = 0, yi = 0, zi = 0;
        if (active) {
            R4 a = A[t0 + tb + ti];
            xi = a.x;
            yi = a.y;
            zi = a.z;
        }
        real hx = 0, hy = 0, hz = 0;
        int fill = 0;
        for (int e = e0; e <= e1; ++e) {
            int cnt = 0, sb = 0;
            real dx = 0, dy = 0, dz = 0;
            if (e < e1) {
                NearEnt ne = near[e];
                sb = leaf_start[ne.src];
                cnt = leaf_start[ne.src + 1] - sb;
                dx = (real)((double)ne.ox * wx);
                dy = (real)((double)ne.oy * wy);
                dz = (real)((double)ne.oz * wz);
            }
            int done = 0;
            while (true) {
                int take = min(cnt - done, P2P_CH - fill);
                bool flush = (e == e1) ? (fill > 0) : (take < cnt - done || fill + take == P2P_CH);
                for (int j = tid; j < take; j += P2P_T) {
                    R4 a = A[sb + done + j];
                    typename vec2<real>::t b = B[sb + done + j];
                    R4 v;
                    v.x = a.x - dx;
                    v.y = a.y - dy;
                    v.z = a.z - dz;
                    v.w = a.w;
                    sp[fill + j] = v;
                    sm2[fill + j][0] = b.x;
                    sm2[fill + j][1] = b.y;
                }
                fill += take;
                done += take;
                if (flush) {
                    __syncthreads();
                    if (active) {
#pragma unroll 4
                        for (int j = stripe; j < fill; j += S) {
                            R4 s = sp[j];
                            real mx = s.w, my = sm2[j][0], mz = sm2[j][1];
                            real rx = xi - s.x, ry = yi - s.y, rz = zi - s.z;
                            real r2 = rx * rx + ry * ry + rz * rz;
                            real ri = rsqrt_or_zero<real>(r2);
                            real ri2 = ri * ri;
                            real ri3 = ri2 * ri;
                            real mr = mx * rx + my * ry + mz * rz;
                            real t3 = (real)3 * mr * ri2 * ri3;
                            hx += t3 * rx - mx * ri3;
                            hy += t3 * ry - my * ri3;
                            hz += t3 * rz - mz * ri3;
                        }
                    }
                    __syncthreads();
                    fill = 0;
                }
                if (done >= cnt) break;
            }
        }
        // reduce the stripes of each target through shared memory
        real *red = reinterpret_cast<real *>(sp);
        red[3 * tid + 0] = hx;
        red[3 * tid + 1] = hy;
        red[3 * tid + 2] = hz;
        __syncthreads();
        if (tid < ntc) {
            real sx = 0, sy = 0, sz = 0;
            for (int st = 0; st < S; ++st) {
                int q = st * ntc + tid;
                sx += red[3 * q + 0];
                sy += red[3 * q + 1];
                sz += red[3 * q + 2];
            }
            R4 h = H[t0 + tb + tid];
            h.x += sx;
            h.y += sy;
            h.z += sz;
            H[t0 + tb + tid] = h;
        }
        __syncthreads();
    }
}

template <typename real>
void launch_p2p(int L, const int *leaf_start, const int *near_start, const NearEnt *near,
                const Geom *d_geom, const typename vec4<real>::t *A,
                const typename vec2<real>::t *B, typename vec4<real>::t *H, cudaStream_t s)
{
    note_launch();
    k_p2p<real><<<(unsigned)(1ll << L), P2P_T, 0, s>>>(L, leaf_start, near_start, near, d_geom, A,
                                                      B, H);
}

// unpermute to input order in FP64 and form per-block partial sums of m.H
constexpr int FIN_T = 256;

template <typename real>
__global__ void __launch_bounds__(FIN_T) k_finish(const typename vec4<real>::t *H, const int *perm,
                                                  const double *mom, long long n, double *Hout,
                                                  double *partial)
{
    __shared__ double red[FIN_T / 32];
    double e = 0.0;
    long long s = (long long)blockIdx.x * FIN_T + threadIdx.x;
    if (s < n) {
        long long i = perm[s];
        typename vec4<real>::t h = H[s];
        double hx = (double)h.x, hy = (double)h.y, hz = (double)h.z;
        if (Hout) {
            Hout[3 * i] = hx;
            Hout[3 * i + 1] = hy;
            Hout[3 * i + 2] = hz;
        }
        e = mom[3 * i] * hx + mom[3 * i + 1] * hy + mom[3 * i + 2] * hz;
    }
    for (int o = 16; o; o >>= 1) e += __shfl_xor_sync(0xffffffffu, e, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = e;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < FIN_T / 32; ++w) t += red[w];
        partial[blockIdx.x] = t;
    }
}

// E = -1/2 sum of the partials, summed in a fixed order
__global__ void k_energy_final(const double *partial, long long nparts, double *E)
{
    __shared__ double red[256];
    double t = 0.0;
    for (long long b = threadIdx.x; b < nparts; b += 256) t += partial[b];
    red[threadIdx.x] = t;
    __syncthreads();
    for (int w = 128; w; w >>= 1) {
        if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) *E = -0.5 * red[0];
}

template <typename real>
void launch_finish(const typename vec4<real>::t *H, const int *perm, const double *mom,
                   long long n, double *H_out, double *partial, double *d_E, cudaStream_t s)
{
    long long nb = (n + FIN_T - 1) / FIN_T;
    note_launch();
    k_finish<real><<<(unsigned)nb, FIN_T, 0, s>>>(H, perm, mom, n, H_out, partial);
    note_launch();
    k_energy_final<<<1, 256, 0, s>>>(partial, nb, d_E);
}

// FP64 direct sum at selected targets: block of 128 targets, sources staged
// through shared memory 256 at a time.  j == i and r == 0 are skipped.
__global__ void __launch_bounds__(128) k_direct(const double *pos, const double *mom, long long n,
                                                const long long *tgt, long long nt, double *Hout)
{
    __shared__ double sp[256][6];
    long long t = (long long)blockIdx.x * 128 + threadIdx.x;
    long long i = -1;
    double xi = 0, yi = 0, zi = 0;
    if (t < nt) {
        i = tgt ? tgt[t] : t;
        xi = pos[3 * i];
        yi = pos[3 * i + 1];
        zi = pos[3 * i + 2];
    }
    double hx = 0, hy = 0, hz = 0;
    for (long long b = 0; b < n; b += 256) {
        __syncthreads();
        for (int j = threadIdx.x; j < 256; j += 128) {
            long long q = b + j;
            if (q < n)
                for (int c = 0; c < 3; ++c) {
                    sp[j][c] = pos[3 * q + c];
                    sp[j][3 + c] = mom[3 * q + c];
                }
        }
        __syncthreads();
        int m = (int)min((long long)256, n - b);
        for (int j = 0; j < m; ++j) {
            if (b + j == i) continue;
            double rx = xi - sp[j][0], ry = yi - sp[j][1], rz = zi - sp[j][2];
            double r2 = rx * rx + ry * ry + rz * rz;
            if (r2 == 0.0) continue;
            double ri = 1.0 / sqrt(r2);
            double ri3 = ri * ri * ri;
            double mr = sp[j][3] * rx + sp[j][4] * ry + sp[j][5] * rz;
            double t3 = 3.0 * mr * ri * ri * ri3;
            hx += t3 * rx - sp[j][3] * ri3;
            hy += t3 * ry - sp[j][4] * ri3;
            hz += t3 * rz - sp[j][5] * ri3;
        }
    }
    if (t < nt) {
        Hout[3 * t] = hx;
        Hout[3 * t + 1] = hy;
        Hout[3 * t + 2] = hz;
    }
}

void launch_direct(const double *pos, const double *mom, long long n, const long long *tgt,
                   long long nt, double *H_out, cudaStream_t s)
{
    if (nt <= 0) return;
    note_launch();
    k_direct<<<(unsigned)((nt + 127) / 128), 128, 0, s>>>(pos, mom, n, tgt, nt, H_out);
}

// pairs (i, j), j != i, evaluated by the near field: sum over leaves of
// nt * (sum of near-leaf counts) - nt
__global__ void k_pair_count(int L, const int *leaf_start, const int *near_start,
                             const NearEnt *near, unsigned long long *count)
{
    long long key = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (key >= (1ll << L)) return;
    long long nt = leaf_start[key + 1] - leaf_start[key];
    if (!nt) return;
    long long ns = 0;
    for (int e = near_start[key]; e < near_start[key + 1]; ++e)
        ns += leaf_start[near[e].src + 1] - leaf_start[near[e].src];
    atomicAdd(count, (unsigned long long)(nt * ns - nt));
}

void launch_p2p_pair_count(int L, const int *leaf_start, const int *near_start,
                           const NearEnt *near, unsigned long long *d_count, cudaStream_t s)
{
    cudaMemsetAsync(d_count, 0, sizeof(unsigned long long), s);
    long long n = 1ll << L;
    note_launch();
    k_pair_count<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(L, leaf_start, near_start, near,
                                                            d_count);
}

#define INST(real)                                                                              \
    template void launch_p2p<real>(int, const int *, const int *, const NearEnt *,             \
                                   const Geom *, const vec4<real>::t *, const vec2<real>::t *,  \
                                   vec4<real>::t *, cudaStream_t);                             \
    template void launch_finish<real>(const vec4<real>::t *, const int *, const double *,       \
                                      long long, double *, double *, double *, cudaStream_t);
INST(float)
INST(double)
#undef INST

}  // namespace ccfmm
