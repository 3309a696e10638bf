// expand.cu -- Cartesian expansion operators of Sec. III on the GPU:
//   F table of Eqs. Dn / Dnr and the derivative tensors D_n per distinct
//   (level, far offset), P2M (Eq. multipolemoments), M2M (Eq. momentshift),
//   L2L (Eq. taylorshift) and L2P (Eq. H, H = -grad V).  P2M's body
//   (p2m_run) is in stages.cuh.
#include "ccfmm_dev.cuh"
#include "stages.cuh"

namespace ccfmm {

__device__ __forceinline__ int order_of(int t)
{
    int k = 0;
    while (nterms(k) <= t) ++k;
    return k;
}

// position of a multi-index inside its order (library ordering)
__device__ __forceinline__ int loc_in_order(int nx, int ny, int nz)
{
    int k = nx + ny + nz;
    return nz * (2 * k + 3 - nz) / 2 + ny;
}


// ---------------------------------------------------------------------------
// F table (Eqs. Dn, Dnr).  D_n(r) = r^-(2|n|+1) sum_{|q|=|n|} F_n(q) r^q with
// D_{n+e_v} = -d/dx_v D_n, so F_{n} is built from F_{n-e_v} (v = first axis
// with n_v > 0):  F_n(q'+e_v) += (2|m|+1-q'_v) F_m(q'),
//                 F_n(q'-e_v+2e_mu) += -q'_v F_m(q')  (mu != v),  m = n-e_v,
// from F_0(0) = 1.  Dense per-order blocks in scratch, then the non-zeros.
// ---------------------------------------------------------------------------
__host__ __device__ inline long long ft_block_off(int k)
{
    long long off = 0;
    for (int j = 0; j < k; ++j) {
        long long t = (long long)(j + 1) * (j + 2) / 2;
        off += t * t;
    }
    return off;
}

size_t ftable_scratch_bytes(int order) { return (size_t)ft_block_off(order + 1) * sizeof(double); }

__global__ void k_ftable(int O, double *dense, int *f_start, uint16_t *f_q, double *f_val)
{
    if (threadIdx.x == 0) dense[0] = 1.0;
    __syncthreads();
    for (int k = 1; k <= O; ++k) {
        int Tk = (k + 1) * (k + 2) / 2, Tm = k * (k + 1) / 2;
        double *blk = dense + ft_block_off(k);
        const double *pb = dense + ft_block_off(k - 1);
        for (int r = threadIdx.x; r < Tk; r += blockDim.x) {
            int nx, ny, nz;
            midx_inv(nterms(k - 1) + r, nx, ny, nz);
            int n[3] = {nx, ny, nz};
            int v = n[0] > 0 ? 0 : (n[1] > 0 ? 1 : 2);
            int m[3] = {n[0], n[1], n[2]};
            m[v] -= 1;
            int rm = loc_in_order(m[0], m[1], m[2]);
            double *row = blk + (long long)r * Tk;
            for (int q = 0; q < Tk; ++q) row[q] = 0.0;
            for (int j = 0; j < Tm; ++j) {
                double f = pb[(long long)rm * Tm + j];
                if (f == 0.0) continue;
                int qx, qy, qz;
                midx_inv(nterms(k - 2) + j, qx, qy, qz);
                int q[3] = {qx, qy, qz};
                int a[3] = {q[0], q[1], q[2]};
                a[v] += 1;
                row[loc_in_order(a[0], a[1], a[2])] += (double)(2 * (k - 1) + 1 - q[v]) * f;
                if (q[v] > 0) {
                    for (int mu = 0; mu < 3; ++mu) {
                        if (mu == v) continue;
                        int b[3] = {q[0], q[1], q[2]};
                        b[v] -= 1;
                        b[mu] += 2;
                        row[loc_in_order(b[0], b[1], b[2])] += -(double)q[v] * f;
                    }
                }
            }
        }
        __syncthreads();
    }
    // sparse rows: one row per multi-index t, entries (packed q, F_n(q))
    int T = nterms(O);
    if (threadIdx.x == 0) {
        int nnz = 0;
        for (int t = 0; t < T; ++t) {
            f_start[t] = nnz;
            int k = order_of(t), Tk = (k + 1) * (k + 2) / 2;
            const double *row = dense + ft_block_off(k) + (long long)(t - nterms(k - 1)) * Tk;
            for (int q = 0; q < Tk; ++q)
                if (row[q] != 0.0) ++nnz;
        }
        f_start[T] = nnz;
    }
    __syncthreads();
    for (int t = threadIdx.x; t < T; t += blockDim.x) {
        int k = order_of(t), Tk = (k + 1) * (k + 2) / 2;
        const double *row = dense + ft_block_off(k) + (long long)(t - nterms(k - 1)) * Tk;
        int e = f_start[t];
        for (int q = 0; q < Tk; ++q) {
            if (row[q] == 0.0) continue;
            int qx, qy, qz;
            midx_inv(nterms(k - 1) + q, qx, qy, qz);
            f_q[e] = (uint16_t)pack3(qx, qy, qz);
            f_val[e] = row[q];
            ++e;
        }
    }
}

void launch_ftable(int order, double *dense_scratch, int *f_start, uint16_t *f_q, double *f_val,
                   cudaStream_t s)
{
    note_launch();
    k_ftable<<<1, 256, 0, s>>>(order, dense_scratch, f_start, f_q, f_val);
}

// D tensors of one (level, offset) per block, in FP64, at the scaled
// separation c/h (c = o * w_l, h = cell radius of the level):
// D~_n = D_n(c/h) = D_n(c) h^(|n|+1).  Row gid of D, with a zero at column
// T(2p) used for padding.
template <typename real>
__global__ void k_dtables(int O, const int *f_start, const uint16_t *f_q, const double *f_val,
                          const double4 *sep, real *D, int ldD)
{
    __shared__ double xp[2 * PMAX + 1], yp[2 * PMAX + 1], zp[2 * PMAX + 1], rp[2 * PMAX + 1];
    int gid = blockIdx.x;
    if (threadIdx.x == 0) {
        const double4 c = sep[gid];  // separation / cell radius
        double x = c.x, y = c.y, z = c.z;
        double rinv = 1.0 / sqrt(x * x + y * y + z * z);
        double r2inv = rinv * rinv;
        xp[0] = yp[0] = zp[0] = 1.0;
        rp[0] = rinv;
        for (int j = 1; j <= O; ++j) {
            xp[j] = xp[j - 1] * x;
            yp[j] = yp[j - 1] * y;
            zp[j] = zp[j - 1] * z;
            rp[j] = rp[j - 1] * r2inv;
        }
    }
    __syncthreads();
    int T = nterms(O);
    for (int t = threadIdx.x; t < T; t += blockDim.x) {
        double s = 0.0;
        for (int e = f_start[t]; e < f_start[t + 1]; ++e) {
            unsigned q = f_q[e];
            s += f_val[e] * xp[px(q)] * yp[py(q)] * zp[pz(q)];
        }
        D[(long long)gid * ldD + t] = (real)(s * rp[order_of(t)]);
    }
    for (int t = T + threadIdx.x; t < ldD; t += blockDim.x) D[(long long)gid * ldD + t] = (real)0;
}

template <typename real>
void launch_dtables(int p, const int *f_start, const uint16_t *f_q, const double *f_val,
                    const double4 *sep, int nd, real *D, int ldD, cudaStream_t s)
{
    if (nd <= 0) return;
    note_launch();
    k_dtables<real><<<nd, 128, 0, s>>>(2 * p, f_start, f_q, f_val, sep, D, ldD);
}

// M2L index table: it[k][n] = D-row column of multi-index (n + k) for
// coefficient columns n, k < K with |n|+|k| <= maxdeg; the zero column T(2p)
// for padding and for the pairs that the truncation drops.
__global__ void k_itable(int p, int KP, int maxdeg, uint16_t *it)
{
    int K = nterms(p) - 1, zero = nterms(2 * p);
    int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= KP * KP) return;
    int ck = j / KP, cn = j % KP;
    int v = zero;
    if (ck < K && cn < K && ck < m2l_kend(p, maxdeg, cn)) {
        int ax, ay, az, bx, by, bz;
        midx_inv(ck + 1, ax, ay, az);
        midx_inv(cn + 1, bx, by, bz);
        v = midx(ax + bx, ay + by, az + bz);
    }
    it[j] = (uint16_t)v;
}

void launch_itable(int p, int KP, int maxdeg, uint16_t *it, cudaStream_t s)
{
    note_launch();
    k_itable<<<(KP * KP + 255) / 256, 256, 0, s>>>(p, KP, maxdeg, it);
}

template <typename real>
__device__ __forceinline__ void p2m_body(int p, int KP, int L, const int *leaf_start,
                                         const typename vec4<real>::t *A,
                                         const typename vec2<real>::t *B, real *Q, long long blk)
{
    const int w = threadIdx.x >> 5;
    const long long key = blk * P2M_W + w;
    const bool live = key < (1ll << L);
    const int s0 = live ? leaf_start[key] : 0, s1 = live ? leaf_start[key + 1] : 0;
    const long long hid = (1ll << L) + key;
    __shared__ P2MScratch<real> sc;
    p2m_run<real>(p, KP, live, s0, s1, A, B, live ? Q + hid * KP : Q, sc);
}

template <typename real>
__global__ void __launch_bounds__(32 * P2M_W) k_p2m(int p, int KP, int L, const int *leaf_start,
                                                    const typename vec4<real>::t *A,
                                                    const typename vec2<real>::t *B, real *Q)
{
    p2m_body<real>(p, KP, L, leaf_start, A, B, Q, blockIdx.x);
}

__global__ void __launch_bounds__(32 * P2M_W) k_p2m_batch(const P2MArgs *a, const int *bstart,
                                                          int nm)
{
    int blk;
    const P2MArgs &x = a[batch_member(bstart, nm, blockIdx.x, blk)];
    p2m_body<float>(x.p, x.KP, x.L, x.leaf_start, x.A, x.B, x.Q, blk);
}

int p2m_blocks(int L) { return (int)(((1ll << L) + P2M_W - 1) / P2M_W); }

void launch_p2m_batch(const P2MArgs *a, const int *bstart, int nm, int nblocks, cudaStream_t s)
{
    if (nblocks <= 0) return;
    note_launch();
    k_p2m_batch<<<(unsigned)nblocks, 32 * P2M_W, 0, s>>>(a, bstart, nm);
}

template <typename real>
void launch_p2m(int p, int KP, int L, const int *leaf_start, const typename vec4<real>::t *A,
                const typename vec2<real>::t *B, real *Q, cudaStream_t s)
{
    const long long nleaf = 1ll << L;
    note_launch();
    k_p2m<real><<<(unsigned)((nleaf + P2M_W - 1) / P2M_W), 32 * P2M_W, 0, s>>>(p, KP, L,
                                                                             leaf_start, A, B, Q);
}

// P2M of the adaptive-depth tree: one warp per leaf cell (any level), the
// dipoles' coordinates relative to that leaf's centre.
template <typename real>
__global__ void __launch_bounds__(32 * P2M_W) k_ap2m(int p, int KP, int nleaf, const int *leaves,
                                                     const int *p0, const int *np,
                                                     const typename vec4<real>::t *A,
                                                     const typename vec2<real>::t *B, real *Q)
{
    const long long li = (long long)blockIdx.x * P2M_W + (threadIdx.x >> 5);
    const bool live = li < nleaf;
    const int c = live ? leaves[li] : 0;
    const int s0 = live ? p0[c] : 0, s1 = live ? s0 + np[c] : 0;
    __shared__ P2MScratch<real> sc;
    p2m_run<real>(p, KP, live, s0, s1, A, B, Q + (long long)c * KP, sc);
}

template <typename real>
void launch_ap2m(int p, int KP, int nleaf, const int *leaves, const int *p0, const int *np,
                 const typename vec4<real>::t *A, const typename vec2<real>::t *B, real *Q,
                 cudaStream_t s)
{
    if (nleaf <= 0) return;
    note_launch();
    k_ap2m<real><<<(unsigned)((nleaf + P2M_W - 1) / P2M_W), 32 * P2M_W, 0, s>>>(p, KP, nleaf, leaves,
                                                                              p0, np, A, B, Q);
}

// ---------------------------------------------------------------------------
// M2M (Eq. momentshift) and L2L (Eq. taylorshift, FP64), several levels per
// launch.  The child centre sits at -w/2 (bit 0) or +w/2 (bit 1) along the
// axis split at the child's level, so only shifts along that axis appear:
//     M2M  Q_n(parent) = sum_children sum_t c^t/t! Q^child_{n - t e_s},
//     L2L  V^child_n  += sum_t c^t/t! V^parent_{n + t e_s},  |n| + t <= p.
// A block owns a subtree of depth D <= 3 below a cell of level l0 and
// carries the expansions of one level of it in shared memory to the next,
// so that the whole upward pass takes ceil(L / 3) launches (the downward
// pass ceil((L - 1) / 3)).  The shift factors c^t/t! of the two children are
// formed once per level by the recurrence f_t = f_(t-1) c / t.
// ---------------------------------------------------------------------------
constexpr int SUB_T = 256;
constexpr int SUB_D = 3;  // levels per launch
constexpr int SUB_KP = ((nterms(PMAX) - 1 + 7) / 8) * 8;

// Q of the 2^D descendants at level l0 + D (final) -> Q of levels
// l0 + D - 1 .. l0 of the subtree rooted at key r (blockIdx.x) of level l0
template <typename real>
__device__ __forceinline__ void m2m_sub_body(int p, int KP, int l0, int D, const Geom *g, real *Q,
                                             long long r)
{
    __shared__ real qs[2][1 << SUB_D][SUB_KP];
    __shared__ real fs[2][PMAX + 1];
    __shared__ unsigned mi[SUB_KP];
    const int K = nterms(p) - 1;
    fill_mi(mi, K);  // read after the first barrier below
    int cur = 0;
    {
        const int n = 1 << D;
        const long long hid0 = (1ll << (l0 + D)) + (r << D);
        for (int i = threadIdx.x; i < n * KP; i += SUB_T)
            qs[0][i / KP][i % KP] = Q[(hid0 + i / KP) * KP + i % KP];
    }
    for (int d = D - 1; d >= 0; --d) {
        const int lp = l0 + d;  // parent level of this step
        const int sx = g->axis[lp + 1];
        __syncthreads();  // qs[cur] complete, fs free
        if (threadIdx.x < 2) {
            const real hw = (real)(0.5 * g->w[lp + 1][sx]);
            const real cs = threadIdx.x ? hw : -hw;
            real f = (real)1;
            fs[threadIdx.x][0] = f;
            for (int t = 1; t <= p; ++t) {
                f = f * cs / (real)t;
                fs[threadIdx.x][t] = f;
            }
        }
        __syncthreads();
        const int n = 1 << d;
        const long long hidp = (1ll << lp) + (r << d);
        for (int i = threadIdx.x; i < n * KP; i += SUB_T) {
            const int cell = i / KP, c = i - cell * KP;
            real acc = (real)0;
            if (c < K) {
                const unsigned mc = mi[c];
                const int nn[3] = {px(mc), py(mc), pz(mc)};
                for (int b = 0; b < 2; ++b) {
                    const real *Qc = qs[cur][2 * cell + b];
                    for (int t = 0; t <= nn[sx]; ++t) {
                        int m[3] = {nn[0], nn[1], nn[2]};
                        m[sx] -= t;
                        if (m[0] + m[1] + m[2] > 0) acc += fs[b][t] * Qc[midx(m[0], m[1], m[2]) - 1];
                    }
                }
            }
            qs[cur ^ 1][cell][c] = acc;
            Q[(hidp + cell) * KP + c] = acc;
        }
        cur ^= 1;
    }
}

template <typename real>
__global__ void __launch_bounds__(SUB_T) k_m2m_sub(int p, int KP, int l0, int D, const Geom *g,
                                                   real *Q)
{
    m2m_sub_body<real>(p, KP, l0, D, g, Q, blockIdx.x);
}

__global__ void __launch_bounds__(SUB_T) k_m2m_batch(const M2MArgs *a, const int *bstart, int nm)
{
    int r;
    const M2MArgs &x = a[batch_member(bstart, nm, blockIdx.x, r)];
    m2m_sub_body<float>(x.p, x.KP, x.l0, x.D, x.g, x.Q, r);
}

int m2m_rounds(int L, int *l0, int *D)
{
    int n = 0;
    for (int cur = L; cur > 0; ++n) {
        D[n] = cur < SUB_D ? cur : SUB_D;
        l0[n] = cur - D[n];
        cur = l0[n];
    }
    return n;
}

int l2l_rounds(int L, int *l0, int *D)
{
    int n = 0;
    for (int cur = 1; cur < L; ++n) {
        l0[n] = cur;
        D[n] = L - cur < SUB_D ? L - cur : SUB_D;
        cur += D[n];
    }
    return n;
}

template <typename real>
void launch_m2m_all(int p, int KP, int L, const Geom *d_geom, real *Q, cudaStream_t s)
{
    int l0[LCAP + 1], D[LCAP + 1];
    const int n = m2m_rounds(L, l0, D);
    for (int r = 0; r < n; ++r) {
        note_launch();
        k_m2m_sub<real><<<(unsigned)(1ll << l0[r]), SUB_T, 0, s>>>(p, KP, l0[r], D[r], d_geom, Q);
    }
}

void launch_m2m_batch(const M2MArgs *a, const int *bstart, int nm, int nblocks, cudaStream_t s)
{
    if (nblocks <= 0) return;
    note_launch();
    k_m2m_batch<<<(unsigned)nblocks, SUB_T, 0, s>>>(a, bstart, nm);
}

// V of the root (key r of level l0, final) and the levels' own M2L
// contributions -> V of levels l0 + 1 .. l0 + D of the subtree (FP64);
// empty cells are skipped (their coefficients never reach a field point)
__device__ __forceinline__ void l2l_sub_body(int p, int KP, int l0, int D, int L, const Geom *g,
                                             const int *leaf_start, double *V, long long r)
{
    __shared__ double vs[2][1 << SUB_D][SUB_KP];
    __shared__ double fs[2][PMAX + 1];
    __shared__ int full[2][1 << SUB_D];
    __shared__ unsigned mi[SUB_KP];
    const int K = nterms(p) - 1;
    fill_mi(mi, K);  // read after the first barrier below
    int cur = 0;
    const long long hr = (1ll << l0) + r;
    for (int c = threadIdx.x; c < KP; c += SUB_T) vs[0][0][c] = V[hr * KP + c];
    if (threadIdx.x == 0)
        full[0][0] = leaf_start[(r + 1) << (L - l0)] > leaf_start[r << (L - l0)];
    for (int d = 1; d <= D; ++d) {
        const int l = l0 + d;
        const int sx = g->axis[l];
        __syncthreads();  // vs[cur], full[cur] complete; fs free
        if (threadIdx.x < 2) {
            const double cs = threadIdx.x ? 0.5 * g->w[l][sx] : -0.5 * g->w[l][sx];
            double f = 1.0;
            fs[threadIdx.x][0] = 1.0;
            for (int t = 1; t <= p; ++t) {
                f = f * cs / (double)t;
                fs[threadIdx.x][t] = f;
            }
        }
        const int n = 1 << d;
        const long long key0 = r << d;
        if (threadIdx.x < n) {
            const long long key = key0 + threadIdx.x;
            const int sh = L - l;
            full[cur ^ 1][threadIdx.x] =
                full[cur][threadIdx.x >> 1] && leaf_start[(key + 1) << sh] > leaf_start[key << sh];
        }
        __syncthreads();
        const long long hid0 = (1ll << l) + key0;
        for (int i = threadIdx.x; i < n * KP; i += SUB_T) {
            const int cell = i / KP, c = i - cell * KP;
            if (c >= K || !full[cur ^ 1][cell]) continue;
            const unsigned mc = mi[c];
            const int nn[3] = {px(mc), py(mc), pz(mc)};
            const double *f = fs[cell & 1];  // key0 is even: the cell's side is its low bit
            const double *Vp = vs[cur][cell >> 1];
            const int kn = nn[0] + nn[1] + nn[2];
            double acc = 0.0;
            for (int t = 0; t <= p - kn; ++t) {
                int m[3] = {nn[0], nn[1], nn[2]};
                m[sx] += t;
                acc += f[t] * Vp[midx(m[0], m[1], m[2]) - 1];
            }
            const double v = V[(hid0 + cell) * KP + c] + acc;
            V[(hid0 + cell) * KP + c] = v;
            vs[cur ^ 1][cell][c] = v;
        }
        cur ^= 1;
    }
}

__global__ void __launch_bounds__(SUB_T) k_l2l_sub(int p, int KP, int l0, int D, int L,
                                                   const Geom *g, const int *leaf_start, double *V)
{
    l2l_sub_body(p, KP, l0, D, L, g, leaf_start, V, blockIdx.x);
}

__global__ void __launch_bounds__(SUB_T) k_l2l_batch(const L2LArgs *a, const int *bstart, int nm)
{
    int r;
    const L2LArgs &x = a[batch_member(bstart, nm, blockIdx.x, r)];
    l2l_sub_body(x.p, x.KP, x.l0, x.D, x.L, x.g, x.leaf_start, x.V, r);
}

void launch_l2l_all(int p, int KP, int L, const Geom *d_geom, const int *leaf_start, double *V,
                    cudaStream_t s)
{
    int l0[LCAP + 1], D[LCAP + 1];
    const int n = l2l_rounds(L, l0, D);
    for (int r = 0; r < n; ++r) {
        note_launch();
        k_l2l_sub<<<(unsigned)(1ll << l0[r]), SUB_T, 0, s>>>(p, KP, l0[r], D[r], L, d_geom,
                                                              leaf_start, V);
    }
}

void launch_l2l_batch(const L2LArgs *a, const int *bstart, int nm, int nblocks, cudaStream_t s)
{
    if (nblocks <= 0) return;
    note_launch();
    k_l2l_batch<<<(unsigned)nblocks, SUB_T, 0, s>>>(a, bstart, nm);
}

#define INST(real)                                                                              \
    template void launch_dtables<real>(int, const int *, const uint16_t *, const double *,      \
                                       const double4 *, int, real *, int, cudaStream_t);        \
    template void launch_p2m<real>(int, int, int, const int *, const vec4<real>::t *,           \
                                   const vec2<real>::t *, real *, cudaStream_t);                \
    template void launch_m2m_all<real>(int, int, int, const Geom *, real *, cudaStream_t);      \
    template void launch_ap2m<real>(int, int, int, const int *, const int *, const int *,       \
                                    const vec4<real>::t *, const vec2<real>::t *, real *,       \
                                    cudaStream_t);                                              \

INST(float)
INST(double)
#undef INST

}  // namespace ccfmm
