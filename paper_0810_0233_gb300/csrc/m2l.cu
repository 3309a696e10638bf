// m2l.cu -- M2L (Eq. taylorcalc) as offset-grouped dense contractions.
//
// V_n = (-1)^|n| sum_k D_{n+k}(c) Q_k, c = field-cell centre - partner centre,
// square truncation 1 <= |n|, |k| <= p.  All cells of a level are congruent,
// so c = o * w_l for an integer offset o and D depends only on (level, o).
// A tile holds up to TT field cells of one level and one parity (keys
// 2(first+i)+parity); for every far offset present among them the tile has
// one entry: the offset's D row and the partner of each field cell (or -1).
// Per entry the block computes, for all TT cells at once,
//     acc[t][n] += sum_k M[n][k] * Qs[k][t],   M[n][k] = D~_{n+k},
//     Qs[k][t] = h^(1-|k|) Q_k(partner of t),
// with D~ = D(c/h) (h = cell radius of the level), i.e. operands scaled to
// O(1) so that FP32 neither overflows nor underflows; the epilogue applies
// (-1)^|n| h^-(|n|+2) in FP64 and stores V of each field cell in FP64.
// Thread layout: warp w owns coefficient rows 8w..8w+7, lane owns field
// cells 4*lane..4*lane+3, so each thread keeps a 4 x 8 accumulator tile.
#include "ccfmm_dev.cuh"

namespace ccfmm {

template <typename real> struct v4;
template <> struct v4<float> {
    static __device__ __forceinline__ void ld(const float *p, float o[4])
    {
        float4 v = *reinterpret_cast<const float4 *>(p);
        o[0] = v.x; o[1] = v.y; o[2] = v.z; o[3] = v.w;
    }
};
template <> struct v4<double> {
    static __device__ __forceinline__ void ld(const double *p, double o[4])
    {
        double2 a = *reinterpret_cast<const double2 *>(p);
        double2 b = *reinterpret_cast<const double2 *>(p + 2);
        o[0] = a.x; o[1] = a.y; o[2] = b.x; o[3] = b.y;
    }
};

template <typename real, int KP, int KC>
__global__ void __launch_bounds__(KP * 4) k_m2l(int p, const Tile *tiles, const int *ent_u,
                                                const int *ent_src, const real *Q, const real *D,
                                                int ldD, const uint16_t *it, const Geom *g,
                                                double *V)
{
    extern __shared__ __align__(16) unsigned char smraw[];
    real *Qs = reinterpret_cast<real *>(smraw);            // [KC][TT]
    real *Ms = Qs + KC * TT;                               // [KC][KP]
    real *Dl = Ms + KC * KP;                               // [ldD]
    real *gk = Dl + ldD;                                   // [KP]
    double *en = reinterpret_cast<double *>(gk + KP + (KP & 1));  // [KP]
    int *srcs = reinterpret_cast<int *>(en + KP);          // [TT]

    const int K = nterms(p) - 1;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const Tile t = tiles[blockIdx.x];
    const double h = g->h[t.level];
    for (int c = tid; c < KP; c += blockDim.x) {
        double gv = 0.0, ev = 0.0;
        if (c < K) {
            int nx, ny, nz;
            midx_inv(c + 1, nx, ny, nz);
            int kk = nx + ny + nz;
            gv = pow(h, (double)(1 - kk));
            ev = ((kk & 1) ? -1.0 : 1.0) * pow(h, -(double)(kk + 2));
        }
        gk[c] = (real)gv;
        en[c] = ev;
    }
    real acc[4][8];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[i][j] = (real)0;

    for (int e = 0; e < t.ent_count; ++e) {
        __syncthreads();
        const long long row = (long long)t.ent_start + e;
        for (int i = tid; i < TT; i += blockDim.x) srcs[i] = ent_src[row * TT + i];
        const real *Drow = D + (long long)ent_u[row] * ldD;
        for (int i = tid; i < ldD; i += blockDim.x) Dl[i] = Drow[i];
        __syncthreads();
        for (int k0 = 0; k0 < KP; k0 += KC) {
            if (k0) __syncthreads();
            for (int idx = tid; idx < KC * TT; idx += blockDim.x) {
                int kk = idx / TT, ti = idx - kk * TT, col = k0 + kk;
                int sr = srcs[ti];
                real v = (real)0;
                if (sr >= 0 && col < K) v = Q[(long long)sr * KP + col] * gk[col];
                Qs[idx] = v;
            }
            for (int idx = tid; idx < KC * KP; idx += blockDim.x) {
                int kk = idx / KP, n = idx - kk * KP;
                Ms[idx] = Dl[it[(k0 + kk) * KP + n]];
            }
            __syncthreads();
#pragma unroll 4
            for (int kk = 0; kk < KC; ++kk) {
                real q[4], m0[4], m1[4];
                v4<real>::ld(Qs + kk * TT + 4 * lane, q);
                v4<real>::ld(Ms + kk * KP + 8 * warp, m0);
                v4<real>::ld(Ms + kk * KP + 8 * warp + 4, m1);
#pragma unroll
                for (int i = 0; i < 4; ++i) {
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        acc[i][j] += q[i] * m0[j];
                        acc[i][4 + j] += q[i] * m1[j];
                    }
                }
            }
        }
    }
    // epilogue: V_n = (-1)^|n| h^-(|n|+2) acc_n, FP64, one writer per (cell, n)
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        int ti = 4 * lane + i;
        if (ti >= t.nt) continue;
        long long hid = (1ll << t.level) + 2ll * (t.first + ti) + t.parity;
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            int n = 8 * warp + j;
            if (n < K) V[hid * KP + n] = (double)acc[i][j] * en[n];
        }
    }
}

template <typename real, int KP, int KC>
static void run_m2l(int p, const Tile *tiles, int ntiles, const int *ent_u, const int *ent_src,
                    const real *Q, const real *D, int ldD, const uint16_t *it, const Geom *g,
                    double *V, cudaStream_t s)
{
    size_t smem = sizeof(real) * ((size_t)KC * TT + (size_t)KC * KP + ldD + KP + (KP & 1)) +
                  sizeof(double) * KP + sizeof(int) * TT + 64;
    auto kern = k_m2l<real, KP, KC>;
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    note_launch();
    kern<<<ntiles, KP * 4, smem, s>>>(p, tiles, ent_u, ent_src, Q, D, ldD, it, g, V);
}

template <typename real>
void launch_m2l(int p, int KP, const Tile *tiles, int ntiles, const int *ent_u,
                const int *ent_src, const real *Q, const real *D, int ldD, const uint16_t *it,
                const Geom *d_geom, double *V, cudaStream_t s)
{
    if (ntiles <= 0) return;
    const bool dbl = sizeof(real) == 8;
    switch (KP) {
    case 8: run_m2l<real, 8, 8>(p, tiles, ntiles, ent_u, ent_src, Q, D, ldD, it, d_geom, V, s); break;
    case 16: run_m2l<real, 16, 16>(p, tiles, ntiles, ent_u, ent_src, Q, D, ldD, it, d_geom, V, s); break;
    case 24: run_m2l<real, 24, 24>(p, tiles, ntiles, ent_u, ent_src, Q, D, ldD, it, d_geom, V, s); break;
    case 40: run_m2l<real, 40, 40>(p, tiles, ntiles, ent_u, ent_src, Q, D, ldD, it, d_geom, V, s); break;
    case 56: run_m2l<real, 56, 56>(p, tiles, ntiles, ent_u, ent_src, Q, D, ldD, it, d_geom, V, s); break;
    case 88: run_m2l<real, 88, 88>(p, tiles, ntiles, ent_u, ent_src, Q, D, ldD, it, d_geom, V, s); break;
    case 120:
        if (dbl) run_m2l<real, 120, 40>(p, tiles, ntiles, ent_u, ent_src, Q, D, ldD, it, d_geom, V, s);
        else run_m2l<real, 120, 120>(p, tiles, ntiles, ent_u, ent_src, Q, D, ldD, it, d_geom, V, s);
        break;
    case 168:
        if (dbl) run_m2l<real, 168, 56>(p, tiles, ntiles, ent_u, ent_src, Q, D, ldD, it, d_geom, V, s);
        else run_m2l<real, 168, 168>(p, tiles, ntiles, ent_u, ent_src, Q, D, ldD, it, d_geom, V, s);
        break;
    default: break;
    }
}

template void launch_m2l<float>(int, int, const Tile *, int, const int *, const int *,
                                const float *, const float *, int, const uint16_t *, const Geom *,
                                double *, cudaStream_t);
template void launch_m2l<double>(int, int, const Tile *, int, const int *, const int *,
                                 const double *, const double *, int, const uint16_t *,
                                 const Geom *, double *, cudaStream_t);

}  // namespace ccfmm
