// m2l.cu -- M2L (Eq. taylorcalc) as offset-grouped dense contractions.
// (The adaptive tree's tensor-core item bodies and the moment fold are in
// stages.cuh; their kernels are here.)
//
// V_n = (-1)^|n| sum_k D_{n+k}(c) Q_k, c = field-cell centre - partner centre,
// 1 <= |n|, |k| <= p: the square truncation, or, on request, only the terms
// with |n|+|k| <= maxdeg (the index table maps the dropped pairs to a zero
// column, and each warp stops at the last moment column its rows can meet).  All cells of a level are congruent,
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
#include "stages.cuh"

#include <stdlib.h>
#include <string.h>

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
                                                int ldD, const uint16_t *it, int maxdeg,
                                                const Geom *g, double *V)
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
    // moment columns this warp's rows 8w.. can meet (warp-uniform)
    const int kend = m2l_kend(p, maxdeg, 8 * warp);
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
    // gk and en are read across warps; a tile may have no entries, in which
    // case the entry loop (and its barriers) does not run
    __syncthreads();
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
            const int kc = min(KC, kend - k0);
#pragma unroll 4
            for (int kk = 0; kk < kc; ++kk) {
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
        long long hid = (1ll << t.level) + t.keys[ti];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            int n = 8 * warp + j;
            if (n < K) V[hid * KP + n] = (double)acc[i][j] * en[n];
        }
    }
}

// ---------------------------------------------------------------------------
// FP32 M2L with split work and asynchronous operand staging.
//
// A work item is (tile, a run of at most M2L_EC consecutive entries of that
// tile); items write FP32 partial sums Ps[item][t][n] that m2l_reduce adds in
// FP64, in item order, into V.  Per entry the partners' moment rows are
// copied with cp.async into a row-major buffer Qr[t][k] (row stride KP+4
// floats: 16-byte aligned rows whose 16-byte reads by consecutive cells fall
// in distinct banks) while the previous entry is being multiplied; M is
// rebuilt in shared memory from the entry's D row, M[k][n] = D~_{n+k} h^(1-|k|).
// Thread (warp w, lane): cells lane + 32i (i < 4) x coefficients 8w..8w+7.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void cp_async16(void *smem, const void *gmem, int bytes)
{
    unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(s), "l"(gmem), "r"(bytes));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N> __device__ __forceinline__ void cp_async_wait()
{
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N));
}

template <int KP>
__global__ void __launch_bounds__(KP * 4) k_m2l_f32(int p, const Tile *tiles, const M2LItem *items,
                                                    const int *ent_u, const int *ent_src,
                                                    const float *Q, const float *D, int ldD,
                                                    const uint16_t *it_g, int maxdeg,
                                                    const Geom *g, float *Ps)
{
    constexpr int RS = KP + 4;               // Qr row stride (floats)
    constexpr int NT = KP * 4;               // threads
    constexpr int CHQ = KP / 4;              // 16-byte chunks per moment row
    extern __shared__ __align__(16) unsigned char smraw[];
    float *Qr = reinterpret_cast<float *>(smraw);          // [2][TT][RS]
    float *Ms = Qr + 2 * TT * RS;                           // [KP][KP]
    float *Db = Ms + KP * KP;                               // [2][ldD]
    float *gk = Db + 2 * ldD;                               // [KP]
    uint16_t *its = reinterpret_cast<uint16_t *>(gk + KP);  // [KP*KP]

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const M2LItem item = items[blockIdx.x];
    const Tile t = tiles[item.tile];
    const int K = nterms(p) - 1;
    // moment columns this warp's rows 8w.. can meet, in whole float4 steps
    const int kend4 = min(KP, (m2l_kend(p, maxdeg, 8 * warp) + 3) & ~3);
    const double h = g->h[t.level];
    for (int c = tid; c < KP; c += NT) {
        double gv = 0.0;
        if (c < K) {
            int nx, ny, nz;
            midx_inv(c + 1, nx, ny, nz);
            gv = pow(h, (double)(1 - (nx + ny + nz)));
        }
        gk[c] = (float)gv;
    }
    for (int i = tid; i < KP * KP; i += NT) its[i] = it_g[i];

    auto issue = [&](int row, int buf) {
        float *dq = Qr + buf * TT * RS;
        const int *srow = ent_src + (long long)row * TT;
        for (int i = tid; i < TT * CHQ; i += NT) {
            int ti = i / CHQ, ch = i - ti * CHQ;
            int sr = srow[ti];
            const float *src = sr >= 0 ? Q + (long long)sr * KP + 4 * ch : Q;
            cp_async16(dq + ti * RS + 4 * ch, src, sr >= 0 ? 16 : 0);
        }
        const float *drow = D + (long long)ent_u[row] * ldD;
        float *dd = Db + buf * ldD;
        for (int i = tid; i < ldD / 4; i += NT) cp_async16(dd + 4 * i, drow + 4 * i, 16);
        cp_async_commit();
    };

    float acc[4][8];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[i][j] = 0.f;

    const int ne = item.e1 - item.e0;
    if (ne > 0) issue(item.e0, 0);
    for (int e = 0; e < ne; ++e) {
        const int buf = e & 1;
        if (e + 1 < ne) {
            issue(item.e0 + e + 1, buf ^ 1);
            cp_async_wait<1>();
        } else {
            cp_async_wait<0>();
        }
        __syncthreads();
        const float *Dl = Db + buf * ldD;
        for (int i = tid; i < KP * KP; i += NT) {
            int kk = i / KP;
            Ms[i] = Dl[its[i]] * gk[kk];
        }
        __syncthreads();
        const float *q0 = Qr + buf * TT * RS + lane * RS;
#pragma unroll 2
        for (int k4 = 0; k4 < kend4; k4 += 4) {
            float4 qv[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) qv[i] = *reinterpret_cast<const float4 *>(q0 + 32 * i * RS + k4);
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const float *mr = Ms + (k4 + j) * KP + 8 * warp;
                float4 m0 = *reinterpret_cast<const float4 *>(mr);
                float4 m1 = *reinterpret_cast<const float4 *>(mr + 4);
                float mm[8] = {m0.x, m0.y, m0.z, m0.w, m1.x, m1.y, m1.z, m1.w};
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    float qj = j == 0 ? qv[i].x : (j == 1 ? qv[i].y : (j == 2 ? qv[i].z : qv[i].w));
#pragma unroll
                    for (int c = 0; c < 8; ++c) acc[i][c] += qj * mm[c];
                }
            }
        }
        __syncthreads();
    }
    float *out = Ps + (long long)blockIdx.x * TT * KP;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        float *o = out + (lane + 32 * i) * KP + 8 * warp;
        *reinterpret_cast<float4 *>(o) = make_float4(acc[i][0], acc[i][1], acc[i][2], acc[i][3]);
        *reinterpret_cast<float4 *>(o + 4) = make_float4(acc[i][4], acc[i][5], acc[i][6], acc[i][7]);
    }
}

// V_n of each field cell = (-1)^|n| h^-(|n|+2) * sum over the tile's items
// of the partial sums, in FP64 and in item order.  A tile's outputs are
// split over RED_SPLIT blocks (blockIdx.y); each block forms the scale
// en[n] = (-1)^|n| h^-(|n|+2) by repeated multiplication with 1/h (FP64
// pow and division are slow on this part: one division per block).
constexpr int RED_SPLIT = 4;

__device__ __forceinline__ void m2l_reduce_body(int p, int KP, const Tile *tiles,
                                                const int *tile_item0, const int *tile_nitems,
                                                const float *Ps, const Geom *g, double *V,
                                                int tile)
{
    extern __shared__ double en[];
    const Tile t = tiles[tile];
    const int K = nterms(p) - 1;
    const double hinv = 1.0 / g->h[t.level];
    for (int n = threadIdx.x; n < K; n += blockDim.x) {
        int nx, ny, nz;
        midx_inv(n + 1, nx, ny, nz);
        const int kn = nx + ny + nz;
        double q = hinv * hinv;
        for (int d = 0; d < kn; ++d) q *= hinv;
        en[n] = (kn & 1) ? -q : q;
    }
    __syncthreads();
    const int i0 = tile_item0[tile], ni = tile_nitems[tile];
    for (int j = blockIdx.y * blockDim.x + threadIdx.x; j < t.nt * K;
         j += gridDim.y * blockDim.x) {
        int ti = j / K, n = j - ti * K;
        double s = 0.0;
        for (int it = 0; it < ni; ++it) s += (double)Ps[((long long)(i0 + it) * TT + ti) * KP + n];
        long long hid = (1ll << t.level) + t.keys[ti];
        V[hid * KP + n] = s * en[n];
    }
}

__global__ void k_m2l_reduce(int p, int KP, const Tile *tiles, const int *tile_item0,
                             const int *tile_nitems, const float *Ps, const Geom *g, double *V)
{
    m2l_reduce_body(p, KP, tiles, tile_item0, tile_nitems, Ps, g, V, blockIdx.x);
}

// every member's tiles in one launch (ensemble step)
__global__ void k_m2l_reduce_batch(const ReduceArgs *a, const int *bstart, int nm)
{
    int tile;
    const ReduceArgs &x = a[batch_member(bstart, nm, blockIdx.x, tile)];
    m2l_reduce_body(x.p, x.KP, x.tiles, x.tile_item0, x.tile_nitems, x.Ps, x.g, x.V, tile);
}

void launch_reduce_batch(int p, const ReduceArgs *a, const int *bstart, int nm, int nblocks,
                         cudaStream_t s)
{
    if (nblocks <= 0) return;
    note_launch();
    k_m2l_reduce_batch<<<dim3((unsigned)nblocks, RED_SPLIT), 256,
                         sizeof(double) * (nterms(p) - 1), s>>>(a, bstart, nm);
}

size_t m2l_f32_smem(int KP, int ldD)
{
    return sizeof(float) * ((size_t)2 * TT * (KP + 4) + (size_t)KP * KP + 2 * ldD + KP) +
           sizeof(uint16_t) * (size_t)KP * KP + 64;
}

bool m2l_f32_supported(int KP, int ldD)
{
    return (KP == 8 || KP == 16 || KP == 24 || KP == 40 || KP == 56 || KP == 88 || KP == 120) &&
           m2l_f32_smem(KP, ldD) <= 227 * 1024;
}

void launch_m2l_f32(int p, int KP, const Tile *tiles, int ntiles, const M2LItem *items,
                    int nitems, const int *tile_item0, const int *tile_nitems, const int *ent_u,
                    const int *ent_src, const float *Q, const float *D, int ldD,
                    const uint16_t *it, int maxdeg, const Geom *g, float *Ps, double *V,
                    cudaStream_t s)
{
    if (nitems > 0) {
        size_t smem = m2l_f32_smem(KP, ldD);
#define M2LF(KPV)                                                                               \
    case KPV:                                                                                   \
        cudaFuncSetAttribute(k_m2l_f32<KPV>, cudaFuncAttributeMaxDynamicSharedMemorySize,      \
                             (int)smem);                                                        \
        note_launch();                                                                          \
        k_m2l_f32<KPV><<<nitems, KPV * 4, smem, s>>>(p, tiles, items, ent_u, ent_src, Q, D,    \
                                                     ldD, it, maxdeg, g, Ps);                   \
        break;
        switch (KP) {
            M2LF(8) M2LF(16) M2LF(24) M2LF(40) M2LF(56) M2LF(88) M2LF(120)
        default: break;
        }
#undef M2LF
    }
    launch_m2l_reduce(p, KP, tiles, ntiles, tile_item0, tile_nitems, Ps, g, V, s);
}

void launch_m2l_reduce(int p, int KP, const Tile *tiles, int ntiles, const int *tile_item0,
                       const int *tile_nitems, const float *Ps, const Geom *g, double *V,
                       cudaStream_t s)
{
    if (ntiles <= 0) return;
    note_launch();
    k_m2l_reduce<<<dim3((unsigned)ntiles, RED_SPLIT), 256, sizeof(double) * (nterms(p) - 1), s>>>(
        p, KP, tiles, tile_item0, tile_nitems, Ps, g, V);
}

template <typename real, int KP, int KC>
static void run_m2l(int p, const Tile *tiles, int ntiles, const int *ent_u, const int *ent_src,
                    const real *Q, const real *D, int ldD, const uint16_t *it, int maxdeg,
                    const Geom *g, double *V, cudaStream_t s)
{
    size_t smem = sizeof(real) * ((size_t)KC * TT + (size_t)KC * KP + ldD + KP + (KP & 1)) +
                  sizeof(double) * KP + sizeof(int) * TT + 64;
    auto kern = k_m2l<real, KP, KC>;
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    note_launch();
    kern<<<ntiles, KP * 4, smem, s>>>(p, tiles, ent_u, ent_src, Q, D, ldD, it, maxdeg, g, V);
}

template <typename real>
void launch_m2l(int p, int KP, const Tile *tiles, int ntiles, const int *ent_u,
                const int *ent_src, const real *Q, const real *D, int ldD, const uint16_t *it,
                int maxdeg, const Geom *d_geom, double *V, cudaStream_t s)
{
    if (ntiles <= 0) return;
    const bool dbl = sizeof(real) == 8;
    switch (KP) {
    case 8: run_m2l<real, 8, 8>(p, tiles, ntiles, ent_u, ent_src, Q, D, ldD, it, maxdeg, d_geom, V, s); break;
    case 16: run_m2l<real, 16, 16>(p, tiles, ntiles, ent_u, ent_src, Q, D, ldD, it, maxdeg, d_geom, V, s); break;
    case 24: run_m2l<real, 24, 24>(p, tiles, ntiles, ent_u, ent_src, Q, D, ldD, it, maxdeg, d_geom, V, s); break;
    case 40: run_m2l<real, 40, 40>(p, tiles, ntiles, ent_u, ent_src, Q, D, ldD, it, maxdeg, d_geom, V, s); break;
    case 56: run_m2l<real, 56, 56>(p, tiles, ntiles, ent_u, ent_src, Q, D, ldD, it, maxdeg, d_geom, V, s); break;
    case 88: run_m2l<real, 88, 88>(p, tiles, ntiles, ent_u, ent_src, Q, D, ldD, it, maxdeg, d_geom, V, s); break;
    case 120:
        if (dbl) run_m2l<real, 120, 40>(p, tiles, ntiles, ent_u, ent_src, Q, D, ldD, it, maxdeg, d_geom, V, s);
        else run_m2l<real, 120, 120>(p, tiles, ntiles, ent_u, ent_src, Q, D, ldD, it, maxdeg, d_geom, V, s);
        break;
    case 168:
        if (dbl) run_m2l<real, 168, 56>(p, tiles, ntiles, ent_u, ent_src, Q, D, ldD, it, maxdeg, d_geom, V, s);
        else run_m2l<real, 168, 168>(p, tiles, ntiles, ent_u, ent_src, Q, D, ldD, it, maxdeg, d_geom, V, s);
        break;
    default: break;
    }
}

// ---------------------------------------------------------------------------
// M2L of the adaptive-depth tree, grouped by derivative tensor.  The far
// pairs (target cell, source cell) are sorted so that pairs with the same
// separation c = target centre - source centre (one D row) are contiguous;
// a work item is a run of pairs of one such group, (first pair, count, D
// row).  Per item the block forms M[k][n] = D~_{n+k} (once, when the
// coefficient columns fit one chunk) and then, for AP pairs at a time,
//     acc[pair][n] = sum_k M[k][n] Qs[k][pair],   Qs[k] = rho^-|k| Q_k(source),
// with D~ = D(c / rho), rho = |c| (the D row is computed at the unit vector,
// so every operand is O(1) for any pair of levels); the epilogue applies
// (-1)^|n| rho^-(|n|+1) and adds the result to the target's accumulator VF
// with vector atomics (FP32) or FP64 atomics: the order of the additions
// into one target is not fixed.  The powers of 1/rho are formed once per
// item by repeated multiplication (FP64, then rounded for FP32 operands).
// Thread layout: pair group pg (4 pairs) x column group ng (8 columns), so
// each thread keeps a 4 x 8 accumulator tile; columns are consumed in chunks
// of KC.
// ---------------------------------------------------------------------------
template <typename real> __device__ __forceinline__ void vf_add8(real *dst, const real (&o)[8]);
template <> __device__ __forceinline__ void vf_add8<float>(float *dst, const float (&o)[8])
{
    asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(dst), "f"(o[0]), "f"(o[1]),
                 "f"(o[2]), "f"(o[3])
                 : "memory");
    asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(dst + 4), "f"(o[4]),
                 "f"(o[5]), "f"(o[6]), "f"(o[7])
                 : "memory");
}
template <> __device__ __forceinline__ void vf_add8<double>(double *dst, const double (&o)[8])
{
#pragma unroll
    for (int j = 0; j < 8; ++j) atomicAdd(dst + j, o[j]);
}

template <typename real, int AP> struct am2l_shape {
    static constexpr int QSTR = AP + (sizeof(real) == 4 ? 4 : 2);  // Qs row stride
};

template <typename real, int KP, int AP, int KC>
__global__ void __launch_bounds__(((KP / 8) * (AP / 4) + 31) / 32 * 32)
    k_am2l(int p, const int4 *items, const int *pt, const int *ps, const double4 *sep,
           const real *D, int ldD, const uint16_t *it, int maxdeg, const real *Q, real *VF)
{
    constexpr int NG = KP / 8, PG = AP / 4, NT = NG * PG;
    constexpr int QSTR = am2l_shape<real, AP>::QSTR;
    extern __shared__ __align__(16) unsigned char smraw[];
    real *Ms = reinterpret_cast<real *>(smraw);  // [KC][KP]
    real *Qs = Ms + KC * KP;                     // [KC][QSTR]
    real *Dl = Qs + KC * QSTR;                   // [ldD]
    real *gk = Dl + ldD;                         // [KP] rho^-|k|
    real *en = gk + KP;                          // [KP] (-1)^|n| rho^-(|n|+1)
    real *pw = en + KP;                          // [PMAX + 4] rho^-d
    int *tg = reinterpret_cast<int *>(pw + PMAX + 4);  // [AP]
    int *sr = tg + AP;                                 // [AP]

    const int4 item = items[blockIdx.x];
    const int tid = threadIdx.x;
    const int K = nterms(p) - 1;
    if (tid == 0) {
        const double ri = 1.0 / sep[item.z].w;
        double v = 1.0;
        for (int d = 0; d <= p + 1; ++d) {
            pw[d] = (real)v;
            v *= ri;
        }
    }
    const real *Drow = D + (long long)item.z * ldD;
    for (int i = tid; i < ldD; i += blockDim.x) Dl[i] = Drow[i];
    __syncthreads();
    for (int c = tid; c < KP; c += blockDim.x) {
        real gv = (real)0, ev = (real)0;
        if (c < K) {
            int d = 1;
            while (nterms(d) <= c + 1) ++d;  // degree of multi-index c + 1
            gv = pw[d];
            ev = (d & 1) ? -pw[d + 1] : pw[d + 1];
        }
        gk[c] = gv;
        en[c] = ev;
    }
    const int pg = tid % PG, ng = tid / PG;
    const bool act = tid < NT;
    const int kend = act ? m2l_kend(p, maxdeg, 8 * ng) : 0;
    constexpr bool ONE = KC >= KP;  // M built once per item
    if (ONE) {
        for (int idx = tid; idx < KP * KP; idx += blockDim.x) Ms[idx] = Dl[it[idx]];
    }
    for (int c0 = 0; c0 < item.y; c0 += AP) {
        const int cnt = min(AP, item.y - c0);
        __syncthreads();  // scale tables and M ready; the previous chunk's reads done
        for (int i = tid; i < AP; i += blockDim.x) {
            const bool v = i < cnt;
            tg[i] = v ? pt[item.x + c0 + i] : -1;
            sr[i] = v ? ps[item.x + c0 + i] : -1;
        }
        __syncthreads();
        real acc[4][8];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 8; ++j) acc[i][j] = (real)0;
        for (int k0 = 0; k0 < KP; k0 += KC) {
            if (k0) __syncthreads();
            // moments of the chunk's sources, a row per pair read along k
            for (int idx = tid; idx < KC * AP; idx += blockDim.x) {
                const int i = idx / KC, kk = idx - i * KC, col = k0 + kk;
                const int sidx = sr[i];
                real v = (real)0;
                if (sidx >= 0 && col < K) v = Q[(long long)sidx * KP + col] * gk[col];
                Qs[kk * QSTR + i] = v;
            }
            if (!ONE)
                for (int idx = tid; idx < KC * KP; idx += blockDim.x) {
                    const int kk = idx / KP, n = idx - kk * KP;
                    Ms[idx] = (k0 + kk < KP) ? Dl[it[(k0 + kk) * KP + n]] : (real)0;
                }
            __syncthreads();
            if (act) {
                const int kc = min(KC, kend - k0);
                const real *Mk = ONE ? Ms + k0 * KP : Ms;
#pragma unroll 4
                for (int kk = 0; kk < kc; ++kk) {
                    real q[4], m0[4], m1[4];
                    v4<real>::ld(Qs + kk * QSTR + 4 * pg, q);
                    v4<real>::ld(Mk + kk * KP + 8 * ng, m0);
                    v4<real>::ld(Mk + kk * KP + 8 * ng + 4, m1);
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
        if (act) {
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const int t = tg[4 * pg + i];
                if (t < 0) continue;
                real o[8];
#pragma unroll
                for (int j = 0; j < 8; ++j) o[j] = acc[i][j] * en[8 * ng + j];
                vf_add8<real>(VF + (long long)t * KP + 8 * ng, o);
            }
        }
    }
}

template <typename real, int KP, int AP, int KC>
static void run_am2l(int p, const int4 *items, int nitems, const int *pt, const int *ps,
                     const double4 *sep, const real *D, int ldD, const uint16_t *it, int maxdeg,
                     const real *Q, real *VF, cudaStream_t s)
{
    constexpr int NT = ((KP / 8) * (AP / 4) + 31) / 32 * 32;
    const size_t smem = sizeof(real) * ((size_t)KC * KP + (size_t)KC * am2l_shape<real, AP>::QSTR +
                                        ldD + 2 * KP + PMAX + 4) +
                        sizeof(int) * 2 * AP + 64;
    auto kern = k_am2l<real, KP, AP, KC>;
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    note_launch();
    kern<<<(unsigned)nitems, NT, smem, s>>>(p, items, pt, ps, sep, D, ldD, it, maxdeg, Q, VF);
}

template <typename real, int AP>
static void am2l_dispatch(int p, int KP, const int4 *items, int nitems, const int *pt,
                          const int *ps, const double4 *sep, const real *D, int ldD,
                          const uint16_t *it, int maxdeg, const real *Q, real *VF, cudaStream_t s)
{
#define AM2L(KPV, KCV)                                                                           \
    case KPV:                                                                                    \
        run_am2l<real, KPV, AP, KCV>(p, items, nitems, pt, ps, sep, D, ldD, it, maxdeg, Q, VF, s); \
        break;
    switch (KP) {
        AM2L(8, 8) AM2L(16, 16) AM2L(24, 24) AM2L(40, 40) AM2L(56, 56) AM2L(88, 88)
        AM2L(120, 40) AM2L(168, 56)
    default: break;
    }
#undef AM2L
}

template <int KP>
__global__ void __launch_bounds__(128) k_am2l_mma_big(int p, const int4 *items, const int *pt,
                                                      const int *ps, const float *rpow,
                                                      const float *D, int ldD,
                                                      const uint16_t *it, const float *Q,
                                                      float *VF)
{
    extern __shared__ __align__(16) unsigned char smraw[];
    am2l_big_item<KP>(p, items[blockIdx.x], pt, ps, rpow, D, ldD, it, Q, VF, smraw);
}

template <int KP>
__global__ void __launch_bounds__(128) k_am2l_mma_small(int p, const int4 *items, int nitems,
                                                        const int *pt, const int *ps,
                                                        const float *rpow, const float *D,
                                                        int ldD, const uint16_t *it,
                                                        const float *Q, float *VF)
{
    extern __shared__ __align__(16) unsigned char smraw[];
    am2l_small_items<KP>(p, items, nitems, blockIdx.x, pt, ps, rpow, D, ldD, it, Q, VF, smraw);
}

template <int KP>
static void run_am2l_mma(int p, const int4 *items, int nitems, bool big, const int *pt,
                         const int *ps, const float *rpow, const float *D, int ldD,
                         const uint16_t *it, const float *Q, float *VF, cudaStream_t s)
{
    note_launch();
    if (big) {
        const size_t smem = am2l_big_smem<KP>(ldD);
        cudaFuncSetAttribute(k_am2l_mma_big<KP>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem);
        k_am2l_mma_big<KP><<<(unsigned)nitems, 128, smem, s>>>(p, items, pt, ps, rpow, D, ldD,
                                                                it, Q, VF);
    } else {
        const size_t smem = am2l_small_smem<KP>(ldD);
        cudaFuncSetAttribute(k_am2l_mma_small<KP>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem);
        k_am2l_mma_small<KP><<<(unsigned)((nitems + 3) / 4), 128, smem, s>>>(
            p, items, nitems, pt, ps, rpow, D, ldD, it, Q, VF);
    }
}

// the tensor-core form serves the FP32 path for p <= 6 (the split operator
// of one item fits shared memory) unless CCFMM_AM2L=fma
bool am2l_mma_ok(int p)
{
    static int env = -1;
    if (env < 0) {
        const char *e = getenv("CCFMM_AM2L");
        env = (e && strcmp(e, "fma") == 0) ? 0 : 1;
    }
    return env == 1 && p <= 6;
}

// folds every cell's moments (rows of KPF floats) into the reduced rows of
// KRP floats (zero padding), one warp per cell
constexpr int AF_W = 8;
__global__ void __launch_bounds__(32 * AF_W) k_afold(int p, int KPF, int KRP, int nc,
                                                     const float *Q, float *Qr)
{
    __shared__ float row[AF_W][AF_ROW];
    const int w = threadIdx.x >> 5;
    const long long c = (long long)blockIdx.x * AF_W + w;
    if (c >= nc) return;
    afold_cell(p, KPF, KRP, c, Q, Qr, row[w]);
}

// the reduced index table from the full one: itr[k][n] = it[full k][full n]
// (the zero column beyond the reduced count)
__global__ void k_itable_red(int p, int KPF, int KRP, const uint16_t *it, uint16_t *itr)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= KRP * KRP) return;
    const int k = j / KRP, n = j - k * KRP, KR = red_count(p);
    itr[j] = (k < KR && n < KR) ? it[red_full(k) * KPF + red_full(n)] : it[(KPF - 1) * KPF + KPF - 1];
}

void launch_afold(int p, int KPF, int KRP, int nc, const float *Q, float *Qr, cudaStream_t s)
{
    if (nc <= 0) return;
    note_launch();
    k_afold<<<(unsigned)((nc + AF_W - 1) / AF_W), 32 * AF_W, 0, s>>>(p, KPF, KRP, nc, Q, Qr);
}

void launch_itable_red(int p, int KPF, int KRP, const uint16_t *it, uint16_t *itr, cudaStream_t s)
{
    note_launch();
    k_itable_red<<<(KRP * KRP + 255) / 256, 256, 0, s>>>(p, KPF, KRP, it, itr);
}

// reduced contraction on the tensor cores (FP32): KRP the reduced width
void launch_am2l_red(int p, int KRP, const int4 *items, int nitems, int ap, const int *pt,
                     const int *ps, const float *rpow, const float *D, int ldD,
                     const uint16_t *itr, const float *Qr, float *VFr, cudaStream_t s)
{
    if (nitems <= 0) return;
    const bool big = ap == 64;
    switch (KRP) {
    case 8: run_am2l_mma<8>(p, items, nitems, big, pt, ps, rpow, D, ldD, itr, Qr, VFr, s); break;
    case 16: run_am2l_mma<16>(p, items, nitems, big, pt, ps, rpow, D, ldD, itr, Qr, VFr, s); break;
    case 24: run_am2l_mma<24>(p, items, nitems, big, pt, ps, rpow, D, ldD, itr, Qr, VFr, s); break;
    case 40: run_am2l_mma<40>(p, items, nitems, big, pt, ps, rpow, D, ldD, itr, Qr, VFr, s); break;
    case 48: run_am2l_mma<48>(p, items, nitems, big, pt, ps, rpow, D, ldD, itr, Qr, VFr, s); break;
    default: break;
    }
}

template <typename real>
void launch_am2l(int p, int KP, const int4 *items, int nitems, int ap, const int *pt,
                 const int *ps, const double4 *sep, const float *rpow, const real *D, int ldD,
                 const uint16_t *it, int maxdeg, const real *Q, real *VF, cudaStream_t s)
{
    (void)rpow;
    if (nitems <= 0) return;
    if (ap == 64)
        am2l_dispatch<real, 64>(p, KP, items, nitems, pt, ps, sep, D, ldD, it, maxdeg, Q, VF, s);
    else
        am2l_dispatch<real, 16>(p, KP, items, nitems, pt, ps, sep, D, ldD, it, maxdeg, Q, VF, s);
}

template void launch_am2l<float>(int, int, const int4 *, int, int, const int *, const int *,
                                 const double4 *, const float *, const float *, int,
                                 const uint16_t *, int, const float *, float *, cudaStream_t);
template void launch_am2l<double>(int, int, const int4 *, int, int, const int *, const int *,
                                  const double4 *, const float *, const double *, int,
                                  const uint16_t *, int, const double *, double *, cudaStream_t);

template void launch_m2l<float>(int, int, const Tile *, int, const int *, const int *,
                                const float *, const float *, int, const uint16_t *, int, const Geom *,
                                double *, cudaStream_t);
template void launch_m2l<double>(int, int, const Tile *, int, const int *, const int *,
                                 const double *, const double *, int, const uint16_t *,
                                 int, const Geom *, double *, cudaStream_t);

}  // namespace ccfmm
