// m2l_tc.cu -- M2L (Eq. taylorcalc) on the fifth-generation tensor cores.
//
// Work decomposition: the FP32 path's items (a tile of 128 same-parity field
// cells x a run of at most M2L_EC of its offset entries).  Per entry the
// contraction
//     acc[t][n] += sum_k  Qt_k(partner of t) * D~_{n+k}(offset),
//     Qt_k = Q_k h^(1-|k|)  (the level's scale carried by the moments),
// is a tcgen05 MMA with M = 128 cells, N = coefficients n (padded to a
// multiple of 16) and K = coefficients k (padded to chunks of 32),
// accumulated in tensor memory over all entries of the item.  FP32 accuracy
// from TF32 operands: x = x_hi + x_lo, x_hi = x rounded to TF32 (cvt.rna),
// x_lo = x - x_hi (exact), and A B ~ A_hi B_hi + A_hi B_lo + A_lo B_hi.
// Both operands are split outside the contraction loop: the scaled moments
// once per evaluation (k_q_split, hi and lo planes of rows of KT floats), the
// operators once per tree build (k_m2l_ops, one per far offset class),
// stored in exactly the shared-memory layout the MMA reads so that a unit's
// operator chunk is one bulk copy.  B_lo follows B_hi in shared memory, so
// one MMA of width 2N forms A_hi [B_hi | B_lo] (two accumulator halves,
// added in the epilogue) and a second of width N adds A_lo B_hi: A_hi is
// read once per k-step, which matters because at TF32 the MMAs' operand
// reads are what bounds shared-memory bandwidth.
//
// K is padded to chunks of 32; the k-steps of 8 that lie wholly beyond KP
// (the last chunk's padding) are skipped, and the gather copies none of
// their bytes.
//
// Shared-memory operands use the 128-byte-swizzled K-major layout: a unit's
// row of 32 TF32 is one 128-byte line, 8-row atoms of 1024 bytes (stride
// offset), and the 16-byte chunk j of row r sits in slot j ^ (r mod 8), so
// that the chunks of one row, and chunk j of eight rows, fall in different
// banks (the gather's shared-memory writes are conflict-free).  Stage bases
// are 1024-byte aligned; a k-step of 8 advances the start address by 32 B.
//
// Pipeline, 3 or 4 stages (as many as fit) of one unit = (entry, 32-wide K
// chunk) each.  Two ways to fill a stage:
//   TMA gather (CCFMM_TC_GATHER=tma; measured slower, not the default)
//              producer warp 0 alone: lane 0 posts the stage's
//              byte count on its barrier and starts the bulk copy of the
//              operator chunk; every lane gathers its 4 partner rows of the
//              hi and the lo plane with one tile::gather4 tensor copy each
//              (a 128-byte row per cell, written in the 128-byte-swizzled
//              layout by the copy engine; cells without that partner read
//              row 0, which holds zeros).  The barrier completes when all
//              bytes have landed, so all stages can be in flight;
//   cp.async gather  (the default) producers (4 or 8 warps) wait for
//              the stage to be free, gather the 128 partner rows of the
//              chunk (cp.async, hi and lo; zero rows for cells without that
//              partner), and thread 0 starts the bulk copy of the operator
//              chunk.  stages - 1 units later, before waiting for the next
//              free stage, each warp marks the unit's stage full once its
//              own copies have landed (one arrival per warp);
//   last warp  one thread issues the unit's 8 MMAs once the rows and the
//              operator chunk have landed and frees the stage with
//              tcgen05.commit;
//   producers  finally read the accumulator (tcgen05.ld; warp w reads TMEM
//              lanes 32 (w mod 4) ..) into the item's FP32 partial sums,
//              which k_m2l_reduce adds in FP64.
// Every wait is bounded; on time-out the kernel raises FLAG_TIMEOUT, lets
// its copies and MMAs finish (again bounded), frees its tensor memory and
// returns.
#include "ccfmm_dev.cuh"

#include <cuda.h>
#include <cudaTypedefs.h>
#include <stdlib.h>
#include <string.h>

namespace ccfmm {

constexpr int TC_M = 128;       // field cells per tile (MMA M = TMEM lanes)
constexpr int TC_KC = 32;       // K per unit: 4 MMA k-steps of 8
constexpr int TC_SMEM = 227 * 1024;
// at most this many pipeline stages (as many as fit, 2 at least; fewer
// stages leave room on the SM for a second CTA or near-field blocks)
#ifndef CCFMM_TC_MAXST
#define CCFMM_TC_MAXST 2
#endif
#ifndef CCFMM_TC_PROD
#define CCFMM_TC_PROD 256
#endif
constexpr int TC_PROD = CCFMM_TC_PROD;  // producer / epilogue threads (128 or 256)
static_assert(TC_PROD == 128 || TC_PROD == 256, "4 or 8 producer warps");
constexpr int TC_THREADS = TC_PROD + 32;
constexpr int TC_SBO = 1024;               // bytes between 8-row atoms
constexpr long long TC_SPIN = 1ll << 22;

template <int KP> struct TcShape {
    static constexpr int N = ((KP + 15) / 16) * 16;               // MMA N
    static constexpr int KT = ((KP + TC_KC - 1) / TC_KC) * TC_KC;  // padded K
    static constexpr int NCH = KT / TC_KC;                        // units per entry
    static constexpr int A_BYTES = TC_M * TC_KC * 4;
    static constexpr int B_BYTES = N * TC_KC * 4;
    static constexpr int STAGE = 2 * A_BYTES + 2 * B_BYTES;
    static constexpr int OP_BYTES = NCH * 2 * B_BYTES;            // one offset class
    // pipeline stages that fit (at most 4), and how many units a producer
    // keeps in flight before marking the oldest one full
    static constexpr int FIT = (TC_SMEM - 2048) / STAGE;
    static constexpr int ST = FIT < CCFMM_TC_MAXST ? (FIT < 2 ? 2 : FIT) : CCFMM_TC_MAXST;
    static constexpr int LAG = ST - 1;
    static constexpr int TMEM_COLS = 2 * N <= 64 ? 64 : (2 * N <= 128 ? 128 : 256);
};

// Harmonic reduction of the contraction.  D_m is a derivative of 1/r, so
// sum_a D_{m+2e_a} = 0 (Laplace): a moment Q_k with k_z >= 2 folds into
// Q_{k-2e_z+2e_x} and Q_{k-2e_z+2e_y} (with a minus sign) without changing
// any V_n, leaving per order k the 2k + 1 moments with k_z <= 1; and V_n
// with n_z >= 2 follows from V_{n-2e_z+2e_x} + V_{n-2e_z+2e_y} = -V_n by the
// same identity.  So the MMA contracts (p+1)^2 - 1 coefficients on either
// side instead of T(p) - 1 (48 instead of 83 at p = 6).  In the library's
// order the k_z <= 1 multi-indices are the first 2k + 1 of each order: the
// reduced column r of order k (k^2 - 1 <= r < (k+1)^2 - 1) is the full
// column T(k-1) - 1 + r - (k^2 - 1).  The kernels below are instantiated on
// the reduced width (padded to 8) of each full width KP.
constexpr int tc_red_kp(int KP)
{
    return KP == 40 ? 24 : KP == 56 ? 40 : KP == 88 ? 48 : KP == 120 ? 64 : 0;
}

__device__ __forceinline__ uint32_t smem_u32(const void *p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ uint64_t umma_desc(uint32_t saddr)
{
    uint64_t d = 0;
    d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
    d |= (uint64_t)1 << 16;                                    // leading offset (unused)
    d |= (uint64_t)(((uint32_t)TC_SBO >> 4) & 0x3FFFu) << 32;  // stride offset: 8-row atoms
    d |= (uint64_t)1 << 46;                                    // descriptor version (tcgen05)
    d |= (uint64_t)2 << 61;                                    // 128-byte swizzle
    return d;                                                  // base offset 0
}

// byte offset of (row r, 16-byte chunk j) in a 128-byte-swizzled operand
__host__ __device__ constexpr uint32_t sw128(int r, int j)
{
    return (uint32_t)((r >> 3) * 1024 + (r & 7) * 128 + ((j ^ (r & 7)) << 4));
}

__device__ __forceinline__ float to_tf32(float x)
{
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return __uint_as_float(r);
}

__device__ __forceinline__ void tc_cp16(uint32_t dst, const void *src, int bytes)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(dst), "l"(src), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void mbar_init(uint32_t a, int count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(a), "r"(count));
}

__device__ __forceinline__ void mbar_arrive(uint32_t a)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(a) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t a, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(a), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try(uint32_t a, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(a), "r"(parity)
        : "memory");
    return ok != 0;
}

// bounded wait (spin iterations); gives up early once another thread has
// given up
__device__ __forceinline__ bool mbar_wait(uint32_t a, uint32_t parity, volatile int *abort,
                                          long long spin)
{
    for (long long i = 0; i < spin; ++i) {
        if (mbar_try(a, parity)) return true;
        if ((i & 31) == 31 && *abort) return false;
    }
    return false;
}

// bounded wait used while tearing down after a time-out
__device__ __forceinline__ bool mbar_wait_plain(uint32_t a, uint32_t parity)
{
    for (long long i = 0; i < TC_SPIN; ++i)
        if (mbar_try(a, parity)) return true;
    return false;
}

__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void *src, uint32_t bytes,
                                         uint32_t bar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, "
        "[%3];" ::"r"(dst),
        "l"(src), "r"(bytes), "r"(bar)
        : "memory");
}

// four 128-byte rows (x = first column, rows r.x .. r.w) of a 2-D tensor
// into 512 consecutive bytes of shared memory, swizzled as the map says
__device__ __forceinline__ void tma_gather4(uint32_t dst, const void *map, int x, int4 r,
                                            uint32_t bar)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cta.global.tile::gather4.mbarrier::complete_tx::bytes "
        "[%0], [%1, {%2, %3, %4, %5, %6}], [%7];" ::"r"(dst),
        "l"(map), "r"(x), "r"(r.x), "r"(r.y), "r"(r.z), "r"(r.w), "r"(bar)
        : "memory");
}

__device__ __forceinline__ void tc_mma(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc,
                                       uint32_t acc)
{
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ void tc_commit(uint32_t bar)
{
    asm volatile(
        "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
        : "memory");
}

// ---------------------------------------------------------------- prologue
// gk[l][k] = h_l^(1-|k|) for the multi-index k+1 (k < K), zero beyond.
__global__ void k_tc_scale(int p, int KT, int L, const Geom *g, float *gk)
{
    const int l = blockIdx.x;
    const int KR = red_count(p);
    for (int k = threadIdx.x; k < KT; k += blockDim.x) {
        float v = 0.f;
        if (k < KR && l <= L) v = (float)pow(g->h[l], (double)(1 - red_order(k)));
        gk[l * KT + k] = v;
    }
}

// Operator chunks of every far offset class: for chunk c and part (hi, lo),
// the N x 32 block M[n][k] = D~_{n+k}, k = 32c + kl, in canonical layout.
template <int KP>
__global__ void k_m2l_ops(int p, int KPF, const float *D, int ldD, const uint16_t *it_g,
                          float *Bop)
{
    typedef TcShape<KP> S;
    extern __shared__ float Dl[];
    const int K = red_count(p);
    const long long gid = blockIdx.x;
    for (int i = threadIdx.x; i < ldD; i += blockDim.x) Dl[i] = D[gid * ldD + i];
    __syncthreads();
    float *out = Bop + gid * (S::OP_BYTES / 4);
    constexpr int PER = S::N * TC_KC;  // floats per (chunk, part)
    for (int o = threadIdx.x; o < S::NCH * PER; o += blockDim.x) {
        const int c = o / PER, q = o - c * PER;
        // float index q = (n>>3)*256 + (n&7)*32 + ((kl>>2) ^ (n&7))*4 + (kl&3)
        const int n = ((q >> 5) & 7) | ((q >> 8) << 3);
        const int kl = (q & 3) | ((((q >> 2) & 7) ^ (n & 7)) << 2);
        const int k = c * TC_KC + kl;
        const float v = (n < K && k < K) ? Dl[it_g[red_full(k) * KPF + red_full(n)]] : 0.f;
        const float hi = to_tf32(v);
        out[c * 2 * PER + q] = hi;
        out[c * 2 * PER + PER + q] = v - hi;
    }
}

// Scaled, folded moments split into TF32 pairs: Qs[part][hid][r], rows of
// KT floats over the reduced columns r (SPLIT), or the scaled FP32 values
// alone in plane 0 (the kernel that splits them in registers on the way to
// tensor memory).  One warp per cell: the full row into shared memory, lane
// k - 1 folds order k (k_z from high to low, in FP32), then the reduced
// columns are scaled by h^(1-|k|) and split.
constexpr int QF_W = 8;  // cells (warps) per block
constexpr int QF_ROW = ((nterms(PMAX) - 1 + 7) / 8) * 8;

template <int KP, bool SPLIT>
__device__ __forceinline__ void q_fold_body(int p, int KPF, long long ncell, const float *Q,
                                            const float *gk, float *Qs, long long blk)
{
    typedef TcShape<KP> S;
    constexpr int KT = S::KT;
    __shared__ float row[QF_W][QF_ROW];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const long long hid = blk * QF_W + w;
    if (hid >= ncell) return;
    const int K = nterms(p) - 1, KR = red_count(p);
    // heap id 0 is no cell: its row stays zero (the gather's empty partner)
    for (int c = lane; c < K; c += 32) row[w][c] = hid > 0 ? Q[hid * KPF + c] : 0.f;
    __syncwarp();
    if (lane >= 1 && lane < p) {
        const int k = lane + 1, base = nterms(k - 1) - 1;
        for (int z = k; z >= 2; --z)
            for (int y = 0; y <= k - z; ++y) {
                const int x = k - z - y;
                const float v = row[w][base + z * (2 * k + 3 - z) / 2 + y];
                const int zt = z - 2, lt = base + zt * (2 * k + 3 - zt) / 2;
                row[w][lt + y] -= v;       // (x + 2, y, z - 2)
                row[w][lt + y + 2] -= v;   // (x, y + 2, z - 2)
                (void)x;
            }
    }
    __syncwarp();
    const int level = hid > 0 ? 63 - __clzll(hid) : 0;
    for (int r = lane; r < KT; r += 32) {
        const float v = (r < KR && hid > 0) ? row[w][red_full(r)] * gk[level * KT + r] : 0.f;
        if (!SPLIT) {
            Qs[hid * KT + r] = v;
        } else {
            const float hi = to_tf32(v);
            Qs[hid * KT + r] = hi;
            Qs[(ncell + hid) * KT + r] = v - hi;
        }
    }
}

template <int KP, bool SPLIT>
__global__ void __launch_bounds__(32 * QF_W) k_q_fold(int p, int KPF, long long ncell,
                                                      const float *Q, const float *gk, float *Qs)
{
    q_fold_body<KP, SPLIT>(p, KPF, ncell, Q, gk, Qs, blockIdx.x);
}

template <int KP>
__global__ void __launch_bounds__(32 * QF_W) k_q_fold_batch(int KPF, const QSplitArgs *a,
                                                            const int *bstart, int nm)
{
    int blk;
    const QSplitArgs &x = a[batch_member(bstart, nm, blockIdx.x, blk)];
    q_fold_body<KP, true>(x.p, KPF, x.ncell, x.Q, x.gk, x.Qs, blk);
}

// V of each field cell from the tile's partial sums over the reduced
// columns: FP64 sums in item order times (-1)^|n| h^-(|n|+2), then the
// columns with n_z >= 2 by -V_{n-2e_z+2e_x} - V_{n-2e_z+2e_y} in the library's
// order (within an order by increasing n_z, so both are known).  A tile's
// cells are split over RED_H blocks (blockIdx.y), 128 / RED_H cells each.
constexpr int RED_H = 4, RED_HC = TT / RED_H;

__device__ __forceinline__ void m2l_reduce_h_body(int p, int KPF, int KRP, const Tile *tiles,
                                                  const int *tile_item0, const int *tile_nitems,
                                                  const float *Ps, const Geom *g, double *V,
                                                  int tile)
{
    extern __shared__ double smd[];
    const int K = nterms(p) - 1, KR = red_count(p);
    double *en = smd;              // [KR]
    double *rows = smd + KR;       // [RED_HC][K]
    // completion table: for full column c with n_z >= 2 its n_z and the full
    // columns of n - 2e_z + 2e_x and n - 2e_z + 2e_y
    __shared__ unsigned char cz[QF_ROW], cs1[QF_ROW], cs2[QF_ROW];
    const Tile t = tiles[tile];
    const double hinv = 1.0 / g->h[t.level];
    for (int r = threadIdx.x; r < KR; r += blockDim.x) {
        const int kn = red_order(r);
        double q = hinv * hinv;
        for (int d = 0; d < kn; ++d) q *= hinv;
        en[r] = (kn & 1) ? -q : q;
    }
    for (int c = threadIdx.x; c < K; c += blockDim.x) {
        int nx, ny, nz;
        midx_inv(c + 1, nx, ny, nz);
        cz[c] = (unsigned char)nz;
        cs1[c] = nz >= 2 ? (unsigned char)(midx(nx + 2, ny, nz - 2) - 1) : 0;
        cs2[c] = nz >= 2 ? (unsigned char)(midx(nx, ny + 2, nz - 2) - 1) : 0;
    }
    __syncthreads();
    const int i0 = tile_item0[tile], ni = tile_nitems[tile];
    const int tb = blockIdx.y * RED_HC;
    const int nc = min(RED_HC, t.nt - tb);
    for (int j = threadIdx.x; j < nc * KR; j += blockDim.x) {
        const int ci = j / KR, r = j - ci * KR;
        double s = 0.0;
        for (int it = 0; it < ni; ++it)
            s += (double)Ps[((long long)(i0 + it) * TT + tb + ci) * KRP + r];
        rows[ci * K + red_full(r)] = s * en[r];
    }
    __syncthreads();
    // columns with n_z = z from those with n_z = z - 2, z = 2 .. p in turn
    for (int z = 2; z <= p; ++z) {
        for (int j = threadIdx.x; j < nc * K; j += blockDim.x) {
            const int ci = j / K, c = j - ci * K;
            if (cz[c] != z) continue;
            double *v = rows + ci * K;
            v[c] = -v[cs1[c]] - v[cs2[c]];
        }
        __syncthreads();
    }
    for (int j = threadIdx.x; j < nc * K; j += blockDim.x) {
        const int ci = j / K, c = j - ci * K;
        const long long hid = (1ll << t.level) + t.keys[tb + ci];
        V[hid * KPF + c] = rows[j];
    }
}

__global__ void k_m2l_reduce_h(int p, int KPF, int KRP, const Tile *tiles, const int *tile_item0,
                               const int *tile_nitems, const float *Ps, const Geom *g, double *V)
{
    m2l_reduce_h_body(p, KPF, KRP, tiles, tile_item0, tile_nitems, Ps, g, V, blockIdx.x);
}

__global__ void k_m2l_reduce_h_batch(int KRP, const ReduceArgs *a, const int *bstart, int nm)
{
    int tile;
    const ReduceArgs &x = a[batch_member(bstart, nm, blockIdx.x, tile)];
    m2l_reduce_h_body(x.p, x.KP, KRP, x.tiles, x.tile_item0, x.tile_nitems, x.Ps, x.g, x.V, tile);
}

static size_t reduce_h_smem(int p)
{
    return sizeof(double) * ((size_t)red_count(p) + (size_t)RED_HC * (nterms(p) - 1));
}

void launch_reduce_h(int p, int KPF, const Tile *tiles, int ntiles, const int *tile_item0,
                     const int *tile_nitems, const float *Ps, const Geom *g, double *V,
                     cudaStream_t s)
{
    if (ntiles <= 0) return;
    const size_t smem = reduce_h_smem(p);
    cudaFuncSetAttribute(k_m2l_reduce_h, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    note_launch();
    k_m2l_reduce_h<<<dim3((unsigned)ntiles, RED_H), 256, smem, s>>>(
        p, KPF, tc_red_kp(KPF), tiles, tile_item0, tile_nitems, Ps, g, V);
}

void launch_reduce_h_batch(int p, int KPF, const ReduceArgs *a, const int *bstart, int nm,
                           int nblocks, cudaStream_t s)
{
    if (nblocks <= 0) return;
    const size_t smem = reduce_h_smem(p);
    cudaFuncSetAttribute(k_m2l_reduce_h_batch, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)smem);
    note_launch();
    k_m2l_reduce_h_batch<<<dim3((unsigned)nblocks, RED_H), 256, smem, s>>>(tc_red_kp(KPF), a,
                                                                           bstart, nm);
}

// 16 consecutive accumulator columns of this warp's 32 TMEM lanes
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&r)[16])
{
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,"
        "%14,%15}, [%16];\n"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
          "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
}

// ------------------------------------------------------------ contraction
template <int KP, bool TMA>
__device__ __forceinline__ void m2l_tc_body(const M2LItem *items, const int *ent_u,
                                            const int *ent_src, const float *Qs, long long qplane,
                                            const CUtensorMap *qmap, int ncell,
                                            const unsigned char *Bop, float *Ps, int *flags,
                                            long long spin, int stall, int itx)
{
    typedef TcShape<KP> S;
    extern __shared__ __align__(1024) unsigned char smraw[];
    constexpr int TC_ST = S::ST;
    __shared__ __align__(8) unsigned long long bar_full[TC_ST], bar_b[TC_ST], bar_empty[TC_ST];
    __shared__ __align__(8) unsigned long long bar_done;
    __shared__ uint32_t tmem_slot;
    __shared__ int s_abort;
    volatile int *abort = &s_abort;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const M2LItem item = items[itx];
    const int ne = item.e1 - item.e0;
    const int nunits = ne * S::NCH;
    const uint32_t sbase = (smem_u32(smraw) + 1023u) & ~1023u;  // swizzle atoms
    const uint32_t done = smem_u32(&bar_done);

    if (tid == 0) {
        *abort = 0;
        for (int s = 0; s < TC_ST; ++s) {
            mbar_init(smem_u32(&bar_full[s]), TC_PROD / 32);
            mbar_init(smem_u32(&bar_b[s]), 1);
            mbar_init(smem_u32(&bar_empty[s]), 1);
        }
        mbar_init(done, 1);
        asm volatile("fence.mbarrier_init.release.cluster;");
    }
    constexpr int MMA_WARP = TC_PROD / 32;
    if (warp == MMA_WARP) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(&tmem_slot)),
                     "r"(S::TMEM_COLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tmem = tmem_slot;

    if (warp < MMA_WARP) {
        int issued = 0;
        bool ok = true;
        if constexpr (TMA) {
            // ---------------- producer warp 0: lane l gathers rows 4l .. 4l+3
            // of the tile (hi and lo plane, one tile::gather4 copy each);
            // lane 0 posts the stage's bytes and copies the operator chunk
            if (warp == 0) {
                int4 rw = make_int4(0, 0, 0, 0), rwn = rw;
                int gid = 0, gidn = 0;
                if (ne > 0) {
                    rwn = *reinterpret_cast<const int4 *>(ent_src + (long long)item.e0 * TT +
                                                           4 * lane);
                    if (lane == 0) gidn = ent_u[item.e0];
                }
                const uint32_t dsta = (uint32_t)(4 * lane) * 128u;  // 4 rows, linear
                for (int u = 0; u < nunits; ++u) {
                    const int s = u % TC_ST, r = u / TC_ST;
                    const int e = u / S::NCH, c = u - e * S::NCH;
                    if (c == 0) {
                        rw = rwn;
                        gid = gidn;
                        if (e + 1 < ne) {
                            const long long nrow = (long long)item.e0 + e + 1;
                            rwn = *reinterpret_cast<const int4 *>(ent_src + nrow * TT + 4 * lane);
                            if (lane == 0) gidn = ent_u[nrow];
                        }
                    }
                    if (r > 0 && !__all_sync(0xffffffffu, mbar_wait(smem_u32(&bar_empty[s]),
                                                                    (r - 1) & 1, abort, spin))) {
                        ok = false;
                        break;
                    }
                    const uint32_t st = sbase + (uint32_t)(s * S::STAGE);
                    const uint32_t bb = smem_u32(&bar_b[s]);
                    if (lane == 0) {
                        mbar_expect_tx(bb, S::STAGE);
                        bulk_g2s(st + 2 * S::A_BYTES,
                                 Bop + ((long long)gid * S::NCH + c) * (2 * S::B_BYTES),
                                 2 * S::B_BYTES, bb);
                    }
                    __syncwarp();
                    // a cell without this partner reads row 0 (zeros)
                    const int4 q = make_int4(rw.x >= 0 ? rw.x : 0, rw.y >= 0 ? rw.y : 0,
                                             rw.z >= 0 ? rw.z : 0, rw.w >= 0 ? rw.w : 0);
                    tma_gather4(st + dsta, qmap, c * TC_KC, q, bb);
                    tma_gather4(st + S::A_BYTES + dsta, qmap, c * TC_KC,
                                make_int4(q.x + ncell, q.y + ncell, q.z + ncell, q.w + ncell), bb);
                    issued = u + 1;
                }
            }
        } else {
            // ---------------- producers: a warp instruction copies 4 whole unit
            // rows (128 B each, one global line and one shared line): lane ->
            // (row r = 4 (warp + NW m) + lane / 8, 16-byte chunk j = lane mod 8)
            constexpr int NW = TC_PROD / 32, MR = 32 / NW;
            const int j = lane & 7, rq = lane >> 3;
            const uint32_t dst0 = sw128(4 * warp + rq, j);  // + m NW/2 atoms
            auto rowof = [&](int m) { return 4 * (warp + NW * m) + rq; };
            // partner rows and operator class of the current entry, and of the
            // next one, loaded an entry ahead so that no gather waits on them
            int src[MR], srcn[MR], gid = 0, gidn = 0;
            if (ne > 0) {
                const int *sr = ent_src + (long long)item.e0 * TT;
#pragma unroll
                for (int m = 0; m < MR; ++m) srcn[m] = sr[rowof(m)];
                if (tid == 0) gidn = ent_u[item.e0];
            }
            // unit v: this warp's rows have landed (the caller waited for them);
            // make them visible to the tensor cores and mark the stage full
            auto finish = [&](int v) {
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                __syncwarp();
                if (lane == 0) mbar_arrive(smem_u32(&bar_full[v % TC_ST]));
            };
            for (int u = 0; u < nunits; ++u) {
                const int s = u % TC_ST, r = u / TC_ST;
                const int e = u / S::NCH, c = u - e * S::NCH;
                if (u >= S::LAG) {
                    // unit u - LAG: own rows landed (at most LAG - 1 newer groups
                    // pending), split, mark full
                    asm volatile("cp.async.wait_group %0;\n" ::"n"(S::LAG - 1) : "memory");
                    finish(u - S::LAG);
                }
                if (c == 0) {
#pragma unroll
                    for (int m = 0; m < MR; ++m) src[m] = srcn[m];
                    gid = gidn;
                    if (e + 1 < ne) {
                        const long long nrow = (long long)item.e0 + e + 1;
                        const int *sr = ent_src + nrow * TT;
#pragma unroll
                        for (int m = 0; m < MR; ++m) srcn[m] = sr[rowof(m)];
                        if (tid == 0) gidn = ent_u[nrow];
                    }
                }
                if (r > 0 && !__all_sync(0xffffffffu, mbar_wait(smem_u32(&bar_empty[s]),
                                                                (r - 1) & 1, abort, spin))) {
                    ok = false;
                    break;
                }
                const uint32_t st = sbase + (uint32_t)(s * S::STAGE);
                if (tid == 0) {
                    const uint32_t bb = smem_u32(&bar_b[s]);
                    mbar_expect_tx(bb, 2 * S::B_BYTES);
                    bulk_g2s(st + 2 * S::A_BYTES,
                             Bop + ((long long)gid * S::NCH + c) * (2 * S::B_BYTES),
                             2 * S::B_BYTES, bb);
                }
                // 16-byte chunks wholly beyond KP feed no MMA (their k-steps are
                // skipped): not copied
                if (c * TC_KC + 4 * j < KP) {
#pragma unroll
                    for (int part = 0; part < 2; ++part) {
                        const float *qb = Qs + part * qplane + c * TC_KC + 4 * j;
#pragma unroll
                        for (int m = 0; m < MR; ++m) {
                            const bool v = src[m] >= 0;
                            tc_cp16(st + part * S::A_BYTES + dst0 + m * (NW / 2) * TC_SBO,
                                    qb + (v ? (long long)src[m] * S::KT : 0ll), v ? 16 : 0);
                        }
                    }
                }
                asm volatile("cp.async.commit_group;\n" ::: "memory");
                issued = u + 1;
            }
            asm volatile("cp.async.wait_all;\n" ::: "memory");
            if (ok)
                for (int u = nunits - S::LAG > 0 ? nunits - S::LAG : 0; u < nunits; ++u) finish(u);
        }
        if (!ok) {
            *abort = 1;
            atomicOr(flags, FLAG_TIMEOUT);
        }
        // operator copies still in flight after a time-out: wait for the
        // last one issued on each stage (phases of a stage complete in order)
        if (tid == 0 && *abort) {
            for (int s = 0; s < TC_ST; ++s) {
                int last = -1;
                for (int u = s; u < issued; u += TC_ST) last = u;
                if (last >= 0) mbar_wait_plain(smem_u32(&bar_b[s]), (last / TC_ST) & 1);
            }
        }
        // ---------------- epilogue: accumulator -> partial sums
        const bool have = nunits > 0 && mbar_wait(done, 0, abort, spin) && !*abort;
        asm volatile("tcgen05.fence::after_thread_sync;");
        if (!*abort) {
            const int quad = warp & 3, half = warp >> 2;
            float *out = Ps + ((long long)itx * TT + quad * 32 + lane) * KP;
            const uint32_t trow = tmem + ((uint32_t)(quad * 32) << 16);
#pragma unroll
            for (int c0 = 16 * half; c0 < S::N; c0 += 16 * (TC_PROD / 128)) {
                uint32_t rh[16], rl2[16];
                if (have) {
                    tmem_ld16(trow + (uint32_t)c0, rh);
                    tmem_ld16(trow + (uint32_t)(S::N + c0), rl2);
                    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
                } else {
#pragma unroll
                    for (int q = 0; q < 16; ++q) rh[q] = rl2[q] = 0u;
                }
#pragma unroll
                for (int q = 0; q < 16; q += 4)
                    if (c0 + q < KP)
                        *reinterpret_cast<float4 *>(out + c0 + q) = make_float4(
                            __uint_as_float(rh[q]) + __uint_as_float(rl2[q]),
                            __uint_as_float(rh[q + 1]) + __uint_as_float(rl2[q + 1]),
                            __uint_as_float(rh[q + 2]) + __uint_as_float(rl2[q + 2]),
                            __uint_as_float(rh[q + 3]) + __uint_as_float(rl2[q + 3]));
            }
        }
    } else if (lane == 0) {
        // ---------------- MMA issue (one thread)
        const uint32_t idesc2 = (1u << 4) | (2u << 7) | (2u << 10) |
                                ((uint32_t)(2 * S::N >> 3) << 17) | ((uint32_t)(TC_M >> 4) << 24);
        const uint32_t idesc1 = (1u << 4) | (2u << 7) | (2u << 10) |
                                ((uint32_t)(S::N >> 3) << 17) | ((uint32_t)(TC_M >> 4) << 24);
        bool ok = true;
        // stall (failure-path tests only): issue nothing, so that the
        // producers' bounded waits for a free stage run out
        for (int u = 0; u < (stall ? 0 : nunits); ++u) {
            const int s = u % TC_ST, r = u / TC_ST;
            if ((!TMA && !mbar_wait(smem_u32(&bar_full[s]), r & 1, abort, spin)) ||
                !mbar_wait(smem_u32(&bar_b[s]), r & 1, abort, spin)) {
                ok = false;
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;");
            const uint32_t a0 = sbase + (uint32_t)(s * S::STAGE), a1 = a0 + S::A_BYTES;
            const uint32_t b0 = a0 + 2 * S::A_BYTES;  // B_hi, then B_lo: 2N rows
            const int c = u % S::NCH;
#pragma unroll
            for (int kk = 0; kk < TC_KC / 8; ++kk) {
                if (c * TC_KC + 8 * kk >= KP) break;  // all-zero K columns
                const uint32_t o = kk * 32;
                // [acc_hi | acc_lo] += A_hi [B_hi | B_lo];  acc_hi += A_lo B_hi
                tc_mma(tmem, umma_desc(a0 + o), umma_desc(b0 + o), idesc2,
                       (u == 0 && kk == 0) ? 0u : 1u);
                tc_mma(tmem, umma_desc(a1 + o), umma_desc(b0 + o), idesc1, 1u);
            }
            tc_commit(smem_u32(&bar_empty[s]));
        }
        if (!ok) {
            *abort = 1;
            atomicOr(flags, FLAG_TIMEOUT);
        }
        // arrives once every MMA issued above has completed
        tc_commit(done);
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (warp == MMA_WARP) {
        if (*abort && lane == 0) mbar_wait_plain(done, 0);
        __syncwarp();
        asm volatile("tcgen05.fence::after_thread_sync;");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                     "r"(S::TMEM_COLS));
    }
}

template <int KP, bool TMA>
__global__ void __launch_bounds__(TC_THREADS, 1)
    k_m2l_tc(const M2LItem *items, const int *ent_u, const int *ent_src, const float *Qs,
             long long qplane, const __grid_constant__ CUtensorMap qmap, int ncell,
             const unsigned char *Bop, float *Ps, int *flags, long long spin, int stall)
{
    m2l_tc_body<KP, TMA>(items, ent_u, ent_src, Qs, qplane, &qmap, ncell, Bop, Ps, flags, spin,
                         stall, blockIdx.x);
}

// every member's items in one launch (ensemble step; cp.async gather)
template <int KP>
__global__ void __launch_bounds__(TC_THREADS, 1)
    k_m2l_tc_batch(const M2LTCArgs *a, const int *bstart, int nm, long long spin, int stall)
{
    int itx;
    const M2LTCArgs &x = a[batch_member(bstart, nm, blockIdx.x, itx)];
    m2l_tc_body<KP, false>(x.items, x.ent_u, x.ent_src, x.Qs, x.qplane, nullptr, 0, x.Bop, x.Ps,
                           x.flags, spin, stall, itx);
}

// ------------------------------------------- contraction, A in tensor memory
// The same contraction with the gathered operand A (partner moments of the
// tile's 128 cells) in tensor memory instead of shared memory.  Per unit the
// producers load their cells' 32 scaled FP32 moments straight from global
// memory into registers (one warp per 32 TMEM lanes and 16 of the 32 K
// columns, one unit ahead), split them into TF32 hi and lo there, and store
// both with tcgen05.st into the unit's TMEM stage; only the operator chunk
// (B) passes through shared memory.  This removes the A writes and the MMA's
// A reads from shared memory (about half its traffic per unit) and halves
// the gathered bytes (one FP32 plane instead of two TF32 planes).
//   TMEM: columns [0, 2N) the accumulator halves [acc_hi | acc_lo]; the
//   last ST x 64 columns the A stages, each [A_hi (32) | A_lo (32)].
//   k-steps whose 8 K columns all lie beyond KP are skipped.
// The shared memory request is at least 116 KB, so that two of these CTAs
// never share an SM (each allocates all 512 TMEM columns); the rest of the
// SM's shared memory is left to near-field blocks running concurrently.
// units whose moments each producer thread keeps in flight
#ifndef CCFMM_TCT_D
#define CCFMM_TCT_D 4
#endif
constexpr int TCT_D = CCFMM_TCT_D;

template <int KP> struct TctShape {
    typedef TcShape<KP> S;
    static constexpr int A_COLS = 2 * TC_KC;
    static constexpr int ST = (512 - 2 * S::N) / A_COLS > 6 ? 6 : (512 - 2 * S::N) / A_COLS;
    static constexpr int ACOL0 = 512 - ST * A_COLS;
    static constexpr int BSTAGE = 2 * S::B_BYTES;
    static constexpr int SMEM_USE = ST * BSTAGE + 1024;
    static constexpr int SMEM = SMEM_USE > 116 * 1024 ? SMEM_USE : 116 * 1024;
    static_assert(ST >= 3 && ACOL0 >= 2 * S::N, "tensor memory plan");
};

__device__ __forceinline__ void tmem_st16(uint32_t taddr, const float (&v)[16])
{
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,"
        "%13,%14,%15,%16};\n" ::"r"(taddr),
        "r"(__float_as_uint(v[0])), "r"(__float_as_uint(v[1])), "r"(__float_as_uint(v[2])),
        "r"(__float_as_uint(v[3])), "r"(__float_as_uint(v[4])), "r"(__float_as_uint(v[5])),
        "r"(__float_as_uint(v[6])), "r"(__float_as_uint(v[7])), "r"(__float_as_uint(v[8])),
        "r"(__float_as_uint(v[9])), "r"(__float_as_uint(v[10])), "r"(__float_as_uint(v[11])),
        "r"(__float_as_uint(v[12])), "r"(__float_as_uint(v[13])), "r"(__float_as_uint(v[14])),
        "r"(__float_as_uint(v[15]))
        : "memory");
}

// D (tmem) [+]= A (tmem) x B (smem descriptor)
__device__ __forceinline__ void tc_mma_ts(uint32_t d_tmem, uint32_t a_tmem, uint64_t b,
                                          uint32_t idesc, uint32_t acc)
{
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::tf32 [%0], [%1], %2, %3, p;\n}\n" ::"r"(d_tmem),
        "r"(a_tmem), "l"(b), "r"(idesc), "r"(acc));
}

template <int KP>
__global__ void __launch_bounds__(TC_THREADS, 1)
    k_m2l_tct(const M2LItem *items, const int *ent_u, const int *ent_src, const float *Qf,
              const unsigned char *Bop, float *Ps, int *flags, long long spin, int stall)
{
    typedef TcShape<KP> S;
    typedef TctShape<KP> T;
    constexpr int ST = T::ST;
    static_assert(TC_PROD == 256, "eight producer warps: two per TMEM lane quarter");
    extern __shared__ __align__(1024) unsigned char smraw[];
    __shared__ __align__(8) unsigned long long bar_full[ST], bar_b[ST], bar_empty[ST];
    __shared__ __align__(8) unsigned long long bar_done;
    __shared__ uint32_t tmem_slot;
    __shared__ int s_abort;
    volatile int *abort = &s_abort;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const M2LItem item = items[blockIdx.x];
    const int ne = item.e1 - item.e0;
    const int nunits = ne * S::NCH;
    const uint32_t sbase = (smem_u32(smraw) + 1023u) & ~1023u;  // swizzle atoms
    const uint32_t done = smem_u32(&bar_done);

    if (tid == 0) {
        *abort = 0;
        for (int s = 0; s < ST; ++s) {
            mbar_init(smem_u32(&bar_full[s]), TC_PROD / 32);
            mbar_init(smem_u32(&bar_b[s]), 1);
            mbar_init(smem_u32(&bar_empty[s]), 1);
        }
        mbar_init(done, 1);
        asm volatile("fence.mbarrier_init.release.cluster;");
    }
    constexpr int MMA_WARP = TC_PROD / 32;
    if (warp == MMA_WARP) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;" ::"r"(
            smem_u32(&tmem_slot)));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tmem = tmem_slot;

    if (warp < MMA_WARP) {
        // ---------------- producers: warp w owns TMEM lanes 32 (w mod 4) ..
        // (the tile's cells) and K columns 16 (w / 4) .. of every unit
        const int quad = warp & 3, half = warp >> 2;
        const int row = 32 * quad + lane;
        const uint32_t tl = tmem + ((uint32_t)(32 * quad) << 16) + (uint32_t)(T::ACOL0 + 16 * half);
        // this thread's 16 moments of a unit (zeros for a cell without the
        // partner)
        auto load = [&](int src, int c, float4 (&r)[4]) {
            if (src >= 0) {
                const float4 *q = reinterpret_cast<const float4 *>(
                    Qf + (long long)src * S::KT + c * TC_KC + 16 * half);
#pragma unroll
                for (int j = 0; j < 4; ++j) r[j] = __ldg(q + j);
            } else {
#pragma unroll
                for (int j = 0; j < 4; ++j) r[j] = make_float4(0.f, 0.f, 0.f, 0.f);
            }
        };
        // Loads run TCT_D units ahead of the stores, in unit order, through a
        // ring of register buffers: ld_e / ld_src are the entry and partner
        // row of the latest load, pf_src the row of entry ld_e + 1 (fetched
        // one entry ahead, so that no data load waits on its index).
        int ld_u = 0, ld_e = 0, ld_src = -1, pf_src = -1;
        if (ne > 0) {
            ld_src = ent_src[(long long)item.e0 * TT + row];
            if (ne > 1) pf_src = ent_src[(long long)(item.e0 + 1) * TT + row];
        }
        auto issue = [&](float4 (&r)[4]) {
            if (ld_u < nunits) {
                const int e = ld_u / S::NCH, c = ld_u - e * S::NCH;
                if (e != ld_e) {  // the next entry (units advance one at a time)
                    ld_e = e;
                    ld_src = pf_src;
                    pf_src = e + 1 < ne ? ent_src[((long long)item.e0 + e + 1) * TT + row] : -1;
                }
                load(ld_src, c, r);
            }
            ++ld_u;
        };
        // operator class of the current entry and of the next one (thread 0)
        int gid_cur = 0, gid_nx = 0;
        if (tid == 0 && ne > 0) {
            gid_cur = ent_u[item.e0];
            if (ne > 1) gid_nx = ent_u[item.e0 + 1];
        }
        float4 buf[TCT_D][4];
#pragma unroll
        for (int d = 0; d < TCT_D; ++d) issue(buf[d]);
        int issued = 0;
        bool ok = true;
        for (int u0 = 0; u0 < nunits && ok; u0 += TCT_D) {
#pragma unroll
            for (int d = 0; d < TCT_D; ++d) {
                const int u = u0 + d;
                if (u >= nunits) break;
                const int s = u % ST, r = u / ST;
                const int e = u / S::NCH, c = u - e * S::NCH;
                if (tid == 0 && c == 0 && e > 0) {
                    gid_cur = gid_nx;
                    gid_nx = e + 1 < ne ? ent_u[item.e0 + e + 1] : 0;
                }
                if (r > 0 && !__all_sync(0xffffffffu, mbar_wait(smem_u32(&bar_empty[s]),
                                                                (r - 1) & 1, abort, spin))) {
                    ok = false;
                    break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;");
                if (tid == 0) {
                    const uint32_t bb = smem_u32(&bar_b[s]);
                    mbar_expect_tx(bb, T::BSTAGE);
                    bulk_g2s(sbase + (uint32_t)(s * T::BSTAGE),
                             Bop + ((long long)gid_cur * S::NCH + c) * T::BSTAGE, T::BSTAGE, bb);
                }
                issued = u + 1;
                float hi[16], lo[16];
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const float v[4] = {buf[d][j].x, buf[d][j].y, buf[d][j].z, buf[d][j].w};
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        hi[4 * j + q] = to_tf32(v[q]);
                        lo[4 * j + q] = v[q] - hi[4 * j + q];
                    }
                }
                // unit u + TCT_D into the buffer just consumed
                issue(buf[d]);
                const uint32_t ta = tl + (uint32_t)(s * T::A_COLS);
                tmem_st16(ta, hi);
                tmem_st16(ta + TC_KC, lo);
                asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
                asm volatile("tcgen05.fence::before_thread_sync;");
                __syncwarp();
                if (lane == 0) mbar_arrive(smem_u32(&bar_full[s]));
            }
        }
        if (!ok) {
            *abort = 1;
            atomicOr(flags, FLAG_TIMEOUT);
        }
        // operator copies still in flight after a time-out: wait for the
        // last one issued on each stage (phases of a stage complete in order)
        if (tid == 0 && *abort) {
            for (int s = 0; s < ST; ++s) {
                int last = -1;
                for (int u = s; u < issued; u += ST) last = u;
                if (last >= 0) mbar_wait_plain(smem_u32(&bar_b[s]), (last / ST) & 1);
            }
        }
        // ---------------- epilogue: accumulator -> partial sums
        const bool have = nunits > 0 && mbar_wait(done, 0, abort, spin) && !*abort;
        asm volatile("tcgen05.fence::after_thread_sync;");
        if (!*abort) {
            float *out = Ps + ((long long)blockIdx.x * TT + quad * 32 + lane) * KP;
            const uint32_t trow = tmem + ((uint32_t)(quad * 32) << 16);
#pragma unroll
            for (int c0 = 16 * half; c0 < S::N; c0 += 32) {
                uint32_t rh[16], rl2[16];
                if (have) {
                    tmem_ld16(trow + (uint32_t)c0, rh);
                    tmem_ld16(trow + (uint32_t)(S::N + c0), rl2);
                    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
                } else {
#pragma unroll
                    for (int q = 0; q < 16; ++q) rh[q] = rl2[q] = 0u;
                }
#pragma unroll
                for (int q = 0; q < 16; q += 4)
                    if (c0 + q < KP)
                        *reinterpret_cast<float4 *>(out + c0 + q) = make_float4(
                            __uint_as_float(rh[q]) + __uint_as_float(rl2[q]),
                            __uint_as_float(rh[q + 1]) + __uint_as_float(rl2[q + 1]),
                            __uint_as_float(rh[q + 2]) + __uint_as_float(rl2[q + 2]),
                            __uint_as_float(rh[q + 3]) + __uint_as_float(rl2[q + 3]));
            }
        }
    } else if (lane == 0) {
        // ---------------- MMA issue (one thread)
        const uint32_t idesc2 = (1u << 4) | (2u << 7) | (2u << 10) |
                                ((uint32_t)(2 * S::N >> 3) << 17) | ((uint32_t)(TC_M >> 4) << 24);
        const uint32_t idesc1 = (1u << 4) | (2u << 7) | (2u << 10) |
                                ((uint32_t)(S::N >> 3) << 17) | ((uint32_t)(TC_M >> 4) << 24);
        bool ok = true;
        for (int u = 0; u < (stall ? 0 : nunits); ++u) {
            const int s = u % ST, r = u / ST;
            const int c = u % S::NCH;
            if (!mbar_wait(smem_u32(&bar_full[s]), r & 1, abort, spin) ||
                !mbar_wait(smem_u32(&bar_b[s]), r & 1, abort, spin)) {
                ok = false;
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;");
            const uint32_t a0 = tmem + (uint32_t)(T::ACOL0 + s * T::A_COLS), a1 = a0 + TC_KC;
            const uint32_t b0 = sbase + (uint32_t)(s * T::BSTAGE);  // B_hi, then B_lo: 2N rows
#pragma unroll
            for (int kk = 0; kk < TC_KC / 8; ++kk) {
                if (c * TC_KC + 8 * kk >= KP) break;  // all-zero K columns
                // [acc_hi | acc_lo] += A_hi [B_hi | B_lo];  acc_hi += A_lo B_hi
                tc_mma_ts(tmem, a0 + 8 * kk, umma_desc(b0 + kk * 32), idesc2,
                          (u == 0 && kk == 0) ? 0u : 1u);
                tc_mma_ts(tmem, a1 + 8 * kk, umma_desc(b0 + kk * 32), idesc1, 1u);
            }
            tc_commit(smem_u32(&bar_empty[s]));
        }
        if (!ok) {
            *abort = 1;
            atomicOr(flags, FLAG_TIMEOUT);
        }
        // arrives once every MMA issued above has completed
        tc_commit(done);
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (warp == MMA_WARP) {
        if (*abort && lane == 0) mbar_wait_plain(done, 0);
        __syncwarp();
        asm volatile("tcgen05.fence::after_thread_sync;");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" ::"r"(tmem));
    }
}

template <int KP> static size_t tc_smem()
{
    return (size_t)TcShape<KP>::ST * TcShape<KP>::STAGE + 1024;
}

// blocks of the fold for ncell cells (full width KP)
int q_split_blocks(int KP, long long ncell)
{
    (void)KP;
    return (int)((ncell + QF_W - 1) / QF_W);
}

void launch_q_split_batch(int KP, const QSplitArgs *a, const int *bstart, int nm, int nblocks,
                          cudaStream_t s)
{
    if (nblocks <= 0) return;
    note_launch();
    switch (KP) {
    case 40: k_q_fold_batch<24><<<(unsigned)nblocks, 32 * QF_W, 0, s>>>(KP, a, bstart, nm); break;
    case 56: k_q_fold_batch<40><<<(unsigned)nblocks, 32 * QF_W, 0, s>>>(KP, a, bstart, nm); break;
    case 88: k_q_fold_batch<48><<<(unsigned)nblocks, 32 * QF_W, 0, s>>>(KP, a, bstart, nm); break;
    case 120: k_q_fold_batch<64><<<(unsigned)nblocks, 32 * QF_W, 0, s>>>(KP, a, bstart, nm); break;
    default: break;
    }
}

void launch_m2l_tc_batch(int KP, const M2LTCArgs *a, const int *bstart, int nm, int nblocks,
                         long long spin, int stall, cudaStream_t s)
{
    if (nblocks <= 0) return;
#define M2LTCB(KPV, KRV)                                                                        \
    case KPV: {                                                                                 \
        const int smem = (int)tc_smem<KRV>();                                                   \
        cudaFuncSetAttribute(k_m2l_tc_batch<KRV>, cudaFuncAttributeMaxDynamicSharedMemorySize,  \
                             smem);                                                             \
        note_launch();                                                                          \
        k_m2l_tc_batch<KRV><<<(unsigned)nblocks, TC_THREADS, smem, s>>>(a, bstart, nm, spin,     \
                                                                        stall);                 \
    } break;
    switch (KP) {
        M2LTCB(40, 24) M2LTCB(56, 40) M2LTCB(88, 48) M2LTCB(120, 64)
    default: break;
    }
#undef M2LTCB
}

bool m2l_tc_supported(int KP)
{
    switch (KP) {
    case 40: return tc_smem<24>() <= 227 * 1024;
    case 56: return tc_smem<40>() <= 227 * 1024;
    case 88: return tc_smem<48>() <= 227 * 1024;
    case 120: return tc_smem<64>() <= 227 * 1024;
    default: return false;
    }
}

size_t m2l_tc_op_bytes(int KP)
{
    switch (KP) {
    case 40: return TcShape<24>::OP_BYTES;
    case 56: return TcShape<40>::OP_BYTES;
    case 88: return TcShape<48>::OP_BYTES;
    case 120: return TcShape<64>::OP_BYTES;
    default: return 0;
    }
}

int m2l_tc_kt(int KP)
{
    switch (KP) {
    case 40: return TcShape<24>::KT;
    case 56: return TcShape<40>::KT;
    case 88: return TcShape<48>::KT;
    case 120: return TcShape<64>::KT;
    default: return 0;
    }
}

void launch_m2l_tc_ops(int p, int KP, int L, int n_off, const Geom *g, const float *D, int ldD,
                       const uint16_t *it, float *gk, float *Bop, cudaStream_t s)
{
    const int KT = m2l_tc_kt(KP);
    note_launch();
    k_tc_scale<<<LCAP + 1, 128, 0, s>>>(p, KT, L, g, gk);
    if (n_off <= 0) return;
    const size_t smem = sizeof(float) * (size_t)ldD;
#define M2LOPS(KPV, KRV)                                                                       \
    case KPV:                                                                                  \
        note_launch();                                                                         \
        k_m2l_ops<KRV><<<n_off, 256, smem, s>>>(p, KPV, D, ldD, it, Bop);                      \
        break;
    switch (KP) {
        M2LOPS(40, 24) M2LOPS(56, 40) M2LOPS(88, 48) M2LOPS(120, 64)
    default: break;
    }
#undef M2LOPS
}

// Tensor map of the split moments for the TMA gather: rows of KT floats, the
// hi plane (rows 0 .. ncell-1) then the lo plane; box = one 128-byte row,
// 128-byte swizzle (the MMA operand layout).  map: 128 bytes, 64-byte aligned.
bool m2l_tc_qmap(void *map, const float *Qs, long long ncell, int KP)
{
    // resolved once (thread-safe static initialisation); nullptr if the
    // driver does not provide it
    static const PFN_cuTensorMapEncodeTiled_v12000 encode = []() {
        void *fn = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000,
                                             cudaEnableDefault, &q) != cudaSuccess ||
            q != cudaDriverEntryPointSuccess) {
            cudaGetLastError();
            fn = nullptr;
        }
        return reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
    }();
    if (!encode) return false;
    const int KT = m2l_tc_kt(KP);
    if (KT <= 0 || 2 * ncell >= (1ll << 31)) return false;
    cuuint64_t dim[2] = {(cuuint64_t)KT, (cuuint64_t)(2 * ncell)};
    cuuint64_t stride[1] = {(cuuint64_t)KT * sizeof(float)};
    cuuint32_t box[2] = {(cuuint32_t)TC_KC, 1u};
    cuuint32_t estr[2] = {1u, 1u};
    return encode(reinterpret_cast<CUtensorMap *>(map), CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2,
                  const_cast<float *>(Qs), dim, stride, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                  CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

void launch_m2l_tc(int p, int KP, const Tile *tiles, int ntiles, const M2LItem *items, int nitems,
                   const int *tile_item0, const int *tile_nitems, const int *ent_u,
                   const int *ent_src, const float *Q, long long ncell, const float *gk,
                   float *Qs, const void *qmap, bool a_tmem, const float *Bop, const Geom *g,
                   float *Ps, double *V, int *flags, cudaStream_t s)
{
    // qmap (a tensor map from m2l_tc_qmap) selects the TMA gather, nullptr
    // the cp.async gather
    CUtensorMap none;
    memset(&none, 0, sizeof(none));
    const CUtensorMap &qm = qmap ? *reinterpret_cast<const CUtensorMap *>(qmap) : none;
    // CCFMM_TC_STALL=1 (failure-path tests): the MMA thread issues nothing
    // and the waits give up after 2^12 polls; the evaluation then reports
    // CCFMM_ERR_TIMEOUT
    const char *sv = getenv("CCFMM_TC_STALL");
    const int stall = (sv && atoi(sv)) ? 1 : 0;
    const long long spin = stall ? (1ll << 12) : TC_SPIN;
    if (nitems > 0 && a_tmem) {
#define M2LTCT(KPV, KRV)                                                                        \
    case KPV: {                                                                                 \
        note_launch();                                                                          \
        k_q_fold<KRV, false><<<(unsigned)((ncell + QF_W - 1) / QF_W), 32 * QF_W, 0, s>>>(        \
            p, KPV, ncell, Q, gk, Qs);                                                          \
        const int smem = TctShape<KRV>::SMEM;                                                   \
        cudaFuncSetAttribute(k_m2l_tct<KRV>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem); \
        note_launch();                                                                          \
        k_m2l_tct<KRV><<<nitems, TC_THREADS, smem, s>>>(                                        \
            items, ent_u, ent_src, Qs, reinterpret_cast<const unsigned char *>(Bop), Ps, flags, \
            spin, stall);                                                                       \
    } break;
        switch (KP) {
            M2LTCT(40, 24) M2LTCT(56, 40) M2LTCT(88, 48) M2LTCT(120, 64)
        default: break;
        }
#undef M2LTCT
    } else if (nitems > 0) {
#define M2LTC(KPV, KRV)                                                                         \
    case KPV: {                                                                                 \
        typedef TcShape<KRV> S;                                                                 \
        note_launch();                                                                          \
        k_q_fold<KRV, true><<<(unsigned)((ncell + QF_W - 1) / QF_W), 32 * QF_W, 0, s>>>(         \
            p, KPV, ncell, Q, gk, Qs);                                                          \
        size_t smem = tc_smem<KRV>();                                                           \
        auto kern = qmap ? k_m2l_tc<KRV, true> : k_m2l_tc<KRV, false>;                          \
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);    \
        note_launch();                                                                          \
        kern<<<nitems, TC_THREADS, smem, s>>>(                                                  \
            items, ent_u, ent_src, Qs, ncell * S::KT, qm, (int)ncell,                           \
            reinterpret_cast<const unsigned char *>(Bop), Ps, flags, spin, stall);              \
    } break;
        switch (KP) {
            M2LTC(40, 24) M2LTC(56, 40) M2LTC(88, 48) M2LTC(120, 64)
        default: break;
        }
#undef M2LTC
    }
    launch_reduce_h(p, KP, tiles, ntiles, tile_item0, tile_nitems, Ps, g, V, s);
}

}  // namespace ccfmm
