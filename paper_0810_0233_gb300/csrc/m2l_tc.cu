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
// once per evaluation (k_q_split, rows of KT floats), the operators once per
// tree build (k_m2l_ops, one per far offset class), stored in global memory
// in exactly the shared-memory layout the MMA reads, so that a unit's
// operator chunk arrives with one bulk copy.
//
// Shared-memory operands use the no-swizzle K-major canonical layout: core
// matrices of 8 rows x 16 bytes (4 TF32), adjacent along K at 128 bytes
// (leading-dimension offset), 8-row groups at 1024 bytes (stride offset).
//
// Pipeline, TC_ST stages of one unit = (entry, 32-wide K chunk) each:
//   warps 0-3  wait for the stage to be free, gather the 128 partner rows of
//              the chunk (cp.async; zero rows for cells without that
//              partner), and thread 0 starts the bulk copy of the operator
//              chunk; a thread marks the stage full after its own copies of
//              the unit have landed (one unit later, so two are in flight);
//   warp 4     one thread issues the unit's 12 MMAs once the stage is full
//              and frees the stage with tcgen05.commit;
//   warps 0-3  finally read the accumulator (tcgen05.ld) into the item's
//              FP32 partial sums, which k_m2l_reduce adds in FP64.
// Every wait is bounded; on time-out the kernel raises FLAG_TIMEOUT, lets
// its copies and MMAs finish (again bounded), frees its tensor memory and
// returns.
#include "ccfmm_dev.cuh"

namespace ccfmm {

constexpr int TC_M = 128;       // field cells per tile (MMA M = TMEM lanes)
constexpr int TC_KC = 32;       // K per unit: 4 MMA k-steps of 8
constexpr int TC_ST = 3;        // pipeline stages
constexpr int TC_PROD = 128;    // producer / epilogue threads (warps 0-3)
constexpr int TC_THREADS = TC_PROD + 32;
constexpr int TC_SBO = (TC_KC / 4) * 128;  // bytes between 8-row groups
constexpr long long TC_SPIN = 1ll << 22;

template <int KP> struct TcShape {
    static constexpr int N = ((KP + 15) / 16) * 16;               // MMA N
    static constexpr int KT = ((KP + TC_KC - 1) / TC_KC) * TC_KC;  // padded K
    static constexpr int NCH = KT / TC_KC;                        // units per entry
    static constexpr int A_BYTES = TC_M * TC_KC * 4;
    static constexpr int B_BYTES = N * TC_KC * 4;
    static constexpr int STAGE = 2 * A_BYTES + 2 * B_BYTES;
    static constexpr int OP_BYTES = NCH * 2 * B_BYTES;            // one offset class
    static constexpr int TMEM_COLS = N <= 32 ? 32 : (N <= 64 ? 64 : (N <= 128 ? 128 : 256));
};

__device__ __forceinline__ uint32_t smem_u32(const void *p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ uint64_t umma_desc(uint32_t saddr)
{
    uint64_t d = 0;
    d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
    d |= (uint64_t)((128u >> 4) & 0x3FFFu) << 16;              // leading-dimension offset
    d |= (uint64_t)(((uint32_t)TC_SBO >> 4) & 0x3FFFu) << 32;  // stride offset
    d |= (uint64_t)1 << 46;  // descriptor version for tcgen05
    return d;                // base offset 0, no swizzle
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

// bounded wait; gives up early once another thread has given up
__device__ __forceinline__ bool mbar_wait(uint32_t a, uint32_t parity, volatile int *abort)
{
    for (long long i = 0; i < TC_SPIN; ++i) {
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
    const int K = nterms(p) - 1;
    for (int k = threadIdx.x; k < KT; k += blockDim.x) {
        float v = 0.f;
        if (k < K && l <= L) {
            int nx, ny, nz;
            midx_inv(k + 1, nx, ny, nz);
            v = (float)pow(g->h[l], (double)(1 - (nx + ny + nz)));
        }
        gk[l * KT + k] = v;
    }
}

// Operator chunks of every far offset class: for chunk c and part (hi, lo),
// the N x 32 block M[n][k] = D~_{n+k}, k = 32c + kl, in canonical layout.
template <int KP>
__global__ void k_m2l_ops(int p, const float *D, int ldD, const uint16_t *it_g, float *Bop)
{
    typedef TcShape<KP> S;
    extern __shared__ float Dl[];
    const int K = nterms(p) - 1;
    const long long gid = blockIdx.x;
    for (int i = threadIdx.x; i < ldD; i += blockDim.x) Dl[i] = D[gid * ldD + i];
    __syncthreads();
    float *out = Bop + gid * (S::OP_BYTES / 4);
    constexpr int PER = S::N * TC_KC;  // floats per (chunk, part)
    for (int o = threadIdx.x; o < S::NCH * PER; o += blockDim.x) {
        const int c = o / PER, q = o - c * PER;
        // float index q = (n&7)*4 + (kl>>2)*32 + (n>>3)*256 + (kl&3)
        const int kl = (q & 3) | (((q >> 5) & 7) << 2);
        const int n = ((q >> 2) & 7) | ((q >> 8) << 3);
        const int k = c * TC_KC + kl;
        const float v = (n < K && k < K) ? Dl[it_g[k * KP + n]] : 0.f;
        const float hi = to_tf32(v);
        out[c * 2 * PER + q] = hi;
        out[c * 2 * PER + PER + q] = v - hi;
    }
}

// Scaled moments split into TF32 pairs: Qs[part][hid][k], rows of KT floats.
template <int KP>
__global__ void k_q_split(int p, long long ncell, const float *Q, const float *gk, float *Qs)
{
    typedef TcShape<KP> S;
    constexpr int KT = S::KT;
    const int K = nterms(p) - 1;
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= ncell * (KT / 4)) return;
    const long long hid = i / (KT / 4);
    const int k4 = (int)(i - hid * (KT / 4)) * 4;
    const int level = hid > 0 ? 63 - __clzll(hid) : 0;
    float v[4] = {0.f, 0.f, 0.f, 0.f};
    if (k4 < KP) {
        const float4 q = *reinterpret_cast<const float4 *>(Q + hid * KP + k4);
        const float4 s = *reinterpret_cast<const float4 *>(gk + level * KT + k4);
        v[0] = q.x * s.x;
        v[1] = q.y * s.y;
        v[2] = q.z * s.z;
        v[3] = q.w * s.w;
    }
    float hi[4], lo[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        if (k4 + j >= K) v[j] = 0.f;
        hi[j] = to_tf32(v[j]);
        lo[j] = v[j] - hi[j];
    }
    *reinterpret_cast<float4 *>(Qs + hid * KT + k4) = make_float4(hi[0], hi[1], hi[2], hi[3]);
    *reinterpret_cast<float4 *>(Qs + (ncell + hid) * KT + k4) =
        make_float4(lo[0], lo[1], lo[2], lo[3]);
}

// ------------------------------------------------------------ contraction
template <int KP>
__global__ void __launch_bounds__(TC_THREADS, 1)
    k_m2l_tc(const M2LItem *items, const int *ent_u, const int *ent_src, const float *Qs,
             long long qplane, const unsigned char *Bop, float *Ps, int *flags)
{
    typedef TcShape<KP> S;
    extern __shared__ __align__(1024) unsigned char smraw[];
    __shared__ __align__(8) unsigned long long bar_full[TC_ST], bar_b[TC_ST], bar_empty[TC_ST];
    __shared__ __align__(8) unsigned long long bar_done;
    __shared__ uint32_t tmem_slot;
    __shared__ int s_abort;
    volatile int *abort = &s_abort;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const M2LItem item = items[blockIdx.x];
    const int ne = item.e1 - item.e0;
    const int nunits = ne * S::NCH;
    const uint32_t sbase = smem_u32(smraw);
    const uint32_t done = smem_u32(&bar_done);

    if (tid == 0) {
        *abort = 0;
        for (int s = 0; s < TC_ST; ++s) {
            mbar_init(smem_u32(&bar_full[s]), TC_PROD);
            mbar_init(smem_u32(&bar_b[s]), 1);
            mbar_init(smem_u32(&bar_empty[s]), 1);
        }
        mbar_init(done, 1);
        asm volatile("fence.mbarrier_init.release.cluster;");
    }
    if (warp == 4) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(&tmem_slot)),
                     "r"(S::TMEM_COLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tmem = tmem_slot;

    if (warp < 4) {
        // ---------------- producers
        const int rl = tid & 7, j = (tid >> 3) & 7, rh0 = tid >> 6;
        const uint32_t dst0 = (uint32_t)(rl * 16 + j * 128 + rh0 * TC_SBO);
        int src[8];
        int issued = 0;
        bool ok = true;
        for (int u = 0; u < nunits; ++u) {
            const int s = u % TC_ST, r = u / TC_ST;
            const int e = u / S::NCH, c = u - e * S::NCH;
            if (r > 0 && !mbar_wait(smem_u32(&bar_empty[s]), (r - 1) & 1, abort)) {
                ok = false;
                break;
            }
            const uint32_t st = sbase + (uint32_t)(s * S::STAGE);
            const long long row = (long long)item.e0 + e;
            if (tid == 0) {
                const uint32_t bb = smem_u32(&bar_b[s]);
                mbar_expect_tx(bb, 2 * S::B_BYTES);
                bulk_g2s(st + 2 * S::A_BYTES,
                         Bop + ((long long)ent_u[row] * S::NCH + c) * (2 * S::B_BYTES),
                         2 * S::B_BYTES, bb);
            }
            if (c == 0) {
                const int *sr = ent_src + row * TT;
#pragma unroll
                for (int m = 0; m < 8; ++m) src[m] = sr[(rh0 + 2 * m) * 8 + rl];
            }
#pragma unroll
            for (int part = 0; part < 2; ++part) {
                const float *qb = Qs + part * qplane + c * TC_KC + 4 * j;
#pragma unroll
                for (int m = 0; m < 8; ++m) {
                    const bool v = src[m] >= 0;
                    tc_cp16(st + part * S::A_BYTES + dst0 + m * 2 * TC_SBO,
                            qb + (v ? (long long)src[m] * S::KT : 0ll), v ? 16 : 0);
                }
            }
            asm volatile("cp.async.commit_group;\n" ::: "memory");
            issued = u + 1;
            if (u > 0) {
                asm volatile("cp.async.wait_group 1;\n" ::: "memory");
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                mbar_arrive(smem_u32(&bar_full[(u - 1) % TC_ST]));
            }
        }
        asm volatile("cp.async.wait_all;\n" ::: "memory");
        if (ok && nunits > 0) {
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            mbar_arrive(smem_u32(&bar_full[(nunits - 1) % TC_ST]));
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
        const bool have = nunits > 0 && mbar_wait(done, 0, abort) && !*abort;
        asm volatile("tcgen05.fence::after_thread_sync;");
        if (!*abort) {
            float *out = Ps + ((long long)blockIdx.x * TT + warp * 32 + lane) * KP;
#pragma unroll
            for (int c0 = 0; c0 < S::N; c0 += 16) {
                uint32_t rr[16];
                if (have) {
                    const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0;
                    asm volatile(
                        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,"
                        "%10,%11,%12,%13,%14,%15}, [%16];\n"
                        : "=r"(rr[0]), "=r"(rr[1]), "=r"(rr[2]), "=r"(rr[3]), "=r"(rr[4]),
                          "=r"(rr[5]), "=r"(rr[6]), "=r"(rr[7]), "=r"(rr[8]), "=r"(rr[9]),
                          "=r"(rr[10]), "=r"(rr[11]), "=r"(rr[12]), "=r"(rr[13]), "=r"(rr[14]),
                          "=r"(rr[15])
                        : "r"(taddr));
                    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
                } else {
#pragma unroll
                    for (int q = 0; q < 16; ++q) rr[q] = 0u;
                }
#pragma unroll
                for (int q = 0; q < 16; q += 4)
                    if (c0 + q < KP)
                        *reinterpret_cast<float4 *>(out + c0 + q) =
                            make_float4(__uint_as_float(rr[q]), __uint_as_float(rr[q + 1]),
                                        __uint_as_float(rr[q + 2]), __uint_as_float(rr[q + 3]));
            }
        }
    } else if (lane == 0) {
        // ---------------- MMA issue (one thread)
        const uint32_t idesc = (1u << 4) | (2u << 7) | (2u << 10) |
                               ((uint32_t)(S::N >> 3) << 17) | ((uint32_t)(TC_M >> 4) << 24);
        bool ok = true;
        for (int u = 0; u < nunits; ++u) {
            const int s = u % TC_ST, r = u / TC_ST;
            if (!mbar_wait(smem_u32(&bar_full[s]), r & 1, abort) ||
                !mbar_wait(smem_u32(&bar_b[s]), r & 1, abort)) {
                ok = false;
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;");
            const uint32_t a0 = sbase + (uint32_t)(s * S::STAGE), a1 = a0 + S::A_BYTES;
            const uint32_t b0 = a0 + 2 * S::A_BYTES, b1 = b0 + S::B_BYTES;
#pragma unroll
            for (int kk = 0; kk < TC_KC / 8; ++kk) {
                const uint32_t o = kk * 256;
                tc_mma(tmem, umma_desc(a0 + o), umma_desc(b0 + o), idesc,
                       (u == 0 && kk == 0) ? 0u : 1u);
                tc_mma(tmem, umma_desc(a0 + o), umma_desc(b1 + o), idesc, 1u);
                tc_mma(tmem, umma_desc(a1 + o), umma_desc(b0 + o), idesc, 1u);
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
    if (warp == 4) {
        if (*abort && lane == 0) mbar_wait_plain(done, 0);
        __syncwarp();
        asm volatile("tcgen05.fence::after_thread_sync;");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                     "r"(S::TMEM_COLS));
    }
}

template <int KP> static size_t tc_smem() { return (size_t)TC_ST * TcShape<KP>::STAGE + 1024; }

bool m2l_tc_supported(int KP)
{
    switch (KP) {
    case 40: return tc_smem<40>() <= 227 * 1024;
    case 56: return tc_smem<56>() <= 227 * 1024;
    case 88: return tc_smem<88>() <= 227 * 1024;
    case 120: return tc_smem<120>() <= 227 * 1024;
    default: return false;
    }
}

size_t m2l_tc_op_bytes(int KP)
{
    switch (KP) {
    case 40: return TcShape<40>::OP_BYTES;
    case 56: return TcShape<56>::OP_BYTES;
    case 88: return TcShape<88>::OP_BYTES;
    case 120: return TcShape<120>::OP_BYTES;
    default: return 0;
    }
}

int m2l_tc_kt(int KP)
{
    switch (KP) {
    case 40: return TcShape<40>::KT;
    case 56: return TcShape<56>::KT;
    case 88: return TcShape<88>::KT;
    case 120: return TcShape<120>::KT;
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
#define M2LOPS(KPV)                                                                            \
    case KPV:                                                                                  \
        note_launch();                                                                         \
        k_m2l_ops<KPV><<<n_off, 256, smem, s>>>(p, D, ldD, it, Bop);                           \
        break;
    switch (KP) {
        M2LOPS(40) M2LOPS(56) M2LOPS(88) M2LOPS(120)
    default: break;
    }
#undef M2LOPS
}

void launch_m2l_tc(int p, int KP, const Tile *tiles, int ntiles, const M2LItem *items, int nitems,
                   const int *tile_item0, const int *tile_nitems, const int *ent_u,
                   const int *ent_src, const float *Q, long long ncell, const float *gk,
                   float *Qs, const float *Bop, const Geom *g, float *Ps, double *V, int *flags,
                   cudaStream_t s)
{
    if (nitems > 0) {
#define M2LTC(KPV)                                                                              \
    case KPV: {                                                                                 \
        typedef TcShape<KPV> S;                                                                 \
        const long long nq = ncell * (S::KT / 4);                                               \
        note_launch();                                                                          \
        k_q_split<KPV><<<(unsigned)((nq + 255) / 256), 256, 0, s>>>(p, ncell, Q, gk, Qs);     \
        size_t smem = tc_smem<KPV>();                                                           \
        cudaFuncSetAttribute(k_m2l_tc<KPV>, cudaFuncAttributeMaxDynamicSharedMemorySize,       \
                             (int)smem);                                                        \
        note_launch();                                                                          \
        k_m2l_tc<KPV><<<nitems, TC_THREADS, smem, s>>>(                                         \
            items, ent_u, ent_src, Qs, ncell * S::KT,                                           \
            reinterpret_cast<const unsigned char *>(Bop), Ps, flags);                           \
    } break;
        switch (KP) {
            M2LTC(40) M2LTC(56) M2LTC(88) M2LTC(120)
        default: break;
        }
#undef M2LTC
    }
    launch_m2l_reduce(p, KP, tiles, ntiles, tile_item0, tile_nitems, Ps, g, V, s);
}

}  // namespace ccfmm
