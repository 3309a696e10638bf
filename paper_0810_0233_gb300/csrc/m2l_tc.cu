// m2l_tc.cu -- M2L (Eq. taylorcalc) on the fifth-generation tensor cores.
//
// Same work decomposition as k_m2l_f32 (items = runs of at most M2L_EC
// offset entries of one tile of 128 same-parity cells), but each entry's
// contraction  acc[t][n] += sum_k Q_k(partner of t) * M[n][k],
// M[n][k] = D~_{n+k} h^(1-|k|),  is a tcgen05 MMA with M = 128 (cells),
// N = coefficients n (padded to a multiple of 16), K = coefficients k
// (padded to chunks of 48), accumulated in tensor memory over all entries of
// the item.  FP32 accuracy from TF32 operands: x = x_hi + x_lo with
// x_hi = x rounded to TF32 (cvt.rna) and x_lo = x - x_hi exactly, and
// A B ~ A_hi B_hi + A_hi B_lo + A_lo B_hi (three MMAs per k-step).
//
// Shared memory operands use the no-swizzle K-major canonical layout: core
// matrices of 8 rows x 16 bytes (4 TF32), adjacent along K at 128 bytes
// (leading-dimension offset), 8-row groups at SBO = 12 x 128 bytes.
// Pipeline unit = (entry, K chunk); two stages, so the gather and operand
// build of a unit overlap the MMAs of the previous one; the MMA issue is one
// thread, completion is tracked with one mbarrier per stage.  Every wait is
// bounded: on time-out the kernel raises FLAG_TIMEOUT, drains its copies,
// frees its tensor memory and returns.
#include "ccfmm_dev.cuh"

namespace ccfmm {

constexpr int TC_M = 128;    // field cells per tile (MMA M = TMEM lanes)
constexpr int TC_KC = 48;    // K per pipeline unit (6 MMA k-steps of 8)
constexpr int TC_THREADS = 128;
constexpr long long TC_SPIN = 1ll << 24;

template <int KP> struct TcShape {
    static constexpr int N = ((KP + 15) / 16) * 16;             // MMA N
    static constexpr int KT = ((KP + TC_KC - 1) / TC_KC) * TC_KC;  // padded K
    static constexpr int NCH = KT / TC_KC;                      // K chunks per entry
    static constexpr int SBO = (TC_KC / 4) * 128;               // 8-row group stride, bytes
    static constexpr int A_BYTES = TC_M * TC_KC * 4;
    static constexpr int B_BYTES = N * TC_KC * 4;
    static constexpr int STAGE = 2 * A_BYTES + 2 * B_BYTES;
    static constexpr int TMEM_COLS = N <= 32 ? 32 : (N <= 64 ? 64 : (N <= 128 ? 128 : 256));
};

__device__ __forceinline__ uint32_t smem_u32(const void *p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ uint64_t umma_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo)
{
    uint64_t d = 0;
    d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
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
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(dst), "l"(src), "r"(bytes));
}

__device__ __forceinline__ bool mbar_wait(uint32_t addr, uint32_t parity)
{
    for (long long i = 0; i < TC_SPIN; ++i) {
        uint32_t ok;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
            " selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(ok)
            : "r"(addr), "r"(parity)
            : "memory");
        if (ok) return true;
    }
    return false;
}

__device__ __forceinline__ void tc_mma(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc,
                                       uint32_t acc)
{
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(acc));
}

// byte offset of element (row r, k) inside a no-swizzle K-major chunk
template <int SBO> __device__ __forceinline__ uint32_t core_off(int r, int k)
{
    return (uint32_t)((r & 7) * 16 + (k >> 2) * 128 + (r >> 3) * SBO + (k & 3) * 4);
}

template <int KP>
__global__ void __launch_bounds__(TC_THREADS, 1)
    k_m2l_tc(int p, const Tile *tiles, const M2LItem *items, const int *ent_u,
             const int *ent_src, const float *Q, const float *D, int ldD, const uint16_t *it_g,
             const Geom *g, float *Ps, int *flags)
{
    typedef TcShape<KP> S;
    extern __shared__ __align__(1024) unsigned char smraw[];
    unsigned char *stage0 = smraw;
    float *Dl = reinterpret_cast<float *>(smraw + 2 * S::STAGE);   // [ldD]
    float *gk = Dl + ldD;                                            // [S::KT]
    __shared__ __align__(8) unsigned long long mbar[2];
    __shared__ uint32_t tmem_slot;
    __shared__ int s_abort;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const M2LItem item = items[blockIdx.x];
    const Tile t = tiles[item.tile];
    const int K = nterms(p) - 1;
    const int ne = item.e1 - item.e0;
    const double h = g->h[t.level];
    for (int c = tid; c < S::KT; c += TC_THREADS) {
        double gv = 0.0;
        if (c < K) {
            int nx, ny, nz;
            midx_inv(c + 1, nx, ny, nz);
            gv = pow(h, (double)(1 - (nx + ny + nz)));
        }
        gk[c] = (float)gv;
    }
    if (tid == 0) {
        s_abort = 0;
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar[0])));
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar[1])));
        asm volatile("fence.mbarrier_init.release.cluster;");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(&tmem_slot)),
                     "r"(S::TMEM_COLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tmem = tmem_slot;
    const uint32_t idesc = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(S::N >> 3) << 17) |
                           ((uint32_t)(TC_M >> 4) << 24);

    const int nunits = ne * S::NCH;
    bool ok = true;
    for (int u = 0; u < nunits && ok; ++u) {
        const int s = u & 1, e = u / S::NCH, c = u - e * S::NCH;
        unsigned char *st = stage0 + s * S::STAGE;
        float *Ahi = reinterpret_cast<float *>(st);
        float *Alo = reinterpret_cast<float *>(st + S::A_BYTES);
        unsigned char *Bhi = st + 2 * S::A_BYTES;
        unsigned char *Blo = Bhi + S::B_BYTES;
        // the MMAs of unit u-2 read this stage: wait for them (the decision
        // to give up is taken by the whole block)
        if (u >= 2) {
            bool w = mbar_wait(smem_u32(&mbar[s]), ((u - 2) >> 1) & 1);
            if (!__syncthreads_and(w)) {
                ok = false;
                break;
            }
        }
        const long long row = (long long)item.e0 + e;
        // gather the partners' moment rows for this K chunk (zero beyond K)
        {
            const int *srow = ent_src + row * TT;
            constexpr int CPR = TC_KC / 4;
            for (int i = tid; i < TC_M * CPR; i += TC_THREADS) {
                int r = i / CPR, j = i - r * CPR;
                int col = c * TC_KC + 4 * j;
                int sr = srow[r];
                bool v = sr >= 0 && col < KP;
                const float *src = v ? Q + (long long)sr * KP + col : Q;
                tc_cp16(smem_u32(st) + core_off<S::SBO>(r, 4 * j), src, v ? 16 : 0);
            }
            asm volatile("cp.async.commit_group;\n" ::);
        }
        if (c == 0) {
            const float *Drow = D + (long long)ent_u[row] * ldD;
            for (int i = tid; i < ldD; i += TC_THREADS) Dl[i] = Drow[i];
            __syncthreads();
        }
        // operator tile M[n][k] for this chunk, split into TF32 hi and lo
        for (int i = tid; i < S::N * TC_KC; i += TC_THREADS) {
            int n = i % S::N, kl = i / S::N, k = c * TC_KC + kl;
            float v = 0.f;
            if (n < K && k < K) v = Dl[it_g[k * KP + n]] * gk[k];
            float hi = to_tf32(v);
            uint32_t off = core_off<S::SBO>(n, kl);
            *reinterpret_cast<float *>(Bhi + off) = hi;
            *reinterpret_cast<float *>(Blo + off) = v - hi;
        }
        asm volatile("cp.async.wait_all;\n" ::);
        __syncthreads();
        for (int i = tid; i < TC_M * TC_KC; i += TC_THREADS) {
            float x = Ahi[i];
            float hi = to_tf32(x);
            Ahi[i] = hi;
            Alo[i] = x - hi;
        }
        asm volatile("fence.proxy.async.shared::cta;");
        __syncthreads();
        if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;");
            const uint32_t a0 = smem_u32(Ahi), a1 = smem_u32(Alo);
            const uint32_t b0 = smem_u32(Bhi), b1 = smem_u32(Blo);
#pragma unroll
            for (int kk = 0; kk < TC_KC / 8; ++kk) {
                const uint32_t o = kk * 256;
                uint32_t acc = (u == 0 && kk == 0) ? 0u : 1u;
                tc_mma(tmem, umma_desc(a0 + o, 128, S::SBO), umma_desc(b0 + o, 128, S::SBO), idesc,
                       acc);
                tc_mma(tmem, umma_desc(a0 + o, 128, S::SBO), umma_desc(b1 + o, 128, S::SBO), idesc,
                       1u);
                tc_mma(tmem, umma_desc(a1 + o, 128, S::SBO), umma_desc(b0 + o, 128, S::SBO), idesc,
                       1u);
            }
            asm volatile(
                "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                    smem_u32(&mbar[s])));
        }
    }
    // wait for the last MMAs, then read the accumulator
    if (ok && nunits > 0) {
        int last = nunits - 1;
        bool w = mbar_wait(smem_u32(&mbar[last & 1]), (last >> 1) & 1);
        if (w && nunits >= 2) w = mbar_wait(smem_u32(&mbar[(last - 1) & 1]), ((last - 1) >> 1) & 1);
        ok = __syncthreads_and(w);
    }
    if (!ok) {
        s_abort = 1;
        atomicOr(flags, FLAG_TIMEOUT);
    }
    asm volatile("cp.async.wait_all;\n" ::);
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    float *out = Ps + ((long long)blockIdx.x * TT + warp * 32 + lane) * KP;
    if (!s_abort) {
#pragma unroll
        for (int c0 = 0; c0 < S::N; c0 += 16) {
            uint32_t r[16];
            if (nunits > 0) {
                uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0;
                asm volatile(
                    "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,"
                    "%12,%13,%14,%15}, [%16];\n"
                    : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]),
                      "=r"(r[6]), "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]),
                      "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
                    : "r"(taddr));
                asm volatile("tcgen05.wait::ld.sync.aligned;");
            } else {
#pragma unroll
                for (int j = 0; j < 16; ++j) r[j] = 0u;
            }
#pragma unroll
            for (int j = 0; j < 16; j += 4)
                if (c0 + j < KP)
                    *reinterpret_cast<float4 *>(out + c0 + j) =
                        make_float4(__uint_as_float(r[j]), __uint_as_float(r[j + 1]),
                                    __uint_as_float(r[j + 2]), __uint_as_float(r[j + 3]));
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                     "r"(S::TMEM_COLS));
}

template <int KP> static size_t tc_smem(int ldD)
{
    return 2 * (size_t)TcShape<KP>::STAGE + sizeof(float) * ((size_t)ldD + TcShape<KP>::KT) + 1024;
}

bool m2l_tc_supported(int KP, int ldD)
{
    switch (KP) {
    case 40: return tc_smem<40>(ldD) <= 227 * 1024;
    case 56: return tc_smem<56>(ldD) <= 227 * 1024;
    case 88: return tc_smem<88>(ldD) <= 227 * 1024;
    case 120: return tc_smem<120>(ldD) <= 227 * 1024;
    default: return false;
    }
}

void launch_m2l_tc(int p, int KP, const Tile *tiles, int ntiles, const M2LItem *items, int nitems,
                   const int *tile_item0, const int *tile_nitems, const int *ent_u,
                   const int *ent_src, const float *Q, const float *D, int ldD, const uint16_t *it,
                   const Geom *g, float *Ps, double *V, int *flags, cudaStream_t s)
{
    if (nitems > 0) {
#define M2LTC(KPV)                                                                              \
    case KPV: {                                                                                 \
        size_t smem = tc_smem<KPV>(ldD);                                                        \
        cudaFuncSetAttribute(k_m2l_tc<KPV>, cudaFuncAttributeMaxDynamicSharedMemorySize,       \
                             (int)smem);                                                        \
        note_launch();                                                                          \
        k_m2l_tc<KPV><<<nitems, TC_THREADS, smem, s>>>(p, tiles, items, ent_u, ent_src, Q, D,  \
                                                       ldD, it, g, Ps, flags);                  \
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
