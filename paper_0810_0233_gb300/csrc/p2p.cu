// p2p.cu -- near field (Eq. H2 as read: field of dipole j at i,
// [3 (m_j.u) u - m_j] / r^3) over each leaf's nearPartners (Appendix,
// updateField), the final unpermute + energy (E = -1/2 sum m.H), and the
// FP64 direct sum used to measure the error of the fast method.  The leaf
// body (p2p_leaf), the pair loops and the L2P sums are in stages.cuh.
#include "ccfmm_dev.cuh"
#include "stages.cuh"

#include <stdlib.h>
#include <string.h>

#include <algorithm>

namespace ccfmm {

template <typename real, bool L2P>
__global__ void __launch_bounds__(P2P_T, p2p_minb<real>())
    k_p2p(int p, int KP, int L, const int *leaf_start, const int2 *near_nl, const NearEnt *near,
          const Geom *g, const typename vec4<real>::t *A, const typename vec2<real>::t *B,
          const double *V, typename vec4<real>::t *H)
{
    p2p_body<real, L2P>(p, KP, L, leaf_start, near_nl, near, g, A, B, V, H, blockIdx.x);
}

// near field + smooth field of the adaptive tree's leaves, one block per
// leaf; PT threads and PCH staged sources (a smaller block for the small
// leaves of adaptive trees: more blocks resident per SM)
template <typename real, bool L2P, int PT, int PCH>
__global__ void __launch_bounds__(PT, p2p_minb<real>() * (P2P_T / PT))
    k_ap2p(int p, int KP, const int *leaves, const int *p0, const int *np, const int *near_first,
           const int *near_num, const int *near_src, const double4 *cen,
           const typename vec4<real>::t *A, const typename vec2<real>::t *B, const double *V,
           typename vec4<real>::t *H)
{
    const int c = leaves[blockIdx.x];
    const double4 cc = cen[c];
    const AdaEnts ents{p0, np, near_src, cen, cc.x, cc.y, cc.z, c};
    const int e0 = near_first[c];
    p2p_leaf<real, AdaEnts, L2P, PT, PCH>(p, p0[c], np[c], e0, e0 + near_num[c], ents,
                                          V ? V + (long long)c * KP : nullptr, A, B, H);
}

template <typename real, int PT, int PCH>
static void run_ap2p(int p, int KP, int nleaf, const int *leaves, const int *p0, const int *np,
                     const int *near_first, const int *near_num, const int *near_src,
                     const double4 *cen, const typename vec4<real>::t *A,
                     const typename vec2<real>::t *B, const double *V, typename vec4<real>::t *H,
                     cudaStream_t s)
{
    static_assert(PCH * 4 >= 3 * P2P_TPT * PT, "the stripe sums reuse the staging buffer");
    const size_t smem = (size_t)PCH * (sizeof(typename vec4<real>::t) + sizeof(typename vec2<real>::t)) +
                        (size_t)P2P_NE * sizeof(typename vec4<real>::t) + (2 * P2P_NE + 4) * sizeof(int) +
                        (size_t)KP * sizeof(real) + 64;
    note_launch();
    if (V) {
        cudaFuncSetAttribute(k_ap2p<real, true, PT, PCH>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        k_ap2p<real, true, PT, PCH><<<(unsigned)nleaf, PT, smem, s>>>(
            p, KP, leaves, p0, np, near_first, near_num, near_src, cen, A, B, V, H);
    } else {
        cudaFuncSetAttribute(k_ap2p<real, false, PT, PCH>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        k_ap2p<real, false, PT, PCH><<<(unsigned)nleaf, PT, smem, s>>>(
            p, KP, leaves, p0, np, near_first, near_num, near_src, cen, A, B, V, H);
    }
}

// block shape of the adaptive near field: 128 threads and 1536 staged
// sources (the complete tree's; default), or CCFMM_AP2P=64 (64 threads, 768
// sources: more blocks per SM, measured slower on the ensemble)
static int ap2p_threads()
{
    static int v = -1;
    if (v < 0) {
        const char *e = getenv("CCFMM_AP2P");
        v = (e && atoi(e) == 64) ? 64 : 128;
    }
    return v;
}

template <typename real>
void launch_ap2p(int p, int KP, int nleaf, const int *leaves, const int *p0, const int *np,
                 const int *near_first, const int *near_num, const int *near_src,
                 const double4 *cen, const typename vec4<real>::t *A,
                 const typename vec2<real>::t *B, const double *V, typename vec4<real>::t *H,
                 cudaStream_t s)
{
    if (nleaf <= 0) return;
    if (ap2p_threads() == 128)
        run_ap2p<real, P2P_T, P2P_CH>(p, KP, nleaf, leaves, p0, np, near_first, near_num,
                                      near_src, cen, A, B, V, H, s);
    else
        run_ap2p<real, 64, P2P_CH / 2>(p, KP, nleaf, leaves, p0, np, near_first, near_num,
                                       near_src, cen, A, B, V, H, s);
}

template void launch_ap2p<float>(int, int, int, const int *, const int *, const int *, const int *,
                                 const int *, const int *, const double4 *, const float4 *,
                                 const float2 *, const double *, float4 *, cudaStream_t);
template void launch_ap2p<double>(int, int, int, const int *, const int *, const int *,
                                  const int *, const int *, const int *, const double4 *,
                                  const double4 *, const double2 *, const double *, double4 *,
                                  cudaStream_t);

// every member's leaves in one launch (ensemble step), near field alone
// (the members' V are not read: the smooth field follows by k_l2p_batch);
// at most 5 blocks per SM: with the member's argument record it spills at 6
constexpr int P2P_MINB_BATCH = CCFMM_P2P_MINB > 5 ? 5 : CCFMM_P2P_MINB;
__global__ void __launch_bounds__(P2P_T, P2P_MINB_BATCH)
    k_p2p_batch(const P2PArgs *a, const int *bstart, int nm)
{
    int key;
    const P2PArgs &x = a[batch_member(bstart, nm, blockIdx.x, key)];
    p2p_body<float, false>(x.p, x.KP, x.L, x.leaf_start, x.near_nl, x.near, x.g, x.A, x.B,
                           nullptr, x.H, key);
}

void launch_p2p_batch(const P2PArgs *d_args, const int *d_bstart, int nm, int nblocks, int KP,
                      cudaStream_t s)
{
    if (nblocks <= 0) return;
    const size_t smem = (size_t)P2P_CH * (sizeof(float4) + sizeof(float2)) +
                        (size_t)P2P_NE * sizeof(float4) + (2 * P2P_NE + 4) * sizeof(int) +
                        (size_t)KP * sizeof(float) + 64;
    cudaFuncSetAttribute(k_p2p_batch, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    note_launch();
    k_p2p_batch<<<(unsigned)nblocks, P2P_T, smem, s>>>(d_args, d_bstart, nm);
}

// ------------------------------------------- symmetric near field (variant)
// Newton's third law: the pair (i, j) of leaves A and B gives the field of j
// at i and of i at j (Eq. H2 as read is symmetric in that sense:
// r -> -r leaves [3 (m.u) u - m] / r^3 unchanged), and the offset, r^2,
// the rsqrt and r^-3 are shared by both directions.  The block of leaf A
// takes its own leaf one-sided (as k_p2p) and every near leaf B with a
// larger key both ways; the leaves with smaller keys reach A through their
// own blocks.  The field at B's dipoles is summed per staged source in
// shared memory (shared atomics; within a stripe the threads of different
// target groups visit the sources in rotated order, so that they seldom
// meet on one source) and then added to H with one vector global reduction
// per source; A's own fields are added the same way.  H must be zero before
// the launch, the smooth field is added afterwards (k_l2p), and the order of
// the global additions is not fixed: results vary in the last bits from run
// to run.  Selected by CCFMM_P2P=sym (FP32, near/far overlap on).
#ifndef CCFMM_P2PS_CH
#define CCFMM_P2PS_CH 1024
#endif
constexpr int P2PS_CH = CCFMM_P2PS_CH;

__device__ __forceinline__ void red_add4(float4 *p, float a, float b, float c)
{
    asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(p), "f"(a), "f"(b), "f"(c),
                 "f"(0.f)
                 : "memory");
}

__global__ void __launch_bounds__(P2P_T, 4)
    k_p2p_sym(int L, const int *leaf_start, const int2 *near_nl, const NearEnt *near,
              const Geom *g, const float4 *A, const float2 *B, float4 *H)
{
    extern __shared__ __align__(16) unsigned char smraw[];
    float4 *sp = reinterpret_cast<float4 *>(smraw);              // [P2PS_CH]
    float2 *sm = reinterpret_cast<float2 *>(sp + P2PS_CH);       // [P2PS_CH]
    float *acc = reinterpret_cast<float *>(sm + P2PS_CH);        // [3 P2PS_CH]
    int *sidx = reinterpret_cast<int *>(acc + 3 * P2PS_CH);      // [P2PS_CH]
    float4 *esh = reinterpret_cast<float4 *>(sidx + P2PS_CH);    // [P2P_NE]
    int *est = reinterpret_cast<int *>(esh + P2P_NE);            // [P2P_NE]
    int *epf = est + P2P_NE;                                     // [P2P_NE + 1]
    __shared__ int wsum[P2P_T / 32];

    const long long key = blockIdx.x;
    const int t0 = leaf_start[key], nt = leaf_start[key + 1] - t0;
    if (nt == 0) return;
    const int2 nlk = near_nl[key];
    const int e0 = nlk.x, e1 = nlk.x + nlk.y;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const double wx = g->w[L][0], wy = g->w[L][1], wz = g->w[L][2];

    for (int tb = 0; tb < nt; tb += 2 * P2P_T) {
        const int ntc = min(nt - tb, 2 * P2P_T);
        const int ngrp = (ntc + 1) / 2;
        const int S = max(1, P2P_T / ngrp);
        const int q = tid % ngrp, stripe = tid / ngrp;
        const bool active = stripe < S;
        const int i0 = tb + 2 * q;
        // a padded second target (odd ntc) repeats the first with zero moment,
        // so that it adds nothing to the sources
        const bool two = i0 + 1 < tb + ntc;
        float tx[2][3], tm[2][3], hs[2][3];
#pragma unroll
        for (int i = 0; i < 2; ++i) {
            const int ti = t0 + min(i0 + i, tb + ntc - 1);
            const float4 a = A[ti];
            const float2 b = B[ti];
            const bool live = i == 0 || two;
            tx[i][0] = a.x;
            tx[i][1] = a.y;
            tx[i][2] = a.z;
            tm[i][0] = live ? a.w : 0.f;
            tm[i][1] = live ? b.x : 0.f;
            tm[i][2] = live ? b.y : 0.f;
            hs[i][0] = hs[i][1] = hs[i][2] = 0.f;
        }
        // 1) the leaf's own dipoles, one-sided, r = 0 possible
        for (int b0 = 0; b0 < nt; b0 += P2PS_CH) {
            const int len = min(P2PS_CH, nt - b0);
            __syncthreads();
            for (int v = tid; v < len; v += P2P_T) {
                sp[v] = A[t0 + b0 + v];
                sm[v] = B[t0 + b0 + v];
            }
            __syncthreads();
            if (active) {
                int j0, j1;
                stripe_range(len, S, stripe, j0, j1);
                p2p_range<float, true>(sp, sm, j0, j1, tx, hs);
            }
        }
        // 2) near leaves with a larger key, both directions
        for (int ec = e0; ec < e1; ec += P2P_NE) {
            const int nec = min(P2P_NE, e1 - ec);
            __syncthreads();
            int c0 = 0, c1 = 0;
            for (int r = 0; r < 2; ++r) {
                const int e = 2 * tid + r;
                int cnt = 0;
                if (e < nec) {
                    const NearEnt x = near[ec + e];
                    const int st = leaf_start[x.src];
                    cnt = (x.src > (int)key) ? leaf_start[x.src + 1] - st : 0;
                    est[e] = st;
                    esh[e] = make_float4((float)((double)x.ox * wx), (float)((double)x.oy * wy),
                                         (float)((double)x.oz * wz), 0.f);
                }
                if (r == 0) c0 = cnt; else c1 = cnt;
            }
            const int v = c0 + c1;
            int x = v;
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, x, o);
                if (lane >= o) x += y;
            }
            if (lane == 31) wsum[warp] = x;
            __syncthreads();
            int base = 0;
            for (int w = 0; w < warp; ++w) base += wsum[w];
            const int ex = base + x - v;
            if (2 * tid < nec) epf[2 * tid] = ex;
            if (2 * tid + 1 < nec) epf[2 * tid + 1] = ex + c0;
            if (tid == 0) {
                int tot = 0;
                for (int w = 0; w < P2P_T / 32; ++w) tot += wsum[w];
                epf[nec] = tot;
            }
            __syncthreads();
            const int total = epf[nec];
            for (int b0 = 0; b0 < total; b0 += P2PS_CH) {
                const int len = min(P2PS_CH, total - b0);
                if (b0) __syncthreads();
                for (int e = warp; e < nec; e += P2P_T / 32) {
                    const int lo = max(epf[e], b0), hi = min(epf[e + 1], b0 + len);
                    if (lo >= hi) continue;
                    const int off = est[e] - epf[e];
                    const float4 sh = esh[e];
                    for (int gv = lo + lane; gv < hi; gv += 32) {
                        const float4 a = A[off + gv];
                        sp[gv - b0] = make_float4(a.x - sh.x, a.y - sh.y, a.z - sh.z, a.w);
                        sm[gv - b0] = B[off + gv];
                        sidx[gv - b0] = off + gv;
                        acc[3 * (gv - b0)] = acc[3 * (gv - b0) + 1] = acc[3 * (gv - b0) + 2] = 0.f;
                    }
                }
                __syncthreads();
                if (active) {
                    int j0, j1;
                    stripe_range(len, S, stripe, j0, j1);
                    const int ls = j1 - j0;
                    int j = ls > 0 ? j0 + q % ls : j0;
                    for (int k = 0; k < ls; ++k) {
                        const float4 s4 = sp[j];
                        const float2 m2 = sm[j];
                        float rv0 = 0.f, rv1 = 0.f, rv2 = 0.f;
#pragma unroll
                        for (int i = 0; i < 2; ++i) {
                            const float rx = tx[i][0] - s4.x, ry = tx[i][1] - s4.y,
                                        rz = tx[i][2] - s4.z;
                            const float r2 = rx * rx + ry * ry + rz * rz;
                            const float ri = rsq<float>(r2);
                            const float ri2 = ri * ri, ri3 = ri2 * ri;
                            // field of j at target i
                            const float t = 3.f * (s4.w * rx + m2.x * ry + m2.y * rz) * ri2;
                            hs[i][0] += ri3 * (t * rx - s4.w);
                            hs[i][1] += ri3 * (t * ry - m2.x);
                            hs[i][2] += ri3 * (t * rz - m2.y);
                            // field of target i at j (the same expression in -r)
                            const float u = 3.f * (tm[i][0] * rx + tm[i][1] * ry + tm[i][2] * rz) * ri2;
                            rv0 += ri3 * (u * rx - tm[i][0]);
                            rv1 += ri3 * (u * ry - tm[i][1]);
                            rv2 += ri3 * (u * rz - tm[i][2]);
                        }
                        atomicAdd(&acc[3 * j], rv0);
                        atomicAdd(&acc[3 * j + 1], rv1);
                        atomicAdd(&acc[3 * j + 2], rv2);
                        j = (j + 1 == j1) ? j0 : j + 1;
                    }
                }
                __syncthreads();
                for (int v2 = tid; v2 < len; v2 += P2P_T)
                    red_add4(H + sidx[v2], acc[3 * v2], acc[3 * v2 + 1], acc[3 * v2 + 2]);
                __syncthreads();
            }
        }
        // 3) reduce the stripes; add the targets' fields to H
        __syncthreads();
        float *red = reinterpret_cast<float *>(sp);
#pragma unroll
        for (int i = 0; i < 2; ++i)
#pragma unroll
            for (int k = 0; k < 3; ++k) red[6 * tid + 3 * i + k] = hs[i][k];
        __syncthreads();
        if (tid < ngrp) {
            float f[2][3] = {{0.f, 0.f, 0.f}, {0.f, 0.f, 0.f}};
            for (int st = 0; st < S; ++st) {
                const float *rr = red + 6 * (st * ngrp + tid);
#pragma unroll
                for (int i = 0; i < 2; ++i)
#pragma unroll
                    for (int k = 0; k < 3; ++k) f[i][k] += rr[3 * i + k];
            }
            red_add4(H + t0 + i0, f[0][0], f[0][1], f[0][2]);
            if (two) red_add4(H + t0 + i0 + 1, f[1][0], f[1][1], f[1][2]);
        }
    }
}

bool p2p_symmetric()
{
    const char *e = getenv("CCFMM_P2P");
    return e && !strcmp(e, "sym");
}

void launch_p2p_sym(int L, const int *leaf_start, const int2 *near_nl, const NearEnt *near,
                    const Geom *d_geom, const float4 *A, const float2 *B, float4 *H,
                    long long N, cudaStream_t s)
{
    const size_t smem = (size_t)P2PS_CH * (16 + 8 + 12 + 4) + (size_t)P2P_NE * 16 +
                        (2 * P2P_NE + 4) * sizeof(int) + 64;
    static_assert(P2PS_CH * 4 >= 6 * P2P_T, "the stripe sums reuse the staging buffer");
    cudaMemsetAsync(H, 0, sizeof(float4) * (size_t)N, s);
    cudaFuncSetAttribute(k_p2p_sym, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    note_launch();
    k_p2p_sym<<<(unsigned)(1ll << L), P2P_T, smem, s>>>(L, leaf_start, near_nl, near, d_geom, A,
                                                         B, H);
}

template <typename real>
void launch_p2p(int p, int KP, int L, const int *leaf_start, const int2 *near_nl,
                const NearEnt *near, const Geom *d_geom, const typename vec4<real>::t *A,
                const typename vec2<real>::t *B, const double *V, typename vec4<real>::t *H,
                cudaStream_t s)
{
    size_t smem = (size_t)P2P_CH * (sizeof(typename vec4<real>::t) + sizeof(typename vec2<real>::t)) +
                  (size_t)P2P_NE * sizeof(typename vec4<real>::t) + (2 * P2P_NE + 4) * sizeof(int) +
                  (size_t)KP * sizeof(real) + 64;
    static_assert(P2P_CH * 4 >= 3 * P2P_TPT * P2P_T, "the stripe sums reuse the staging buffer");
    note_launch();
    if (V) {
        cudaFuncSetAttribute(k_p2p<real, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem);
        k_p2p<real, true><<<(unsigned)(1ll << L), P2P_T, smem, s>>>(p, KP, L, leaf_start, near_nl,
                                                                   near, d_geom, A, B, V, H);
    } else {
        cudaFuncSetAttribute(k_p2p<real, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem);
        k_p2p<real, false><<<(unsigned)(1ll << L), P2P_T, smem, s>>>(p, KP, L, leaf_start,
                                                                    near_nl, near, d_geom, A, B,
                                                                    nullptr, H);
    }
}

// L2P (Eq. H, H = -grad V) of every dipole of a leaf (one warp per leaf),
// added to the near field that k_p2p stored without its fused L2P: the same
// operations in the same order as the fused epilogue.

template <typename real, int P>
__device__ __forceinline__ void l2p_body(int KP, int L, const int *leaf_start,
                                         const typename vec4<real>::t *A, const double *V,
                                         typename vec4<real>::t *H, long long blk)
{
    __shared__ real vs[L2P_W][nterms(PMAX)];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    constexpr int K = nterms(P) - 1;
    const long long key = blk * L2P_W + w;
    const bool live = key < (1ll << L);
    const int t0 = live ? leaf_start[key] : 0, nt = live ? leaf_start[key + 1] - t0 : 0;
    const long long hid = (1ll << L) + key;
    if (nt > 0)
        for (int c = lane; c < K; c += 32) vs[w][c] = (real)V[hid * KP + c];
    __syncwarp();
    for (int i = lane; i < nt; i += 32) {
        const typename vec4<real>::t a = A[t0 + i];
        typename vec4<real>::t h = H[t0 + i];
        const Sum3<real> sl = l2p_fixed<real, P>(vs[w], a.x, a.y, a.z);
        h.x -= sl.x;
        h.y -= sl.y;
        h.z -= sl.z;
        H[t0 + i] = h;
    }
}

template <typename real, int P>
__global__ void __launch_bounds__(32 * L2P_W) k_l2p(int KP, int L, const int *leaf_start,
                                                    const typename vec4<real>::t *A,
                                                    const double *V, typename vec4<real>::t *H)
{
    l2p_body<real, P>(KP, L, leaf_start, A, V, H, blockIdx.x);
}

// L2P of the adaptive tree's leaf cells (one warp per leaf), added to the
// near field that k_ap2p stored without the smooth field
template <typename real, int P>
__global__ void __launch_bounds__(32 * L2P_W) k_al2p(int KP, int nleaf, const int *leaves,
                                                     const int *p0, const int *np,
                                                     const typename vec4<real>::t *A,
                                                     const double *V, typename vec4<real>::t *H)
{
    __shared__ real vs[L2P_W][nterms(PMAX)];
    const int w = threadIdx.x >> 5;
    const int li = blockIdx.x * L2P_W + w;
    if (li >= nleaf) return;
    al2p_leaf<real, P>(KP, leaves[li], p0, np, A, V, H, vs[w]);
}

template <typename real>
void launch_al2p(int p, int KP, int nleaf, const int *leaves, const int *p0, const int *np,
                 const typename vec4<real>::t *A, const double *V, typename vec4<real>::t *H,
                 cudaStream_t s)
{
    if (nleaf <= 0) return;
    const unsigned nb = (unsigned)((nleaf + L2P_W - 1) / L2P_W);
    note_launch();
#define AL2P(PV)                                                                                 \
    case PV: k_al2p<real, PV><<<nb, 32 * L2P_W, 0, s>>>(KP, nleaf, leaves, p0, np, A, V, H); break;
    switch (p) {
        AL2P(1) AL2P(2) AL2P(3) AL2P(4) AL2P(5) AL2P(6) AL2P(7) AL2P(8)
    default: break;
    }
#undef AL2P
}

template void launch_al2p<float>(int, int, int, const int *, const int *, const int *,
                                 const float4 *, const double *, float4 *, cudaStream_t);
template void launch_al2p<double>(int, int, int, const int *, const int *, const int *,
                                  const double4 *, const double *, double4 *, cudaStream_t);

// every member's smooth field in one launch (ensemble step)
template <int P>
__global__ void __launch_bounds__(32 * L2P_W) k_l2p_batch(const P2PArgs *a, const int *bstart,
                                                          int nm)
{
    int blk;
    const P2PArgs &x = a[batch_member(bstart, nm, blockIdx.x, blk)];
    l2p_body<float, P>(x.KP, x.L, x.leaf_start, x.A, x.V, x.H, blk);
}

int l2p_blocks(int L) { return (int)(((1ll << L) + L2P_W - 1) / L2P_W); }

void launch_l2p_batch(int p, const P2PArgs *a, const int *bstart, int nm, int nblocks,
                      cudaStream_t s)
{
    if (nblocks <= 0) return;
    note_launch();
#define L2PB(PV)                                                                                 \
    case PV: k_l2p_batch<PV><<<(unsigned)nblocks, 32 * L2P_W, 0, s>>>(a, bstart, nm); break;
    switch (p) {
        L2PB(1) L2PB(2) L2PB(3) L2PB(4) L2PB(5) L2PB(6) L2PB(7) L2PB(8)
    default: break;
    }
#undef L2PB
}

template <typename real>
void launch_l2p(int p, int KP, int L, const int *leaf_start, const typename vec4<real>::t *A,
                const double *V, typename vec4<real>::t *H, cudaStream_t s)
{
    const long long nleaf = 1ll << L;
    const unsigned nb = (unsigned)((nleaf + L2P_W - 1) / L2P_W);
    note_launch();
#define L2PK(PV)                                                                                 \
    case PV: k_l2p<real, PV><<<nb, 32 * L2P_W, 0, s>>>(KP, L, leaf_start, A, V, H); break;
    switch (p) {
        L2PK(1) L2PK(2) L2PK(3) L2PK(4) L2PK(5) L2PK(6) L2PK(7) L2PK(8)
    default: break;
    }
#undef L2PK
}

// unpermute to input order in FP64 and form per-block partial sums of m.H
constexpr int FIN_T = 256;

template <typename real>
__device__ __forceinline__ void finish_body(const typename vec4<real>::t *H, const int *perm,
                                            const double *mom, long long n, double *Hout,
                                            double *partial, long long blk)
{
    __shared__ double red[FIN_T / 32];
    double e = 0.0;
    long long s = blk * FIN_T + threadIdx.x;
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
        partial[blk] = t;
    }
}

template <typename real>
__global__ void __launch_bounds__(FIN_T) k_finish(const typename vec4<real>::t *H, const int *perm,
                                                  const double *mom, long long n, double *Hout,
                                                  double *partial)
{
    finish_body<real>(H, perm, mom, n, Hout, partial, blockIdx.x);
}

// E = -1/2 sum of the partials, summed in a fixed order
__device__ __forceinline__ void energy_body(const double *partial, long long nparts, double *E)
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

__global__ void k_energy_final(const double *partial, long long nparts, double *E)
{
    energy_body(partial, nparts, E);
}

// every member's unpermute + energy partials, then every member's energy
__global__ void __launch_bounds__(FIN_T) k_finish_batch(const FinishArgs *a, const int *bstart,
                                                        int nm)
{
    int blk;
    const FinishArgs &x = a[batch_member(bstart, nm, blockIdx.x, blk)];
    finish_body<float>(x.H, x.perm, x.mom, x.n, x.Hout, x.partial, blk);
}

__global__ void k_energy_batch(const FinishArgs *a)
{
    const FinishArgs &x = a[blockIdx.x];
    energy_body(x.partial, (x.n + FIN_T - 1) / FIN_T, x.E);
}

void launch_finish_batch(const FinishArgs *d_args, const int *d_bstart, int nm, int nblocks,
                         cudaStream_t s)
{
    if (nblocks <= 0) return;
    note_launch(2);
    k_finish_batch<<<(unsigned)nblocks, FIN_T, 0, s>>>(d_args, d_bstart, nm);
    k_energy_batch<<<(unsigned)nm, 256, 0, s>>>(d_args);
}

int finish_blocks(long long n) { return (int)((n + FIN_T - 1) / FIN_T); }

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
__global__ void k_pair_count(int L, const int *leaf_start, const int2 *near_nl,
                             const NearEnt *near, unsigned long long *count)
{
    long long key = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (key >= (1ll << L)) return;
    long long nt = leaf_start[key + 1] - leaf_start[key];
    if (!nt) return;
    long long ns = 0;
    const int2 nlk = near_nl[key];
    for (int e = nlk.x; e < nlk.x + nlk.y; ++e)
        ns += leaf_start[near[e].src + 1] - leaf_start[near[e].src];
    atomicAdd(count, (unsigned long long)(nt * ns - nt));
}

void launch_p2p_pair_count(int L, const int *leaf_start, const int2 *near_nl,
                           const NearEnt *near, unsigned long long *d_count, cudaStream_t s)
{
    cudaMemsetAsync(d_count, 0, sizeof(unsigned long long), s);
    long long n = 1ll << L;
    note_launch();
    k_pair_count<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(L, leaf_start, near_nl, near,
                                                            d_count);
}

#define INST(real)                                                                              \
    template void launch_p2p<real>(int, int, int, const int *, const int2 *, const NearEnt *,  \
                                   const Geom *, const vec4<real>::t *, const vec2<real>::t *,  \
                                   const double *, vec4<real>::t *, cudaStream_t);              \
    template void launch_finish<real>(const vec4<real>::t *, const int *, const double *,       \
                                      long long, double *, double *, double *, cudaStream_t);  \
    template void launch_l2p<real>(int, int, int, const int *, const vec4<real>::t *,           \
                                   const double *, vec4<real>::t *, cudaStream_t);
INST(float)
INST(double)
#undef INST

}  // namespace ccfmm
