// p2p.cu -- near field (Eq. H2 as read: field of dipole j at i,
// [3 (m_j.u) u - m_j] / r^3) over each leaf's nearPartners (Appendix,
// updateField), the final unpermute + energy (E = -1/2 sum m.H), and the
// FP64 direct sum used to measure the error of the fast method.
#include "ccfmm_dev.cuh"

#include <stdlib.h>
#include <string.h>

#include <algorithm>

namespace ccfmm {

// sources staged per batch and resident blocks per SM of the FP32 kernels
// (the register budget; FP64 keeps 4); compile-time tunables
#ifndef CCFMM_P2P_CH
#define CCFMM_P2P_CH 1024
#endif
#ifndef CCFMM_P2P_MINB
#define CCFMM_P2P_MINB 6
#endif
#ifndef CCFMM_P2P_UNROLL
#define CCFMM_P2P_UNROLL 4
#endif
constexpr int P2P_T = 128;    // threads per block
constexpr int P2P_CH = CCFMM_P2P_CH;  // sources staged in shared memory per batch
constexpr int P2P_UNROLL = CCFMM_P2P_UNROLL;  // unroll of the pair loop
constexpr int P2P_NE = 256;   // near-list entries whose metadata is staged at once
template <typename real> constexpr int p2p_minb() { return sizeof(real) == 4 ? CCFMM_P2P_MINB : 4; }

template <typename real> __device__ __forceinline__ real rsq(real r2);
// one MUFU operation: separations here are never subnormal, so the
// subnormal-range handling that rsqrtf carries is not needed
template <> __device__ __forceinline__ float rsq<float>(float r2)
{
    float r;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(r2));
    return r;
}
template <> __device__ __forceinline__ double rsq<double>(double r2) { return 1.0 / sqrt(r2); }

// Field of dipole (m) at s on the target t: h += [3 (m.u) u - m] / r^3,
// written as h += r^-3 (3 (m.r) r^-2 r - m).  SELF: the source may sit on the
// target (r = 0), which then contributes nothing.
template <typename real, bool SELF>
__device__ __forceinline__ void dip_pair(real tx, real ty, real tz, real sx, real sy, real sz,
                                         real mx, real my, real mz, real &hx, real &hy, real &hz)
{
    real rx = tx - sx, ry = ty - sy, rz = tz - sz;
    real r2 = rx * rx + ry * ry + rz * rz;
    real ri = rsq<real>(r2);
    if (SELF) ri = r2 > (real)0 ? ri : (real)0;
    real ri2 = ri * ri;
    real ri3 = ri2 * ri;
    real t = (real)3 * (mx * rx + my * ry + mz * rz) * ri2;
    hx += ri3 * (t * rx - mx);
    hy += ri3 * (t * ry - my);
    hz += ri3 * (t * rz - mz);
}

// targets per thread, and whether target groups are padded to whole warps
// (then all lanes of a warp share one stripe of sources: broadcast shared
// loads, uniform loop bounds)
#ifndef CCFMM_P2P_TPT
#define CCFMM_P2P_TPT 2
#endif
#ifndef CCFMM_P2P_WARPS
#define CCFMM_P2P_WARPS 0
#endif
constexpr int P2P_TPT = CCFMM_P2P_TPT;
constexpr bool P2P_WARP_STRIPES = CCFMM_P2P_WARPS != 0;

template <typename real, bool SELF>
__device__ __forceinline__ void p2p_range(const typename vec4<real>::t *sp,
                                          const typename vec2<real>::t *sm, int j0, int j1,
                                          const real (&tx)[P2P_TPT][3], real (&hs)[P2P_TPT][3])
{
#pragma unroll P2P_UNROLL
    for (int j = j0; j < j1; ++j) {
        typename vec4<real>::t s = sp[j];
        typename vec2<real>::t m = sm[j];
#pragma unroll
        for (int i = 0; i < P2P_TPT; ++i)
            dip_pair<real, SELF>(tx[i][0], tx[i][1], tx[i][2], s.x, s.y, s.z, s.w, m.x, m.y,
                                 hs[i][0], hs[i][1], hs[i][2]);
    }
}

// contiguous stripe [j0, j1) of a batch of len sources; the chunk length is
// odd so that lanes of different stripes read different shared-memory banks
__device__ __forceinline__ void stripe_range(int len, int S, int stripe, int &j0, int &j1)
{
    int chunk = ((len + S - 1) / S) | 1;
    j0 = min(len, stripe * chunk);
    j1 = min(len, j0 + chunk);
}

// FP32 near field in packed two-lane arithmetic (f32x2 add/mul/fma): the
// staged sources are stored in pairs, {x0 x1 y0 y1} {z0 z1 mx0 mx1}
// {my0 my1 mz0 mz1}, and each step of the pair loop takes two sources in
// the two lanes against one target whose coordinates are duplicated once.
// The two lanes keep separate sums, added at the end of the range.  An odd
// batch is padded with a source of zero moment at 1e30 (r^2 overflows to
// inf, so r^-1 = 0 and it adds exactly zero).  Compile-time switch
// CCFMM_P2P_X2 (FP32 only; the FP64 path is always scalar).
#ifndef CCFMM_P2P_X2
#define CCFMM_P2P_X2 1
#endif
constexpr bool P2P_X2 = CCFMM_P2P_X2 != 0;

__device__ __forceinline__ float2 f2neg(float2 a) { return make_float2(-a.x, -a.y); }

template <bool SELF>
__device__ __forceinline__ void p2p_range_x2(const float4 (*sq)[3], int u0, int u1,
                                             const float (&tx)[P2P_TPT][3],
                                             float (&hs)[P2P_TPT][3])
{
    float2 tp[P2P_TPT][3], h[P2P_TPT][3];
#pragma unroll
    for (int i = 0; i < P2P_TPT; ++i)
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            tp[i][k] = make_float2(tx[i][k], tx[i][k]);
            h[i][k] = make_float2(0.f, 0.f);
        }
    const float2 three = make_float2(3.f, 3.f);
#pragma unroll P2P_UNROLL
    for (int u = u0; u < u1; ++u) {
        const float4 a = sq[u][0], b = sq[u][1], c = sq[u][2];
        const float2 sx = make_float2(a.x, a.y), sy = make_float2(a.z, a.w);
        const float2 sz = make_float2(b.x, b.y), mx = make_float2(b.z, b.w);
        const float2 my = make_float2(c.x, c.y), mz = make_float2(c.z, c.w);
#pragma unroll
        for (int i = 0; i < P2P_TPT; ++i) {
            const float2 rx = __fadd2_rn(tp[i][0], f2neg(sx));
            const float2 ry = __fadd2_rn(tp[i][1], f2neg(sy));
            const float2 rz = __fadd2_rn(tp[i][2], f2neg(sz));
            const float2 r2 = __ffma2_rn(rz, rz, __ffma2_rn(ry, ry, __fmul2_rn(rx, rx)));
            float2 ri = make_float2(rsq<float>(r2.x), rsq<float>(r2.y));
            if (SELF) {
                ri.x = r2.x > 0.f ? ri.x : 0.f;
                ri.y = r2.y > 0.f ? ri.y : 0.f;
            }
            const float2 ri2 = __fmul2_rn(ri, ri);
            const float2 ri3 = __fmul2_rn(ri2, ri);
            const float2 mr = __ffma2_rn(mz, rz, __ffma2_rn(my, ry, __fmul2_rn(mx, rx)));
            const float2 t = __fmul2_rn(__fmul2_rn(three, mr), ri2);
            h[i][0] = __ffma2_rn(ri3, __ffma2_rn(t, rx, f2neg(mx)), h[i][0]);
            h[i][1] = __ffma2_rn(ri3, __ffma2_rn(t, ry, f2neg(my)), h[i][1]);
            h[i][2] = __ffma2_rn(ri3, __ffma2_rn(t, rz, f2neg(mz)), h[i][2]);
        }
    }
#pragma unroll
    for (int i = 0; i < P2P_TPT; ++i)
#pragma unroll
        for (int k = 0; k < 3; ++k) hs[i][k] += h[i][k].x + h[i][k].y;
}

// the staged-source buffer of p2p_leaf (PCH sources, 24 bytes each), in the
// scalar layout (sp[PCH] positions + first moment component, sm[PCH] the
// other two) or the packed pair layout above
template <typename real, int PCH> struct SrcStage {
    typedef typename vec4<real>::t R4;
    typedef typename vec2<real>::t R2;
    static constexpr bool X2 = P2P_X2 && sizeof(real) == 4;
    unsigned char *base;
    __device__ __forceinline__ void put(int v, const R4 &a, const R2 &m) const
    {
        if constexpr (X2) {
            float *q = reinterpret_cast<float *>(base) + 12 * (v >> 1) + (v & 1);
            q[0] = a.x;
            q[2] = a.y;
            q[4] = a.z;
            q[6] = a.w;
            q[8] = m.x;
            q[10] = m.y;
        } else {
            reinterpret_cast<R4 *>(base)[v] = a;
            reinterpret_cast<R2 *>(base + PCH * sizeof(R4))[v] = m;
        }
    }
    // after the len sources of a batch are staged (one thread)
    __device__ __forceinline__ void pad(int len) const
    {
        if constexpr (X2) {
            if (len & 1) {
                R4 a;
                a.x = a.y = a.z = 1e30f;
                a.w = 0.f;
                R2 m;
                m.x = m.y = 0.f;
                put(len, a, m);
            }
        }
    }
    template <bool SELF>
    __device__ __forceinline__ void range(int len, int S, int stripe,
                                          const real (&tx)[P2P_TPT][3],
                                          real (&hs)[P2P_TPT][3]) const
    {
        int j0, j1;
        if constexpr (X2) {
            stripe_range((len + 1) >> 1, S, stripe, j0, j1);
            p2p_range_x2<SELF>(reinterpret_cast<const float4 (*)[3]>(base), j0, j1, tx, hs);
        } else {
            stripe_range(len, S, stripe, j0, j1);
            p2p_range<real, SELF>(reinterpret_cast<const R4 *>(base),
                                  reinterpret_cast<const R2 *>(base + PCH * sizeof(R4)), j0, j1,
                                  tx, hs);
        }
    }
};

// Smooth field (Eq. H, H = -grad V) of one target from its leaf's Taylor
// coefficients vs[] (column t - 1 holds the multi-index t), x relative to
// the leaf centre:  H_a = -sum_{|m| <= p-1} V_{m+e_a} x^m / m!  (returns the
// three sums; the caller subtracts them).  The order
// P = p is a template parameter: the loops over m = (mx, my, mz) unroll, the
// monomial x^m/m! is one product of the per-axis powers' partial products,
// and each term is three FMAs on broadcast coefficient loads.  The fused
// near-field epilogue and the standalone L2P kernel both use it, so the two
// evaluation paths give the same bits.
template <typename real> struct Sum3 {
    real x, y, z;
};

template <typename real, int P>
__device__ __forceinline__ Sum3<real> l2p_fixed(const real *vs, real x, real y, real z)
{
    real px[P], py[P], pz[P];
    px[0] = py[0] = pz[0] = (real)1;
#pragma unroll
    for (int j = 1; j < P; ++j) {
        const real inv = (real)1 / (real)j;  // j is a compile-time constant here
        px[j] = px[j - 1] * x * inv;
        py[j] = py[j - 1] * y * inv;
        pz[j] = pz[j - 1] * z * inv;
    }
    real s0 = (real)0, s1 = (real)0, s2 = (real)0;
#pragma unroll
    for (int mx = 0; mx < P; ++mx) {
#pragma unroll
        for (int my = 0; my < P - mx; ++my) {
            const real b = px[mx] * py[my];
#pragma unroll
            for (int mz = 0; mz < P - mx - my; ++mz) {
                const real mono = b * pz[mz];
                s0 += vs[midx(mx + 1, my, mz) - 1] * mono;
                s1 += vs[midx(mx, my + 1, mz) - 1] * mono;
                s2 += vs[midx(mx, my, mz + 1) - 1] * mono;
            }
        }
    }
    return Sum3<real>{s0, s1, s2};
}

// the sums of l2p_fixed for a run-time order (the field is H - sums)
template <typename real>
__device__ __forceinline__ Sum3<real> l2p_eval(int p, const real *vs, real x, real y, real z)
{
    switch (p) {
    case 1: return l2p_fixed<real, 1>(vs, x, y, z);
    case 2: return l2p_fixed<real, 2>(vs, x, y, z);
    case 3: return l2p_fixed<real, 3>(vs, x, y, z);
    case 4: return l2p_fixed<real, 4>(vs, x, y, z);
    case 5: return l2p_fixed<real, 5>(vs, x, y, z);
    case 6: return l2p_fixed<real, 6>(vs, x, y, z);
    case 7: return l2p_fixed<real, 7>(vs, x, y, z);
    default: return l2p_fixed<real, 8>(vs, x, y, z);
    }
}

// One block per target leaf; writes H = smooth field (L2P) + near field of
// every dipole of the leaf.
//  * Each thread owns two targets and one stripe (a contiguous chunk) of the
//    staged sources; S = floor(128 / target groups) stripes per batch.
//  * Sources are staged in shared memory relative to the target leaf centre,
//    s_j = l_j - (c_target - c_source), so differences are formed between
//    numbers of leaf-size magnitude; the shift is computed once per near
//    entry in FP64.
//  * The leaf's own dipoles are processed first, with the r = 0 test (a
//    source on the field point contributes nothing, Appendix updateField);
//    no other leaf can hold a point at the target's position.
// Near entries of the complete tree: a partner leaf key at the same level
// and its integer cell offset; the shift is the offset times the leaf widths.
struct UniEnts {
    const int *leaf_start;
    const NearEnt *near;
    double wx, wy, wz;
    int self;
    template <typename R4>
    __device__ __forceinline__ int get(int e, int &st, R4 &sh) const
    {
        NearEnt x = near[e];
        st = leaf_start[x.src];
        sh.x = (decltype(sh.x))((double)x.ox * wx);
        sh.y = (decltype(sh.x))((double)x.oy * wy);
        sh.z = (decltype(sh.x))((double)x.oz * wz);
        sh.w = (decltype(sh.x))0;
        return (x.src == self) ? 0 : leaf_start[x.src + 1] - st;
    }
};

template <typename real, typename Ents, bool L2P, int PT = P2P_T, int PCH = P2P_CH>
__device__ __forceinline__ void p2p_leaf(int p, int t0, int nt, int e0, int e1, const Ents &ents,
                                         const double *Vrow, const typename vec4<real>::t *A,
                                         const typename vec2<real>::t *B,
                                         typename vec4<real>::t *H);

template <typename real, bool L2P>
__device__ __forceinline__ void p2p_body(int p, int KP, int L, const int *leaf_start,
                                         const int2 *near_nl, const NearEnt *near, const Geom *g,
                                         const typename vec4<real>::t *A,
                                         const typename vec2<real>::t *B, const double *V,
                                         typename vec4<real>::t *H, long long key)
{
    const int t0 = leaf_start[key], nt = leaf_start[key + 1] - t0;
    if (nt == 0) return;
    const int2 nlk = near_nl[key];  // (first entry, count) of the leaf's near list
    const long long hid = (1ll << L) + key;
    UniEnts ents{leaf_start, near, g->w[L][0], g->w[L][1], g->w[L][2], (int)key};
    // V == nullptr: near field only (L2P by k_l2p once V is complete)
    p2p_leaf<real, UniEnts, L2P>(p, t0, nt, nlk.x, nlk.x + nlk.y, ents,
                                 V ? V + hid * KP : nullptr, A, B, H);
}

// The near field (and, with Vrow, the smooth field) of one leaf's nt dipoles
// at t0..: its own dipoles first, then the entries e0..e1 of its near list,
// each giving a source range and the shift (target centre - source centre).
// L2P = false compiles the near field alone (Vrow is then ignored): without
// the smooth-field epilogue the kernel needs fewer registers.
template <typename real, typename Ents, bool L2P, int PT, int PCH>
__device__ __forceinline__ void p2p_leaf(int p, int t0, int nt, int e0, int e1, const Ents &ents,
                                         const double *Vrow, const typename vec4<real>::t *A,
                                         const typename vec2<real>::t *B,
                                         typename vec4<real>::t *H)
{
    typedef typename vec4<real>::t R4;
    typedef typename vec2<real>::t R2;
    extern __shared__ __align__(16) unsigned char smraw[];
    R4 *sp = reinterpret_cast<R4 *>(smraw);              // [PCH]
    R2 *sm = reinterpret_cast<R2 *>(sp + PCH);         // [PCH]
    R4 *esh = reinterpret_cast<R4 *>(sm + PCH);        // [P2P_NE] source shift
    int *est = reinterpret_cast<int *>(esh + P2P_NE);     // [P2P_NE] source start
    int *epf = est + P2P_NE;                              // [P2P_NE + 1] prefix of counts
    real *vs = reinterpret_cast<real *>(epf + P2P_NE + 4);  // [KP]
    __shared__ int wsum[PT / 32];
    const SrcStage<real, PCH> stage{smraw};
    static_assert(PCH % 2 == 0, "the packed layout stages sources in pairs");

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int K = nterms(p) - 1;
    const bool with_l2p = L2P && Vrow != nullptr;
    constexpr int NE = 2 * PT < P2P_NE ? 2 * PT : P2P_NE;  // entries per metadata chunk
    if (with_l2p)
        for (int c = tid; c < K; c += PT) vs[c] = (real)Vrow[c];

    for (int tb = 0; tb < nt; tb += P2P_TPT * PT) {
        const int ntc = min(nt - tb, P2P_TPT * PT);
        const int ngrp = P2P_WARP_STRIPES ? 32 * ((ntc + 32 * P2P_TPT - 1) / (32 * P2P_TPT))
                                          : (ntc + P2P_TPT - 1) / P2P_TPT;
        const int S = max(1, PT / ngrp);
        const int q = tid % ngrp, stripe = tid / ngrp;
        const bool active = stripe < S;
        const int i0 = tb + P2P_TPT * q;
        real tx[P2P_TPT][3], hs[P2P_TPT][3];
#pragma unroll
        for (int i = 0; i < P2P_TPT; ++i) {
            R4 a = A[t0 + min(i0 + i, tb + ntc - 1)];
            tx[i][0] = a.x;
            tx[i][1] = a.y;
            tx[i][2] = a.z;
            hs[i][0] = hs[i][1] = hs[i][2] = (real)0;
        }

        // 1) the leaf's own dipoles (shift 0), r = 0 possible
        for (int b0 = 0; b0 < nt; b0 += PCH) {
            const int len = min(PCH, nt - b0);
            __syncthreads();
            for (int v = tid; v < len; v += PT) stage.put(v, A[t0 + b0 + v], B[t0 + b0 + v]);
            if (tid == 0) stage.pad(len);
            __syncthreads();
            if (active) stage.template range<true>(len, S, stripe, tx, hs);
        }
        // 2) the other near leaves, in chunks of NE entries (each thread
        // stages the metadata of two entries of a chunk)
        for (int ec = e0; ec < e1; ec += NE) {
            const int nec = min(NE, e1 - ec);
            __syncthreads();
            int c0 = 0, c1 = 0;
            for (int r = 0; r < 2; ++r) {
                int e = 2 * tid + r;
                int cnt = 0;
                if (e < nec) {
                    int st;
                    R4 sh;
                    cnt = ents.get(ec + e, st, sh);
                    est[e] = st;
                    esh[e] = sh;
                }
                if (r == 0) c0 = cnt; else c1 = cnt;
            }
            // exclusive prefix of the counts (two per thread)
            int v = c0 + c1, x = v;
            for (int o = 1; o < 32; o <<= 1) {
                int y = __shfl_up_sync(0xffffffffu, x, o);
                if (lane >= o) x += y;
            }
            if (lane == 31) wsum[warp] = x;
            __syncthreads();
            int base = 0;
            for (int w = 0; w < warp; ++w) base += wsum[w];
            int ex = base + x - v;
            if (2 * tid < nec) epf[2 * tid] = ex;
            if (2 * tid + 1 < nec) epf[2 * tid + 1] = ex + c0;
            if (tid == 0) {
                int tot = 0;
                for (int w = 0; w < PT / 32; ++w) tot += wsum[w];
                epf[nec] = tot;
            }
            __syncthreads();
            const int total = epf[nec];
            for (int b0 = 0; b0 < total; b0 += PCH) {
                const int len = min(PCH, total - b0);
                if (b0) __syncthreads();
                for (int e = warp; e < nec; e += PT / 32) {
                    int lo = max(epf[e], b0), hi = min(epf[e + 1], b0 + len);
                    if (lo >= hi) continue;
                    int off = est[e] - epf[e];
                    R4 sh = esh[e];
                    for (int gv = lo + lane; gv < hi; gv += 32) {
                        R4 a = A[off + gv];
                        R4 o;
                        o.x = a.x - sh.x;
                        o.y = a.y - sh.y;
                        o.z = a.z - sh.z;
                        o.w = a.w;
                        stage.put(gv - b0, o, B[off + gv]);
                    }
                }
                if (tid == 0) stage.pad(len);
                __syncthreads();
                if (active) stage.template range<false>(len, S, stripe, tx, hs);
                __syncthreads();
            }
        }
        // 3) reduce the stripes, add the smooth field, store
        __syncthreads();
        real *red = reinterpret_cast<real *>(sp);
#pragma unroll
        for (int i = 0; i < P2P_TPT; ++i)
#pragma unroll
            for (int k = 0; k < 3; ++k) red[(3 * P2P_TPT) * tid + 3 * i + k] = hs[i][k];
        __syncthreads();
        real f[P2P_TPT][3];
#pragma unroll
        for (int i = 0; i < P2P_TPT; ++i) f[i][0] = f[i][1] = f[i][2] = (real)0;
        if (tid < ngrp) {
            for (int st = 0; st < S; ++st) {
                const real *rr = red + (3 * P2P_TPT) * (st * ngrp + tid);
#pragma unroll
                for (int i = 0; i < P2P_TPT; ++i)
#pragma unroll
                    for (int k = 0; k < 3; ++k) f[i][k] += rr[3 * i + k];
            }
        }
        __syncthreads();
        if (tid < ngrp) {
#pragma unroll
            for (int i = 0; i < P2P_TPT; ++i) {
                if (with_l2p) {
                    const Sum3<real> sl = l2p_eval<real>(p, vs, tx[i][0], tx[i][1], tx[i][2]);
                    f[i][0] -= sl.x;
                    f[i][1] -= sl.y;
                    f[i][2] -= sl.z;
                }
                R4 o;
                o.x = f[i][0];
                o.y = f[i][1];
                o.z = f[i][2];
                o.w = (real)0;
                if (i0 + i < tb + ntc) H[t0 + i0 + i] = o;
            }
        }
    }
}

template <typename real, bool L2P>
__global__ void __launch_bounds__(P2P_T, p2p_minb<real>())
    k_p2p(int p, int KP, int L, const int *leaf_start, const int2 *near_nl, const NearEnt *near,
          const Geom *g, const typename vec4<real>::t *A, const typename vec2<real>::t *B,
          const double *V, typename vec4<real>::t *H)
{
    p2p_body<real, L2P>(p, KP, L, leaf_start, near_nl, near, g, A, B, V, H, blockIdx.x);
}

// Near entries of the adaptive-depth tree: a partner leaf cell of any
// level; the shift is the difference of the two cells' centres, in FP64.
struct AdaEnts {
    const int *p0, *np, *src;
    const double4 *cen;
    double cx, cy, cz;
    int self;
    template <typename R4>
    __device__ __forceinline__ int get(int e, int &st, R4 &sh) const
    {
        const int b = src[e];
        const double4 c = cen[b];
        st = p0[b];
        sh.x = (decltype(sh.x))(cx - c.x);
        sh.y = (decltype(sh.x))(cy - c.y);
        sh.z = (decltype(sh.x))(cz - c.z);
        sh.w = (decltype(sh.x))0;
        return b == self ? 0 : np[b];
    }
};

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
constexpr int L2P_W = 4;  // leaves (warps) per block

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
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    constexpr int K = nterms(P) - 1;
    const int li = blockIdx.x * L2P_W + w;
    if (li >= nleaf) return;
    const int c = leaves[li];
    const int t0 = p0[c], nt = np[c];
    for (int k = lane; k < K; k += 32) vs[w][k] = (real)V[(long long)c * KP + k];
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
