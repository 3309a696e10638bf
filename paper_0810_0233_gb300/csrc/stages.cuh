// stages.cuh -- device bodies of the evaluation stages that more than one
// kernel runs: the near field of a leaf and the smooth field (L2P), P2M, the
// adaptive tree's M2M and L2L, the tensor-core M2L items and the moment fold
// of its harmonic reduction, the rotation of the ensemble's moments.  The
// per-stage kernels and the persistent step kernel of the adaptive tree
// (adaptive.cu) call the same bodies, so both give the same arithmetic.
// Bodies whose kernels keep per-block scratch in shared memory take it as an
// argument: the persistent kernel overlays the scratch of all stages in one
// buffer.  Internal to libccfmm.
#pragma once

#include "ccfmm_dev.cuh"

namespace ccfmm {

// ================================================================ near field
// sources staged per batch and resident blocks per SM of the FP32 kernels
// (the register budget; FP64 keeps 4); compile-time tunables
#ifndef CCFMM_P2P_CH
#define CCFMM_P2P_CH 1280
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

// smooth field (L2P) of one leaf cell c of the adaptive tree by one warp,
// added to the near field already in H; vs: the warp's scratch of
// nterms(PMAX) coefficients
constexpr int L2P_W = 4;  // leaves (warps) per block of the L2P kernels

template <typename real, int P>
__device__ __forceinline__ void al2p_leaf(int KP, int c, const int *p0, const int *np,
                                          const typename vec4<real>::t *A, const double *V,
                                          typename vec4<real>::t *H, real *vs)
{
    const int lane = threadIdx.x & 31;
    constexpr int K = nterms(P) - 1;
    const int t0 = p0[c], nt = np[c];
    for (int k = lane; k < K; k += 32) vs[k] = (real)V[(long long)c * KP + k];
    __syncwarp();
    for (int i = lane; i < nt; i += 32) {
        const typename vec4<real>::t a = A[t0 + i];
        typename vec4<real>::t h = H[t0 + i];
        const Sum3<real> sl = l2p_fixed<real, P>(vs, a.x, a.y, a.z);
        h.x -= sl.x;
        h.y -= sl.y;
        h.z -= sl.z;
        H[t0 + i] = h;
    }
}

// ============================================ adaptive M2L on the tensor cores
// ---------------------------------------------------------------------------
// The same contraction on the tensor cores, FP32 path (3xTF32: each operand
// x = hi + lo with hi = tf32(x), lo = tf32(x - hi); A B ~ Alo Bhi + Ahi Blo +
// Ahi Bhi with FP32 accumulation).  The operator of an item is built from
// its D row for 16-row tiles, which the warp-level MMA (mma.sync m16n8k8,
// TF32) takes directly from registers: a warp owns 16 pairs (rows) x all
// KP columns, K in steps of 8; its A fragments are the scaled moments of the
// 16 sources read from global memory, its B fragments M[k][n] = D~_{n+k}.
//   BIG:   one item per block (groups of more than 16 pairs, items of at
//          most 512): the block first stores every B fragment of the item's
//          operator, split, in shared memory (fragment order), then its four
//          warps take the item's 16-pair chunks in turn.
//   SMALL: one item per warp (groups of at most 16 pairs): B fragments are
//          formed from the D row as they are used.
// The contraction runs over the harmonic reduction (moments folded by the
// Laplace identity of the D tensors, (p+1)^2 - 1 columns on either side):
// Q rows, the index table and the accumulator VF are the reduced ones.
// Fragment layouts (PTX ISA, mma.m16n8k8 with .tf32): g = lane / 4,
// t = lane % 4; A: a0 (g, t), a1 (g + 8, t), a2 (g, t + 4), a3 (g + 8, t + 4);
// B: b0 (k = t, n = g), b1 (k = t + 4, n = g); C: c0 (g, 2t), c1 (g, 2t + 1),
// c2 (g + 8, 2t), c3 (g + 8, 2t + 1).
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t tf32_rna(float x)
{
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ void tf32_split(float x, uint32_t &hi, uint32_t &lo)
{
    hi = tf32_rna(x);
    lo = tf32_rna(x - __uint_as_float(hi));
}
__device__ __forceinline__ void mma_tf32(float (&c)[4], const uint32_t (&a)[4], uint32_t b0,
                                         uint32_t b1)
{
    asm("mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
        "{%8,%9}, {%0,%1,%2,%3};"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}
__device__ __forceinline__ void red_add2(float *p, float a, float b)
{
    asm volatile("red.global.add.v2.f32 [%0], {%1, %2};" ::"l"(p), "f"(a), "f"(b) : "memory");
}

// scale tables of one item from its row of rho^-d (d = 0 .. p + 1, formed in
// FP64 at the build), over the reduced columns: gk[c] = rho^-|k|,
// en[c] = (-1)^|n| rho^-(|n|+1) (zero beyond the reduced count); threads
// tid0.. step nth
__device__ __forceinline__ void am2l_scales(int p, int KP, const float *pw, float *gk,
                                            float *en, int tid0, int nth)
{
    const int K = red_count(p);
    for (int c = tid0; c < KP; c += nth) {
        float gv = 0.f, ev = 0.f;
        if (c < K) {
            const int d = red_order(c);
            gv = pw[d];
            ev = (d & 1) ? -pw[d + 1] : pw[d + 1];
        }
        gk[c] = gv;
        en[c] = ev;
    }
}

// 16 pairs (rows) from pair c0 of the item: A from the sources' moments,
// B from bfrag (BIG, fragment order in shared memory) or from Dl and the
// index table; the results added to the targets' accumulators
// compile-time choice of the chunk's instruction order: 0 (default) forms the
// A fragments of one k-step at a time and issues the three passes of each
// column tile together; 1 loads every A element first and issues the passes
// over all column tiles in turn (more registers)
#ifndef CCFMM_AM2L_PRELOAD
#define CCFMM_AM2L_PRELOAD 0
#endif

template <int KP, bool BIG>
__device__ __forceinline__ void am2l_bfrag(int ks, int nt, const float4 *bfrag, const float *Dl,
                                           const uint16_t *its, uint32_t &bh0, uint32_t &bh1,
                                           uint32_t &bl0, uint32_t &bl1)
{
    constexpr int KS = KP / 8;
    const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    if (BIG) {
        const float4 b = bfrag[(ks * KS + nt) * 32 + lane];
        bh0 = __float_as_uint(b.x);
        bh1 = __float_as_uint(b.y);
        bl0 = __float_as_uint(b.z);
        bl1 = __float_as_uint(b.w);
    } else {
        const int k = 8 * ks + t, n = 8 * nt + g;
        tf32_split(Dl[its[k * KP + n]], bh0, bl0);
        tf32_split(Dl[its[(k + 4) * KP + n]], bh1, bl1);
    }
}

template <int KP, bool BIG>
__device__ __forceinline__ void am2l_mma_chunk(const int4 &item, int c0, const int *pt,
                                               const int *ps, const float *Q, const float *gk,
                                               const float *en, const float4 *bfrag,
                                               const float *Dl, const uint16_t *its, float *VF)
{
    constexpr int KS = KP / 8;
    const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    const int r0 = c0 + g, r1 = c0 + g + 8;
    const bool v0 = r0 < item.y, v1 = r1 < item.y;
    const float *q0 = Q + (long long)(v0 ? ps[item.x + r0] : 0) * KP;
    const float *q1 = Q + (long long)(v1 ? ps[item.x + r1] : 0) * KP;
    float c[KS][4];
#pragma unroll
    for (int n = 0; n < KS; ++n) c[n][0] = c[n][1] = c[n][2] = c[n][3] = 0.f;
#if CCFMM_AM2L_PRELOAD
    float x[KS][4];
#pragma unroll
    for (int ks = 0; ks < KS; ++ks) {
        const int col = 8 * ks + t;
        x[ks][0] = v0 ? q0[col] : 0.f;
        x[ks][1] = v1 ? q1[col] : 0.f;
        x[ks][2] = v0 ? q0[col + 4] : 0.f;
        x[ks][3] = v1 ? q1[col + 4] : 0.f;
    }
#endif
#pragma unroll
    for (int ks = 0; ks < KS; ++ks) {
        const int col = 8 * ks + t;
        const float g0 = gk[col], g4 = gk[col + 4];
#if CCFMM_AM2L_PRELOAD
        const float y0 = x[ks][0], y1 = x[ks][1], y2 = x[ks][2], y3 = x[ks][3];
#else
        const float y0 = v0 ? q0[col] : 0.f, y1 = v1 ? q1[col] : 0.f;
        const float y2 = v0 ? q0[col + 4] : 0.f, y3 = v1 ? q1[col + 4] : 0.f;
#endif
        uint32_t ah[4], al[4];
        tf32_split(y0 * g0, ah[0], al[0]);
        tf32_split(y1 * g0, ah[1], al[1]);
        tf32_split(y2 * g4, ah[2], al[2]);
        tf32_split(y3 * g4, ah[3], al[3]);
#if CCFMM_AM2L_PRELOAD
        uint32_t bh0[KS], bh1[KS], bl0[KS], bl1[KS];
#pragma unroll
        for (int nt = 0; nt < KS; ++nt)
            am2l_bfrag<KP, BIG>(ks, nt, bfrag, Dl, its, bh0[nt], bh1[nt], bl0[nt], bl1[nt]);
#pragma unroll
        for (int nt = 0; nt < KS; ++nt) mma_tf32(c[nt], al, bh0[nt], bh1[nt]);
#pragma unroll
        for (int nt = 0; nt < KS; ++nt) mma_tf32(c[nt], ah, bl0[nt], bl1[nt]);
#pragma unroll
        for (int nt = 0; nt < KS; ++nt) mma_tf32(c[nt], ah, bh0[nt], bh1[nt]);
#else
#pragma unroll
        for (int nt = 0; nt < KS; ++nt) {
            uint32_t bh0, bh1, bl0, bl1;
            am2l_bfrag<KP, BIG>(ks, nt, bfrag, Dl, its, bh0, bh1, bl0, bl1);
            mma_tf32(c[nt], al, bh0, bh1);
            mma_tf32(c[nt], ah, bl0, bl1);
            mma_tf32(c[nt], ah, bh0, bh1);
        }
#endif
    }
    const int t0 = v0 ? pt[item.x + r0] : -1, t1 = v1 ? pt[item.x + r1] : -1;
#pragma unroll
    for (int nt = 0; nt < KS; ++nt) {
        const int col = 8 * nt + 2 * t;
        const float e0 = en[col], e1 = en[col + 1];
        if (t0 >= 0) red_add2(VF + (long long)t0 * KP + col, c[nt][0] * e0, c[nt][1] * e1);
        if (t1 >= 0) red_add2(VF + (long long)t1 * KP + col, c[nt][2] * e0, c[nt][3] * e1);
    }
}

// BIG: one item per block of 128 threads; smraw = the block's shared memory
// (the split B fragments of the item's operator, its D row and scales)
template <int KP>
__device__ __forceinline__ void am2l_big_item(int p, const int4 &item, const int *pt,
                                              const int *ps, const float *rpow, const float *D,
                                              int ldD, const uint16_t *it, const float *Q,
                                              float *VF, unsigned char *smraw)
{
    constexpr int KS = KP / 8;
    float4 *bfrag = reinterpret_cast<float4 *>(smraw);  // [KS * KS * 32]
    float *Dl = reinterpret_cast<float *>(bfrag + KS * KS * 32);  // [ldD]
    float *gk = Dl + ldD, *en = gk + KP;                          // [KP], [KP]
    const int tid = threadIdx.x;
    const float *Drow = D + (long long)item.z * ldD;
    for (int i = tid; i < ldD; i += 128) Dl[i] = Drow[i];
    am2l_scales(p, KP, rpow + (long long)item.z * (PMAX + 2), gk, en, tid, 128);
    __syncthreads();
    for (int idx = tid; idx < KS * KS * 32; idx += 128) {
        const int tile = idx >> 5, ln = idx & 31;
        const int ks = tile / KS, nt = tile - ks * KS;
        const int k = 8 * ks + (ln & 3), n = 8 * nt + (ln >> 2);
        uint32_t h0, l0, h1, l1;
        tf32_split(Dl[it[k * KP + n]], h0, l0);
        tf32_split(Dl[it[(k + 4) * KP + n]], h1, l1);
        bfrag[idx] = make_float4(__uint_as_float(h0), __uint_as_float(h1), __uint_as_float(l0),
                                 __uint_as_float(l1));
    }
    __syncthreads();
    const int warp = tid >> 5;
    for (int c0 = 16 * warp; c0 < item.y; c0 += 64)
        am2l_mma_chunk<KP, true>(item, c0, pt, ps, Q, gk, en, bfrag, Dl, it, VF);
}

template <int KP> constexpr size_t am2l_big_smem(int ldD)
{
    return (size_t)(KP / 8) * (KP / 8) * 32 * sizeof(float4) + sizeof(float) * (ldD + 2 * KP) + 16;
}

// SMALL: items g4 * 4 + warp, one per warp of a 128-thread block, of the
// nitems; smraw: the index table (staged by the whole block) and each
// warp's D row and scales
template <int KP>
__device__ __forceinline__ void am2l_small_items(int p, const int4 *items, int nitems, int g4,
                                                 const int *pt, const int *ps, const float *rpow,
                                                 const float *D, int ldD, const uint16_t *it,
                                                 const float *Q, float *VF, unsigned char *smraw)
{
    uint16_t *its = reinterpret_cast<uint16_t *>(smraw);  // [KP * KP] index table
    float *wbase = reinterpret_cast<float *>(smraw + ((KP * KP * 2 + 15) & ~15));
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int per = ((ldD + 2 * KP) + 3) & ~3;  // floats per warp
    float *Dl = wbase + warp * per;
    float *gk = Dl + ldD, *en = gk + KP;
    for (int i = threadIdx.x; i < KP * KP; i += 128) its[i] = it[i];
    __syncthreads();
    const int ii = g4 * 4 + warp;
    if (ii >= nitems) return;
    const int4 item = items[ii];
    const float *Drow = D + (long long)item.z * ldD;
    for (int i = lane; i < ldD; i += 32) Dl[i] = Drow[i];
    am2l_scales(p, KP, rpow + (long long)item.z * (PMAX + 2), gk, en, lane, 32);
    __syncwarp();
    for (int c0 = 0; c0 < item.y; c0 += 16)
        am2l_mma_chunk<KP, false>(item, c0, pt, ps, Q, gk, en, nullptr, Dl, its, VF);
}

template <int KP> constexpr size_t am2l_small_smem(int ldD)
{
    return ((KP * KP * 2 + 15) & ~15) + sizeof(float) * 4 * (((ldD + 2 * KP) + 3) & ~3) + 16;
}


// fold of one cell's moments (a row of KPF floats) into its reduced row of
// KRP floats (zero padding) by one warp (Laplace identity of the D tensors:
// Q_k with k_z >= 2 moves to k - 2e_z + 2e_x and k - 2e_z + 2e_y with a
// minus sign); row: the warp's scratch of AF_ROW floats
constexpr int AF_ROW = ((nterms(PMAX) - 1 + 7) / 8) * 8;

__device__ __forceinline__ void afold_cell(int p, int KPF, int KRP, long long c, const float *Q,
                                           float *Qr, float *row)
{
    const int lane = threadIdx.x & 31;
    const int K = nterms(p) - 1, KR = red_count(p);
    for (int j = lane; j < K; j += 32) row[j] = Q[c * KPF + j];
    __syncwarp();
    if (lane >= 1 && lane < p) {
        const int k = lane + 1, base = nterms(k - 1) - 1;
        for (int z = k; z >= 2; --z)
            for (int y = 0; y <= k - z; ++y) {
                const float v = row[base + z * (2 * k + 3 - z) / 2 + y];
                const int zt = z - 2, lt = base + zt * (2 * k + 3 - zt) / 2;
                row[lt + y] -= v;      // (x + 2, y, z - 2)
                row[lt + y + 2] -= v;  // (x, y + 2, z - 2)
            }
    }
    __syncwarp();
    for (int r = lane; r < KRP; r += 32) Qr[c * KRP + r] = r < KR ? row[red_full(r)] : 0.f;
}

// ======================================================================= P2M
// multi-indices packed in 5-bit fields (x | y << 5 | z << 10)
__device__ __forceinline__ unsigned pack3(int a, int b, int c)
{
    return (unsigned)a | ((unsigned)b << 5) | ((unsigned)c << 10);
}

// fill an smem table of the coefficient multi-indices mi[c] = index c+1
__device__ __forceinline__ void fill_mi(unsigned *mi, int K)
{
    for (int c = threadIdx.x; c < K; c += blockDim.x) {
        int x, y, z;
        midx_inv(c + 1, x, y, z);
        mi[c] = pack3(x, y, z);
    }
}
__device__ __forceinline__ int px(unsigned v) { return (int)(v & 31u); }
__device__ __forceinline__ int py(unsigned v) { return (int)((v >> 5) & 31u); }
__device__ __forceinline__ int pz(unsigned v) { return (int)((v >> 10) & 31u); }

// P2M (Eq. multipolemoments): Q_n = sum_i sum_a m_ia r_i^(n-e_a)/(n-e_a)!
// about the leaf centre, for every leaf (empty leaves get zeros).
// ---------------------------------------------------------------------------
// One warp per leaf, P2M_W leaves per block: a lane stages one dipole of the
// leaf (powers x^j/j! of its leaf-relative coordinates, by reciprocal
// constants) and then owns coefficients lane, lane + 32, ...
constexpr int P2M_W = 4;
constexpr int P2M_R = (nterms(PMAX) - 1 + 31) / 32;  // coefficient rounds per lane

// the block's shared scratch of p2m_run
template <typename real> struct P2MScratch {
    real pw[P2M_W][32][3][PMAX];  // powers x^j / j! of each staged dipole
    real mm[P2M_W][32][3];        // its moment
    unsigned mi[nterms(PMAX)];    // multi-index table
};

// P2M of the dipoles s0..s1 (coordinates relative to the leaf centre) into
// Qrow[0..KP) by warp w of the block; every thread of the block calls it
// (the multi-index table is filled block-wide), live = false for warps
// without a leaf.
template <typename real>
__device__ __forceinline__ void p2m_run(int p, int KP, bool live, int s0, int s1,
                                        const typename vec4<real>::t *A,
                                        const typename vec2<real>::t *B, real *Qrow,
                                        P2MScratch<real> &sc)
{
    real(*pw)[32][3][PMAX] = sc.pw;
    real(*mm)[32][3] = sc.mm;
    unsigned *mi = sc.mi;
    const real inv[PMAX] = {(real)0, (real)1, (real)0.5, (real)1 / (real)3, (real)0.25,
                            (real)0.2, (real)1 / (real)6, (real)1 / (real)7};
    const int K = nterms(p) - 1;
    fill_mi(mi, K);
    __syncthreads();
    if (!live) return;
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    real acc[P2M_R];
#pragma unroll
    for (int r = 0; r < P2M_R; ++r) acc[r] = (real)0;
    for (int base = s0; base < s1; base += 32) {
        __syncwarp();
        const int i = base + lane;
        if (i < s1) {
            const typename vec4<real>::t a = A[i];
            const typename vec2<real>::t b = B[i];
            const real x[3] = {a.x, a.y, a.z};
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                real v = (real)1;
                pw[w][lane][d][0] = v;
#pragma unroll
                for (int j = 1; j < PMAX; ++j)
                    if (j < p) {
                        v = v * x[d] * inv[j];
                        pw[w][lane][d][j] = v;
                    }
            }
            mm[w][lane][0] = a.w;
            mm[w][lane][1] = b.x;
            mm[w][lane][2] = b.y;
        }
        __syncwarp();
        const int cnt = min(32, s1 - base);
#pragma unroll
        for (int r = 0; r < P2M_R; ++r) {
            const int c = lane + 32 * r;
            if (c < K) {
                const unsigned n = mi[c];
                const int nx = px(n), ny = py(n), nz = pz(n);
                real sum = (real)0;
                for (int d = 0; d < cnt; ++d) {
                    const real(*q)[PMAX] = pw[w][d];
                    if (nx > 0) sum += mm[w][d][0] * q[0][nx - 1] * q[1][ny] * q[2][nz];
                    if (ny > 0) sum += mm[w][d][1] * q[0][nx] * q[1][ny - 1] * q[2][nz];
                    if (nz > 0) sum += mm[w][d][2] * q[0][nx] * q[1][ny] * q[2][nz - 1];
                }
                acc[r] += sum;
            }
        }
    }
#pragma unroll
    for (int r = 0; r < P2M_R; ++r) {
        const int c = lane + 32 * r;
        if (c < KP) Qrow[c] = c < K ? acc[r] : (real)0;
    }
}


// ===================================================== adaptive tree, up and down
constexpr int AMAXL = 40;     // deepest level (keys of 40 bits)
constexpr int AW = 4;         // warps per block of the per-cell kernels

struct AGeom {               // one sample's tree geometry
    double lo[3], ext[3];
    int axis[AMAXL + 1];          // axis halved to make level l (l >= 1)
    int nsplit[AMAXL + 1][3];     // splits of each axis in the first l levels
    double w[AMAXL + 1][3];       // cell widths of level l
    double w2[AMAXL + 1];         // squared diagonal, (w0^2 + w1^2) + w2^2
    double rad[AMAXL + 1];        // half diagonal, 0.5 sqrt(w2)
    double sh[AMAXL + 1][PMAX + 1];  // (w_l / 2)^t / t! along the axis split at level l
    double s;                     // split while a cell holds more than s
};

// Shift tables of the one-axis translations: for coefficient column c
// (multi-index n = c + 1) and axis s, the columns of n - t e_s (M2M, t = 0 ..
// n_s, the zero multi-index left out) and of n + t e_s (L2L, t = 0 .. p - |n|),
// in order of t.
constexpr int KPMAX = ((nterms(PMAX) - 1 + 7) / 8) * 8;
struct ShiftTab {
    uint8_t m2m_n[3][KPMAX], l2l_n[3][KPMAX];
    uint8_t m2m_c[3][KPMAX][PMAX + 1], l2l_c[3][KPMAX][PMAX + 1];
};

// Completion of the harmonic reduction: for full column c the reduced
// column (or -1), n_z, and for n_z >= 2 the full columns of n - 2e_z + 2e_x
// and n - 2e_z + 2e_y (V_n = -V of those two).
struct HarmTab {
    int8_t red[KPMAX];
    uint8_t nz[KPMAX], s1[KPMAX], s2[KPMAX];
};

// M2M (Eq. momentshift) into the internal cell c by one warp: the children
// sit at -/+ half their width along the axis split at their level; ws: the
// warp's scratch
template <typename real> struct AM2MWarp {
    real fs[2][PMAX + 1];  // shift factors (-/+ w/2)^t / t! of the two children
    real qs[2][KPMAX];     // the children's moments
};

template <typename real>
__device__ __forceinline__ void am2m_cell(int p, int KP, int c, const int *smp, const int *lev,
                                          const int *ch, const AGeom *geo, const ShiftTab *tb,
                                          real *Q, AM2MWarp<real> &ws)
{
    const int lane = threadIdx.x & 31;
    const int b0 = ch[2 * c], b1 = ch[2 * c + 1];
    if (b0 < 0 && b1 < 0) return;  // a leaf: P2M wrote its moments
    for (int col = lane; col < KP; col += 32) {
        ws.qs[0][col] = b0 >= 0 ? Q[(long long)b0 * KP + col] : (real)0;
        ws.qs[1][col] = b1 >= 0 ? Q[(long long)b1 * KP + col] : (real)0;
    }
    const AGeom &g = geo[smp[c]];
    const int l = lev[c], sx = g.axis[l + 1];
    if (lane < 2) {
        const real hw = (real)(0.5 * g.w[l + 1][sx]);
        const real cs = lane ? hw : -hw;
        real f = (real)1;
        ws.fs[lane][0] = f;
        for (int t = 1; t <= p; ++t) {
            f = f * cs / (real)t;
            ws.fs[lane][t] = f;
        }
    }
    __syncwarp();
    for (int col = lane; col < KP; col += 32) {
        real acc = (real)0;
        const int n = tb->m2m_n[sx][col];
        const uint8_t *cl = tb->m2m_c[sx][col];
        for (int b = 0; b < 2; ++b) {
            if ((b ? b1 : b0) < 0) continue;
            for (int t = 0; t < n; ++t) acc += ws.fs[b][t] * ws.qs[b][cl[t]];
        }
        Q[(long long)c * KP + col] = acc;
    }
}


// L2L (Eq. taylorshift, FP64) into cell c by one warp: V = the cell's own
// M2L sum + the parent's V shifted to the cell.  RED: the M2L sum is the
// reduced accumulator (rows of KRP), completed to all columns first.  ws: the
// warp's scratch
struct AL2LWarp {
    double fs[PMAX + 1];  // shift factors of the cell's offset from its parent
    double vp[KPMAX];     // the parent's V
    double vm[KPMAX];     // the cell's completed M2L sum (RED)
};

template <typename acc_t, bool RED>
__device__ __forceinline__ void al2l_cell(int p, int KP, int KRP, int c, const int *smp,
                                          const int *lev, const int *par, const int4 *ic,
                                          const AGeom *geo, const ShiftTab *tb, const HarmTab *ht,
                                          const acc_t *VF, double *V, AL2LWarp &ws)
{
    const int lane = threadIdx.x & 31;
    const int pr = par[c];
    const int K = nterms(p) - 1;
    const long long row = (long long)c * KP;
    if (RED) {
        for (int col = lane; col < K; col += 32) {
            const int r = ht->red[col];
            ws.vm[col] = r >= 0 ? (double)VF[(long long)c * KRP + r] : 0.0;
        }
        __syncwarp();
        for (int z = 2; z <= p; ++z) {
            for (int col = lane; col < K; col += 32)
                if (ht->nz[col] == z) ws.vm[col] = -ws.vm[ht->s1[col]] - ws.vm[ht->s2[col]];
            __syncwarp();
        }
    }
    auto m2l = [&](int col) -> double { return RED ? ws.vm[col] : (double)VF[row + col]; };
    if (pr < 0) {
        for (int col = lane; col < KP; col += 32) V[row + col] = col < K ? m2l(col) : 0.0;
        return;
    }
    const AGeom &g = geo[smp[c]];
    const int l = lev[c], sx = g.axis[l];
    if (lane <= p) {
        const double f = g.sh[l][lane];
        ws.fs[lane] = (ic[c].w || !(lane & 1)) ? f : -f;
    }
    for (int col = lane; col < KP; col += 32) ws.vp[col] = V[(long long)pr * KP + col];
    __syncwarp();
    for (int col = lane; col < KP; col += 32) {
        if (col >= K) {
            V[row + col] = 0.0;
            continue;
        }
        const int n = tb->l2l_n[sx][col];
        const uint8_t *cl = tb->l2l_c[sx][col];
        double acc = 0.0;
        for (int t = 0; t < n; ++t) acc += ws.fs[t] * ws.vp[cl[t]];
        V[row + col] = m2l(col) + acc;
    }
}


// field of sorted dipole i back to input order in FP64
template <typename real>
__device__ __forceinline__ void aunperm_one(long long i, const int *perm,
                                            const typename vec4<real>::t *H, double *Hd)
{
    const long long o = perm[i];
    const typename vec4<real>::t h = H[i];
    Hd[3 * o] = (double)h.x;
    Hd[3 * o + 1] = (double)h.y;
    Hd[3 * o + 2] = (double)h.z;
}

// E = -1/2 sum m.H of sample s by a block of NT threads in a fixed order;
// red: NT doubles of shared scratch
template <int NT>
__device__ __forceinline__ void aenergy_sample(int s, const long long *off, const double *mom,
                                               const double *Hd, double *E, double *red)
{
    double e = 0.0;
    for (long long i = off[s] + threadIdx.x; i < off[s + 1]; i += NT)
        e += mom[3 * i] * Hd[3 * i] + mom[3 * i + 1] * Hd[3 * i + 1] + mom[3 * i + 2] * Hd[3 * i + 2];
    red[threadIdx.x] = e;
    __syncthreads();
    for (int o = NT / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) E[s] = -0.5 * red[0];
}

// ============================================================ ensemble rotation
// Moment i of the ensemble turned about a random axis by a random angle:
// Philox4x64-10 (Salmon, Moraes, Dror, Shaw, SC 2011) with key (seed, step)
// and counter (i, 0, 0, 0); u_j = (x_j >> 11) 2^-53; axis z = 1 - 2 u0,
// phi = 2 pi u1; angle = max_angle u2; Rodrigues' formula, FP64.
__device__ __forceinline__ void philox4x64(unsigned long long c[4], unsigned long long k0,
                                           unsigned long long k1)
{
    const unsigned long long M0 = 0xD2E7470EE14C6C93ull, M1 = 0xCA5A826395121157ull;
    const unsigned long long W0 = 0x9E3779B97F4A7C15ull, W1 = 0xBB67AE8584CAA73Bull;
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        unsigned long long hi0 = __umul64hi(M0, c[0]), lo0 = M0 * c[0];
        unsigned long long hi1 = __umul64hi(M1, c[2]), lo1 = M1 * c[2];
        unsigned long long n0 = hi1 ^ c[1] ^ k0, n2 = hi0 ^ c[3] ^ k1;
        c[0] = n0;
        c[1] = lo1;
        c[2] = n2;
        c[3] = lo0;
        k0 += W0;
        k1 += W1;
    }
}

__device__ __forceinline__ void rotate_one(double *mom, long long i, const RotateParams *prm)
{
    const double two53 = 1.0 / 9007199254740992.0;
    unsigned long long x[4] = {(unsigned long long)i, 0ull, 0ull, 0ull};
    philox4x64(x, prm->seed, prm->step);
    double u0 = (double)(x[0] >> 11) * two53, u1 = (double)(x[1] >> 11) * two53;
    double u2 = (double)(x[2] >> 11) * two53;
    // phi = 2 pi u1 by sincospi(2 u1) (no argument reduction by pi), the
    // angle's sine and cosine from one sincos
    double z = 1.0 - 2.0 * u0, s = sqrt(1.0 - z * z), sp, cp;
    sincospi(2.0 * u1, &sp, &cp);
    double k[3] = {s * cp, s * sp, z};
    double a = prm->max_angle * u2, ca, sa;
    sincos(a, &sa, &ca);
    double m[3] = {mom[3 * i], mom[3 * i + 1], mom[3 * i + 2]};
    double kxm[3] = {k[1] * m[2] - k[2] * m[1], k[2] * m[0] - k[0] * m[2], k[0] * m[1] - k[1] * m[0]};
    double km = k[0] * m[0] + k[1] * m[1] + k[2] * m[2];
#pragma unroll
    for (int d = 0; d < 3; ++d) mom[3 * i + d] = m[d] * ca + kxm[d] * sa + k[d] * km * (1.0 - ca);
}

// moment of sorted dipole s (input index perm[s]) into the staged operands
template <typename real>
__device__ __forceinline__ void permute_one(long long s, const double *mom, const int *perm,
                                            typename vec4<real>::t *A,
                                            typename vec2<real>::t *B)
{
    const long long i = perm[s];
    A[s].w = (real)mom[3 * i];
    typename vec2<real>::t bv;
    bv.x = (real)mom[3 * i + 1];
    bv.y = (real)mom[3 * i + 2];
    B[s] = bv;
}

}  // namespace ccfmm
