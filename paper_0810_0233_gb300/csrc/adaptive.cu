// adaptive.cu -- the adaptive-depth tree (a project addition: the paper's
// tree is complete, every leaf at one depth, Sec. II).  The tree keeps the
// complete tree's box, split sequence and point membership, but a cell
// splits only while it holds more than s dipoles, and empty children are not
// created.  Two cells of different levels are near when (r_A + r_B) / d >
// theta (r = half the cell diagonal, d = distance of the centres); for equal
// levels this is the paper's 2r/d > alpha.  The lists are createPartners
// (Appendix) extended to unequal levels: a child takes as near candidates the
// children of every internal cell of its parent's near set and that set's
// leaves as they are; far candidates become Partners (M2L sources), near
// ones stay candidates; at a leaf, near leaves become nearPartners and a
// near internal cell is refined against the leaf (its far descendants become
// Partners, its near leaves nearPartners).
//
// Any number of independent samples form one forest: the build and every
// evaluation kernel work on global cell and dipole numbers, so each stage of
// an ensemble step is one launch (per level for M2M and L2L).
//
// Build (sizes known on the host after a few synchronisations):
//   1. per-sample box and split sequence; a 40-level key per dipole, whose
//      level-l prefix is the dipole's level-l cell (the complete tree's
//      membership rule applied at every level); sort by (sample, key);
//   2. cells: sorted dipole i starts the cells of the levels below its common
//      prefix with dipole i-1; those that exist (parent holds > s dipoles)
//      form a chain numbered by a scan, which numbers the cells in preorder,
//      the oracle's creation order;
//   3. lists level by level, one warp per cell (count, scan, fill);
//   4. far pairs sorted by (sample, separation): one D row per distinct
//      separation, and M2L work items: runs of up to 512 pairs of one row
//      (rows of at most 16 pairs go to a one-warp kernel).
// Evaluation: moments into sorted order, P2M (leaves), M2M (per level, up),
// M2L (items, atomics into an accumulator), L2L (per level, down; V = own
// M2L + parent's shifted V), near + smooth field (leaves), unpermute and the
// per-sample energies; captured once into a CUDA graph.
#include "../../include/ccfmm.h"
#include "ccfmm_dev.cuh"
#include "stages.cuh"

#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <string>
#include <vector>

namespace ccfmm {

constexpr int ASTACK = 96;    // depth-first stack of the leaf refinement

// ------------------------------------------------------------------ keys
// Box and split sequence of each sample (one block per sample): the given
// box, or the bounding box widened by 2^-20 of its largest extent; at each
// level the currently widest axis is halved, ties x < y < z.
__global__ void __launch_bounds__(256) k_ageom(const double *pos, const long long *off,
                                               const double *ubox, const double *sarr,
                                               double s_default, AGeom *geo, int *flags)
{
    __shared__ double red[6][8];
    const int smp = blockIdx.x;
    const long long n0 = off[smp], n1 = off[smp + 1];
    double mn[3] = {INFINITY, INFINITY, INFINITY}, mx[3] = {-INFINITY, -INFINITY, -INFINITY};
    if (!ubox)
        for (long long i = n0 + threadIdx.x; i < n1; i += blockDim.x)
            for (int a = 0; a < 3; ++a) {
                const double v = pos[3 * i + a];
                mn[a] = fmin(mn[a], v);
                mx[a] = fmax(mx[a], v);
            }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int a = 0; a < 3; ++a)
        for (int o = 16; o > 0; o >>= 1) {
            mn[a] = fmin(mn[a], __shfl_xor_sync(0xffffffffu, mn[a], o));
            mx[a] = fmax(mx[a], __shfl_xor_sync(0xffffffffu, mx[a], o));
        }
    if (lane == 0)
        for (int a = 0; a < 3; ++a) {
            red[a][warp] = mn[a];
            red[3 + a][warp] = mx[a];
        }
    __syncthreads();
    if (threadIdx.x != 0) return;
    AGeom g;
    if (ubox) {
        for (int a = 0; a < 3; ++a) {
            g.lo[a] = ubox[a];
            g.ext[a] = ubox[3 + a] - ubox[a];
        }
    } else {
        double blo[3], bhi[3];
        for (int a = 0; a < 3; ++a) {
            blo[a] = red[a][0];
            bhi[a] = red[3 + a][0];
            for (int w = 1; w < (int)(blockDim.x >> 5); ++w) {
                blo[a] = fmin(blo[a], red[a][w]);
                bhi[a] = fmax(bhi[a], red[3 + a][w]);
            }
        }
        double m = 0.0;
        for (int a = 0; a < 3; ++a)
            if (bhi[a] - blo[a] > m) m = bhi[a] - blo[a];
        if (m == 0.0) m = 1.0;
        const double pad = ldexp(m, -20);
        for (int a = 0; a < 3; ++a) {
            const double l0 = blo[a] - pad, h0 = bhi[a] + pad;
            g.lo[a] = l0;
            g.ext[a] = h0 - l0;
        }
    }
    for (int a = 0; a < 3; ++a) {
        g.nsplit[0][a] = 0;
        g.w[0][a] = g.ext[a];
        if (!(g.ext[a] > 0.0) || !isfinite(g.ext[a])) atomicOr(flags, FLAG_NONFINITE);
    }
    g.axis[0] = -1;
    for (int l = 1; l <= AMAXL; ++l) {
        double w[3];
        for (int b = 0; b < 3; ++b) w[b] = ldexp(g.ext[b], -g.nsplit[l - 1][b]);
        int a = 0;
        if (w[1] > w[a]) a = 1;
        if (w[2] > w[a]) a = 2;
        g.axis[l] = a;
        for (int b = 0; b < 3; ++b) g.nsplit[l][b] = g.nsplit[l - 1][b];
        g.nsplit[l][a] += 1;
        for (int b = 0; b < 3; ++b) g.w[l][b] = ldexp(g.ext[b], -g.nsplit[l][b]);
    }
    // integer cell coordinates stay below 2^30
    for (int a = 0; a < 3; ++a)
        if (g.nsplit[AMAXL][a] > 30) atomicOr(flags, FLAG_OFFSET_RANGE);
    for (int l = 0; l <= AMAXL; ++l) {
        g.w2[l] = __dadd_rn(__dadd_rn(__dmul_rn(g.w[l][0], g.w[l][0]), __dmul_rn(g.w[l][1], g.w[l][1])),
                            __dmul_rn(g.w[l][2], g.w[l][2]));
        g.rad[l] = 0.5 * sqrt(g.w2[l]);
        // shift factors of the one-axis translations between level l - 1
        // and level l (the child centre is at +/- w_l / 2 along axis[l])
        const double hw = l ? 0.5 * g.w[l][g.axis[l]] : 0.0;
        double f = 1.0;
        g.sh[l][0] = 1.0;
        for (int t = 1; t <= PMAX; ++t) {
            f = f * hw / (double)t;
            g.sh[l][t] = f;
        }
    }
    g.s = sarr ? sarr[smp] : s_default;
    geo[smp] = g;
}

__device__ __forceinline__ int sample_of(const long long *off, int ns, long long i)
{
    int lo = 0, hi = ns;  // off[lo] <= i < off[hi]
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (off[mid] <= i) lo = mid; else hi = mid;
    }
    return lo;
}

// 40-level key of every dipole (input order): the level-40 integer
// coordinates by the complete tree's rule (floor((x - lo) 2^n / ext), clamped
// to the box), whose bits interleaved in split order give every level's cell
__global__ void k_akeys(const double *pos, long long n, const long long *off, int ns,
                        const AGeom *geo, uint32_t *klo, uint32_t *khi, int *idx, int *flags)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int smp = sample_of(off, ns, i);
    const AGeom &g = geo[smp];
    long long ca[3];
    for (int a = 0; a < 3; ++a) {
        double x = pos[3 * i + a];
        if (!isfinite(x)) {
            atomicOr(flags, FLAG_NONFINITE);
            x = g.lo[a];
        }
        const int nsa = g.nsplit[AMAXL][a];
        const double na = ldexp(1.0, nsa);
        double t = __ddiv_rn(__dmul_rn(__dsub_rn(x, g.lo[a]), na), g.ext[a]);
        t = fmin(fmax(t, -1.0), na);
        long long c = (long long)floor(t);
        if (c > (1ll << nsa) - 1) c = (1ll << nsa) - 1;
        if (c < 0) c = 0;
        ca[a] = c;
    }
    unsigned long long key = 0;
    for (int l = 1; l <= AMAXL; ++l) {
        const int a = g.axis[l];
        const int sh = g.nsplit[AMAXL][a] - g.nsplit[l][a];
        key |= (unsigned long long)((ca[a] >> sh) & 1) << (AMAXL - l);
    }
    klo[i] = (uint32_t)key;
    khi[i] = ((uint32_t)smp << 8) | (uint32_t)(key >> 32);
    idx[i] = (int)i;
}

__global__ void k_gather_u32(const uint32_t *src, const int *idx, long long n, uint32_t *dst)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) dst[i] = src[idx[i]];
}

// ------------------------------------------------------------------ cells
__device__ __forceinline__ unsigned long long akey(const uint32_t *klo, const uint32_t *khi,
                                                   long long i)
{
    return ((unsigned long long)(khi[i] & 0xffu) << 32) | klo[i];
}
// levels shared by two keys (0 .. 40)
__device__ __forceinline__ int cpl(unsigned long long a, unsigned long long b)
{
    const unsigned long long x = a ^ b;
    return x ? __clzll((long long)x) - (64 - AMAXL) : AMAXL;
}
// first j in (i, hi) whose level-l cell differs from that of key ki
__device__ __forceinline__ long long cell_end(const uint32_t *klo, const uint32_t *khi, long long i,
                                              long long hi, unsigned long long ki, int l)
{
    const int sh = AMAXL - l;
    const unsigned long long lim = ((ki >> sh) + 1) << sh;
    long long a = i + 1, b = hi;
    while (a < b) {
        const long long m = (a + b) >> 1;
        if (akey(klo, khi, m) >= lim) b = m; else a = m + 1;
    }
    return a;
}
// first j in [lo, i] in the level-l cell of key ki
__device__ __forceinline__ long long cell_start(const uint32_t *klo, const uint32_t *khi,
                                                long long lo, long long i, unsigned long long ki,
                                                int l)
{
    const int sh = AMAXL - l;
    const unsigned long long base = (ki >> sh) << sh;
    long long a = lo, b = i;
    while (a < b) {
        const long long m = (a + b) >> 1;
        if (akey(klo, khi, m) >= base) b = m; else a = m + 1;
    }
    return a;
}

struct CellOut {
    int *lev, *smp, *p0, *np, *par, *ch;
    int4 *ic;       // integer coordinates at the cell's level, .w = side (child bit)
    double4 *cen;   // centre, .w = half diagonal
};

// The chain of cells that start at sorted dipole i.  Count pass: its length;
// emit pass: the cells, numbered from first[i].
template <bool EMIT>
__global__ void k_chain(long long n, const long long *off, const AGeom *geo, const uint32_t *klo,
                        const uint32_t *khi, int *len, const int *first, CellOut o)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int s = (int)(khi[i] >> 8);
    const long long n0 = off[s], n1 = off[s + 1];
    const AGeom &g = geo[s];
    const double thr = g.s;
    const unsigned long long ki = akey(klo, khi, i);
    int l1 = 0;
    int parent = -1;
    if (i > n0) {
        const int c = cpl(ki, akey(klo, khi, i - 1));
        bool none = c >= AMAXL;
        long long st = 0;
        if (!none) {
            // the level-c cell holding i - 1 and i splits iff it holds > s
            st = cell_start(klo, khi, n0, i, ki, c);
            const long long en = cell_end(klo, khi, i, n1, ki, c);
            none = (double)(en - st) <= thr;
        }
        if (none) {
            if (!EMIT) len[i] = 0;
            return;
        }
        l1 = c + 1;
        if (EMIT) {
            const int cs = (st == n0) ? -1 : cpl(akey(klo, khi, st), akey(klo, khi, st - 1));
            parent = first[st] + (c - (cs + 1));
        }
    }
    int id = EMIT ? first[i] : 0;
    int cnt = 0;
    for (int l = l1;; ++l) {
        const long long cl = cell_end(klo, khi, i, n1, ki, l) - i;
        if (EMIT) {
            const int pr = (l == l1) ? parent : id - 1;
            o.lev[id] = l;
            o.smp[id] = s;
            o.p0[id] = (int)i;
            o.np[id] = (int)cl;
            o.par[id] = pr;
            long long ic[3] = {0, 0, 0};
            int bit = 0;
            for (int lv = 1; lv <= l; ++lv) {
                const int a = g.axis[lv];
                bit = (int)((ki >> (AMAXL - lv)) & 1);
                ic[a] = 2 * ic[a] + bit;
            }
            o.ic[id] = make_int4((int)ic[0], (int)ic[1], (int)ic[2], bit);
            double4 cc;
            cc.x = __dadd_rn(g.lo[0], __dmul_rn((double)ic[0] + 0.5, g.w[l][0]));
            cc.y = __dadd_rn(g.lo[1], __dmul_rn((double)ic[1] + 0.5, g.w[l][1]));
            cc.z = __dadd_rn(g.lo[2], __dmul_rn((double)ic[2] + 0.5, g.w[l][2]));
            cc.w = g.rad[l];
            o.cen[id] = cc;
            if (pr >= 0) o.ch[2 * pr + bit] = id;
        }
        ++cnt;
        ++id;
        if ((double)cl <= thr || l >= AMAXL) break;
    }
    if (!EMIT) len[i] = cnt;
}

__global__ void k_leaf_flag(int nc, const int *ch, int *flag)
{
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c < nc) flag[c] = (ch[2 * c] < 0 && ch[2 * c + 1] < 0) ? 1 : 0;
}

__global__ void k_leaf_list(int nc, const int *flag, const int *rank, int *leaves)
{
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c < nc && flag[c]) leaves[rank[c]] = c;
}

__global__ void k_level_hist(int nc, const int *lev, int *hist)
{
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c < nc) atomicAdd(&hist[lev[c]], 1);
}

__global__ void k_iota(int n, int *v)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) v[i] = i;
}

// dipole coordinates relative to their leaf's centre (one warp per leaf)
template <typename real>
__global__ void __launch_bounds__(32 * AW) k_apoints(int nleaf, const int *leaves, const int *p0,
                                                     const int *np, const double4 *cen,
                                                     const int *perm, const double *pos,
                                                     typename vec4<real>::t *A)
{
    const int li = blockIdx.x * AW + (threadIdx.x >> 5), lane = threadIdx.x & 31;
    if (li >= nleaf) return;
    const int c = leaves[li];
    const double4 cc = cen[c];
    for (int j = p0[c] + lane; j < p0[c] + np[c]; j += 32) {
        const long long o = perm[j];
        typename vec4<real>::t a;
        a.x = (real)(pos[3 * o] - cc.x);
        a.y = (real)(pos[3 * o + 1] - cc.y);
        a.z = (real)(pos[3 * o + 2] - cc.z);
        a.w = (real)0;
        A[j] = a;
    }
}

// ------------------------------------------------------------------ lists
struct ListArgs {
    int nl;
    const int *cells;               // this level's cells
    const AGeom *geo;
    double thth;                    // theta^2
    const int *lev, *smp, *ch;
    const double4 *cen;
    const int *cand, *cand_first, *cand_num;  // near candidates of this level
    int *cnt;                       // count pass: [3][nl] candidates, far, near
    const int *off;                 // fill pass: [3][nl] exclusive offsets
    long long far_base, near_base;
    int *cand_next, *cand_first_w, *cand_num_w;
    int *far_t, *far_s;
    int *near_src, *near_first, *near_num;
    int *flags;
};

// near test of the oracle, in the same operations and order
__device__ __forceinline__ bool anear(double thth, const AGeom *g, int lx, double4 cx, int ly,
                                      double4 cy)
{
    const double dx = __dsub_rn(cx.x, cy.x), dy = __dsub_rn(cx.y, cy.y),
                 dz = __dsub_rn(cx.z, cy.z);
    const double d2 = __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
    const double rhs = __dmul_rn(__dmul_rn(thth, d2), 1.0 + 1e-12);
    if (lx == ly) return g->w2[lx] > rhs;
    const double r = __dadd_rn(cx.w, cy.w);
    return __dmul_rn(r, r) > rhs;
}

__device__ __forceinline__ int warp_excl(int v, int &tot)
{
    const int lane = threadIdx.x & 31;
    int x = v;
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    tot = __shfl_sync(0xffffffffu, x, 31);
    return x - v;
}

// leaf c against the subtree of its near internal candidate x, depth first
// with the lower child first: far cells -> Partners of c, near leaves ->
// nearPartners, near internal cells refined further
template <bool FILL>
__device__ void aresolve(const ListArgs &a, const AGeom *g, int c, int x, int &kn, int &kf,
                         long long pn, long long pf)
{
    const double4 cc = a.cen[c];
    const int lc = a.lev[c];
    int stk[ASTACK];
    int sp = 0;
    const int x0 = a.ch[2 * x], x1 = a.ch[2 * x + 1];
    if (x1 >= 0) stk[sp++] = x1;
    if (x0 >= 0) stk[sp++] = x0;
    while (sp > 0) {
        const int b = stk[--sp];
        if (!anear(a.thth, g, lc, cc, a.lev[b], a.cen[b])) {
            if (FILL) {
                a.far_t[pf] = c;
                a.far_s[pf] = b;
                ++pf;
            }
            ++kf;
            continue;
        }
        const int b0 = a.ch[2 * b], b1 = a.ch[2 * b + 1];
        if (b0 < 0 && b1 < 0) {
            if (FILL) a.near_src[pn++] = b;
            ++kn;
        } else {
            if (sp + 2 > ASTACK) {
                atomicOr(a.flags, FLAG_LIST_OVERFLOW);
                break;
            }
            if (b1 >= 0) stk[sp++] = b1;
            if (b0 >= 0) stk[sp++] = b0;
        }
    }
}

// one level of the lists, one warp per cell of the level: an internal cell
// classifies its children's candidates; a leaf forms its near list and
// refines its near internal candidates.  Outputs in the oracle's order.
template <bool FILL>
__global__ void __launch_bounds__(32 * AW) k_alist(ListArgs a)
{
    const int w = blockIdx.x * AW + (threadIdx.x >> 5), lane = threadIdx.x & 31;
    if (w >= a.nl) return;
    const int c = a.cells[w];
    const AGeom *g = a.geo + a.smp[c];
    const int cf = a.cand_first[c], cn = a.cand_num[c];
    const int c0 = a.ch[2 * c], c1 = a.ch[2 * c + 1];
    int ncand = 0, nfar = 0, nnear = 0;
    long long ob_c = 0, ob_f = 0, ob_n = 0;
    if (FILL) {
        ob_c = a.off[w];
        ob_f = a.far_base + a.off[a.nl + w];
        ob_n = a.near_base + a.off[2 * a.nl + w];
    }
    if (c0 >= 0 || c1 >= 0) {
        for (int t = 0; t < 2; ++t) {
            const int ci = t ? c1 : c0;
            if (ci < 0) continue;
            const double4 cc = a.cen[ci];
            const int lc = a.lev[ci];
            const int cstart = ncand;
            for (int j0 = 0; j0 < cn; j0 += 32) {
                const int j = j0 + lane;
                int b0 = -1, b1 = -1;
                if (j < cn) {
                    const int x = a.cand[cf + j];
                    if (x == c) {
                        b0 = c0;
                        b1 = c1;
                    } else {
                        const int x0 = a.ch[2 * x], x1 = a.ch[2 * x + 1];
                        if (x0 < 0 && x1 < 0) {
                            b0 = x;
                        } else {
                            b0 = x0;
                            b1 = x1;
                        }
                    }
                }
                const bool v0 = b0 >= 0, v1 = b1 >= 0;
                const bool n0 = v0 && (b0 == ci || anear(a.thth, g, lc, cc, a.lev[b0], a.cen[b0]));
                const bool n1 = v1 && (b1 == ci || anear(a.thth, g, lc, cc, a.lev[b1], a.cen[b1]));
                const int kn = (int)n0 + (int)n1, kf = (int)(v0 && !n0) + (int)(v1 && !n1);
                int totn, totf;
                const int en = warp_excl(kn, totn), ef = warp_excl(kf, totf);
                if (FILL) {
                    long long pc = ob_c + ncand + en, pf = ob_f + nfar + ef;
                    if (v0) {
                        if (n0) {
                            a.cand_next[pc++] = b0;
                        } else {
                            a.far_t[pf] = ci;
                            a.far_s[pf] = b0;
                            ++pf;
                        }
                    }
                    if (v1) {
                        if (n1) {
                            a.cand_next[pc++] = b1;
                        } else {
                            a.far_t[pf] = ci;
                            a.far_s[pf] = b1;
                            ++pf;
                        }
                    }
                }
                ncand += totn;
                nfar += totf;
            }
            if (FILL && lane == 0) {
                a.cand_first_w[ci] = (int)(ob_c + cstart);
                a.cand_num_w[ci] = ncand - cstart;
            }
        }
    } else {
        for (int j0 = 0; j0 < cn; j0 += 32) {
            const int j = j0 + lane;
            int kn = 0, kf = 0, x = -1;
            bool direct = false;
            if (j < cn) {
                x = a.cand[cf + j];
                direct = x == c || (a.ch[2 * x] < 0 && a.ch[2 * x + 1] < 0);
                if (direct)
                    kn = 1;
                else
                    aresolve<false>(a, g, c, x, kn, kf, 0, 0);
            }
            int totn, totf;
            const int en = warp_excl(kn, totn), ef = warp_excl(kf, totf);
            if (FILL && j < cn) {
                const long long pn = ob_n + nnear + en, pf = ob_f + nfar + ef;
                if (direct) {
                    a.near_src[pn] = x;
                } else {
                    int dn = 0, df = 0;
                    aresolve<true>(a, g, c, x, dn, df, pn, pf);
                }
            }
            nnear += totn;
            nfar += totf;
        }
        if (FILL && lane == 0) {
            a.near_first[c] = (int)ob_n;
            a.near_num[c] = nnear;
        }
    }
    if (!FILL && lane == 0) {
        a.cnt[w] = ncand;
        a.cnt[a.nl + w] = nfar;
        a.cnt[2 * a.nl + w] = nnear;
    }
}

// each sample's root is its own near candidate
__global__ void k_root_cand(int ns, const int *roots, int *cand, int *cand_first, int *cand_num)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= ns) return;
    const int r = roots[k];
    cand[k] = r;
    cand_first[r] = k;
    cand_num[r] = 1;
}

// dipole pairs of the near field: sum over leaves of n_leaf x n_partner
// (the leaf itself included, as the oracle's nearPartners do)
__global__ void k_near_pairs(int nleaf, const int *leaves, const int *np, const int *near_first,
                             const int *near_num, const int *near_src, unsigned long long *total)
{
    const int li = blockIdx.x * blockDim.x + threadIdx.x;
    unsigned long long s = 0;
    if (li < nleaf) {
        const int c = leaves[li];
        for (int e = near_first[c]; e < near_first[c] + near_num[c]; ++e)
            s += (unsigned long long)np[c] * (unsigned long long)np[near_src[e]];
    }
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0 && s) atomicAdd(total, s);
}

// ----------------------------------------------------- M2L groups and items
constexpr long long AR_BIAS = 1ll << 18;  // separations |R_a| < 2^18 finest units

// key of a far pair's separation: the finer of the two levels L and, per
// axis, (target centre - source centre) in units of half a level-L width
__global__ void k_dkey(long long nf, const int *ft, const int *fs, const int *lev, const int *smp,
                       const int4 *ic, const AGeom *geo, uint32_t *klo, uint32_t *khi,
                       uint32_t *ksm, int *idx, int *flags)
{
    const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nf) return;
    const int t = ft[k], s = fs[k];
    const int lt = lev[t], ls = lev[s], L = max(lt, ls);
    const AGeom &g = geo[smp[t]];
    const int4 it = ic[t], is = ic[s];
    const long long ct[3] = {it.x, it.y, it.z}, cs[3] = {is.x, is.y, is.z};
    unsigned long long key = (unsigned long long)L << 57;
    for (int a = 0; a < 3; ++a) {
        const int m = g.nsplit[L][a];
        long long R = ((2 * ct[a] + 1) << (m - g.nsplit[lt][a])) - ((2 * cs[a] + 1) << (m - g.nsplit[ls][a]));
        if (R <= -AR_BIAS || R >= AR_BIAS) {
            atomicOr(flags, FLAG_OFFSET_RANGE);
            R = 0;
        }
        key |= (unsigned long long)(R + AR_BIAS) << (38 - 19 * a);
    }
    klo[k] = (uint32_t)key;
    khi[k] = (uint32_t)(key >> 32);
    ksm[k] = (uint32_t)smp[t];
    idx[k] = (int)k;
}

// sorted pair arrays, and the first pair of every distinct (sample, key)
__global__ void k_group_flags(long long nf, const int *perm, const uint32_t *klo,
                              const uint32_t *khi, const uint32_t *ksm_sorted, const int *ft,
                              const int *fs, int *pt, int *ps, int *gflag)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nf) return;
    const int k = perm[i];
    pt[i] = ft[k];
    ps[i] = fs[k];
    int f = 1;
    if (i > 0) {
        const int kp = perm[i - 1];
        f = (klo[k] != klo[kp] || khi[k] != khi[kp] || ksm_sorted[i] != ksm_sorted[i - 1]) ? 1 : 0;
    }
    gflag[i] = f;
}

// group starts, the D rows' separations (unit vector, length), and the
// number of 64- and 16-pair work items of each group
__global__ void k_group_sep(long long nf, int p, const int *gflag, const int *grank,
                            const int *pt, const int *ps, const double4 *cen, int *gstart,
                            double4 *sep, float *rpow)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nf || !gflag[i]) return;
    const int d = grank[i];
    gstart[d] = (int)i;
    const double4 a = cen[pt[i]], b = cen[ps[i]];
    const double x = a.x - b.x, y = a.y - b.y, z = a.z - b.z;
    const double r = sqrt(x * x + y * y + z * z);
    sep[d] = make_double4(x / r, y / r, z / r, r);
    const double ri = 1.0 / r;
    double v = 1.0;
    for (int k = 0; k < PMAX + 2; ++k) {
        rpow[(long long)d * (PMAX + 2) + k] = k <= p + 1 ? (float)v : 0.f;
        v *= ri;
    }
}

// work items of a group of n pairs: groups of more than 16 pairs go to the
// 64-pair kernel in items of up to AIT pairs (one M per item), the others
// to the 16-pair kernel as one item
constexpr int AIT = 512;
__device__ __forceinline__ void item_split(int n, int &n64, int &n16)
{
    if (n > 16) {
        n64 = (n + AIT - 1) / AIT;
        n16 = 0;
    } else {
        n64 = 0;
        n16 = 1;
    }
}

__global__ void k_item_count(int nd, const int *gstart, long long nf, int *c64, int *c16)
{
    const int d = blockIdx.x * blockDim.x + threadIdx.x;
    if (d >= nd) return;
    const int n = (int)((d + 1 < nd ? gstart[d + 1] : nf) - gstart[d]);
    int a, b;
    item_split(n, a, b);
    c64[d] = a;
    c16[d] = b;
}

__global__ void k_item_fill(int nd, const int *gstart, long long nf, const int *o64,
                            const int *o16, int4 *it64, int4 *it16)
{
    const int d = blockIdx.x * blockDim.x + threadIdx.x;
    if (d >= nd) return;
    const int g0 = gstart[d];
    const int n = (int)((d + 1 < nd ? gstart[d + 1] : nf) - g0);
    int a, b;
    item_split(n, a, b);
    // equal shares, so that no item is much longer than the others
    for (int j = 0; j < a; ++j) {
        const int lo = (int)((long long)n * j / a), hi = (int)((long long)n * (j + 1) / a);
        it64[o64[d] + j] = make_int4(g0 + lo, hi - lo, d, 0);
    }
    if (b) it16[o16[d]] = make_int4(g0, n, d, 0);
}

// ---------------------------------------------------------------- upward / downward
__global__ void k_shift_tab(int p, ShiftTab *tb)
{
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= KPMAX) return;
    const int K = nterms(p) - 1;
    for (int sx = 0; sx < 3; ++sx) {
        int nm = 0, nl = 0;
        if (c < K) {
            int nn[3];
            midx_inv(c + 1, nn[0], nn[1], nn[2]);
            const int kn = nn[0] + nn[1] + nn[2];
            for (int t = 0; t <= nn[sx]; ++t) {
                int m[3] = {nn[0], nn[1], nn[2]};
                m[sx] -= t;
                if (m[0] + m[1] + m[2] > 0) tb->m2m_c[sx][c][nm++] = (uint8_t)(midx(m[0], m[1], m[2]) - 1);
            }
            for (int t = 0; t <= p - kn; ++t) {
                int m[3] = {nn[0], nn[1], nn[2]};
                m[sx] += t;
                tb->l2l_c[sx][c][nl++] = (uint8_t)(midx(m[0], m[1], m[2]) - 1);
            }
        }
        tb->m2m_n[sx][c] = (uint8_t)nm;
        tb->l2l_n[sx][c] = (uint8_t)nl;
    }
}

// M2M (Eq. momentshift) into every internal cell of one level, one warp per
// cell (am2m_cell)
template <typename real>
__global__ void __launch_bounds__(32 * AW) k_am2m(int p, int KP, const int *cells, int ncl,
                                                  const int *smp, const int *lev, const int *ch,
                                                  const AGeom *geo, const ShiftTab *tb, real *Q)
{
    __shared__ AM2MWarp<real> ws[AW];
    const int w = threadIdx.x >> 5;
    const int idx = blockIdx.x * AW + w;
    if (idx >= ncl) return;
    am2m_cell<real>(p, KP, cells[idx], smp, lev, ch, geo, tb, Q, ws[w]);
}

__global__ void k_harm_tab(int p, HarmTab *ht)
{
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= KPMAX) return;
    const int K = nterms(p) - 1;
    int r = -1, z = 0, a = 0, b = 0;
    if (c < K) {
        int nx, ny, nz;
        midx_inv(c + 1, nx, ny, nz);
        const int k = nx + ny + nz;
        z = nz;
        if (nz <= 1) {
            r = k * k - 1 + nz * (2 * k + 3 - nz) / 2 + ny;
        } else {
            a = midx(nx + 2, ny, nz - 2) - 1;
            b = midx(nx, ny + 2, nz - 2) - 1;
        }
    }
    ht->red[c] = (int8_t)r;
    ht->nz[c] = (uint8_t)z;
    ht->s1[c] = (uint8_t)a;
    ht->s2[c] = (uint8_t)b;
}

// L2L (Eq. taylorshift, FP64) into every cell of one level, one warp per
// cell (al2l_cell)
template <typename acc_t, bool RED>
__global__ void __launch_bounds__(32 * AW) k_al2l(int p, int KP, int KRP, const int *cells,
                                                  int ncl, const int *smp, const int *lev,
                                                  const int *par, const int4 *ic,
                                                  const AGeom *geo, const ShiftTab *tb,
                                                  const HarmTab *ht, const acc_t *VF, double *V)
{
    __shared__ AL2LWarp ws[AW];
    const int w = threadIdx.x >> 5;
    const int idx = blockIdx.x * AW + w;
    if (idx >= ncl) return;
    al2l_cell<acc_t, RED>(p, KP, KRP, cells[idx], smp, lev, par, ic, geo, tb, ht, VF, V, ws[w]);
}

// fields back to input order in FP64
template <typename real>
__global__ void k_aunperm(long long n, const int *perm, const typename vec4<real>::t *H,
                          double *Hd)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) aunperm_one<real>(i, perm, H, Hd);
}

// E = -1/2 sum m.H per sample, one block per sample, fixed order
__global__ void __launch_bounds__(256) k_aenergy(const long long *off, const double *mom,
                                                 const double *Hd, double *E)
{
    __shared__ double red[256];
    aenergy_sample<256>(blockIdx.x, off, mom, Hd, E, red);
}

// ------------------------------------------------------------ persistent step
// The whole evaluation of the forest (FP32 path, tensor-core M2L over the
// harmonic reduction) in one launch of persistent blocks of 128 threads that
// take tasks from one queue.  A task is a (stage, tile) of all samples at
// once: a chunk of dipoles for the rotation, the moment permutation and the
// unpermute, 16 leaves (a warp each, four at a time) for P2M and L2P, 16 cells
// of one level for M2M and L2L, 16 cells for the fold, one M2L item of more
// than 16 pairs or 16 of at most 16, one leaf for the near field, one sample
// for the energy.  The tasks of a stage form a phase; a task may wait for up
// to two phases to be complete (done[ph] == need[ph]), and every phase it
// waits for lies wholly before it in the queue.  Blocks take queue indices in
// order (one atomic counter; a block fetches its next index while its current
// task runs), so the earliest unfinished task never waits on a later one and
// the queue drains whatever number of blocks is resident.  A block remembers
// the phases it has found complete and polls only for new ones.
// Waits poll with a bound (poll_limit polls, nanosleep between them): a wait
// that runs out sets err and its block stops; every block stops once err is
// set, so the launch always ends.  The host zeroes head, err and done before
// each launch.
enum ATask : int {
    AT_ROT = 0,
    AT_PERM,
    AT_P2M,
    AT_M2M,
    AT_FOLD,
    AT_M2L_BIG,
    AT_M2L_SMALL,
    AT_L2L,
    AT_P2P,
    AT_L2P,
    AT_UNPERM,
    AT_ENERGY
};
constexpr int ACHUNK = 2048;  // dipoles per task of the elementwise stages
constexpr int ACELLS = 16;    // cells (leaves) per task of the warp-per-cell stages
constexpr int AGROUPS = 4;    // groups of four small M2L items per task
constexpr int ASEEN = 256;    // phases whose completion a block remembers
constexpr int ASTEP_T = 128;  // threads per block

struct AStepArgs {
    const int4 *tasks;  // x = type | phase << 8, y, z: task range, w = waits + 1 (16 bits each)
    int ntask;
    int *ctl;           // [0] head, [1] err, [2 ..] done per phase
    const int *need;    // tasks per phase
    long long poll_limit;
    int rotate;
    int p, KP, KRP, ldD, n16, nc;
    long long N;
    double *mom;
    const RotateParams *prm;
    const int *perm;
    float4 *A, *H;
    float2 *B;
    double *Hd, *E, *V;
    const long long *offd;
    const int *leaves, *p0, *np, *near_first, *near_num, *near_src;
    const double4 *cen;
    float *Q, *Qr, *VFr;
    const int *lvl_cells, *smp, *lev, *ch, *par;
    const int4 *ic;
    const AGeom *geo;
    const ShiftTab *shift;
    const HarmTab *harm;
    const int4 *it64, *it16;
    const int *pt, *ps;
    const float *rpow, *D;
    const uint16_t *itr;
};

__device__ __forceinline__ int ld_acquire(const int *p)
{
    int v;
    asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// thread 0: wait (bounded) until phase ph is complete; false when the wait
// ran out or another block has given up.  seen: the phases this block has
// already found complete (a phase stays complete for the rest of the launch);
// fresh = true when a phase was newly found complete.
__device__ __forceinline__ bool astep_wait(const AStepArgs &a, int ph, unsigned *seen,
                                           bool &fresh)
{
    if (ph < 0) return true;
    if (ph < ASEEN && ((seen[ph >> 5] >> (ph & 31)) & 1u)) return true;
    const int need = a.need[ph];
    const int *done = a.ctl + 2 + ph;
    for (long long it = 0;; ++it) {
        if (ld_acquire(done) >= need) {
            if (ph < ASEEN) seen[ph >> 5] |= 1u << (ph & 31);
            fresh = true;
            return true;
        }
        if (it >= a.poll_limit || ld_acquire(a.ctl + 1)) return false;
        __nanosleep(it < 32 ? 64 : 512);
    }
}

// thread 0: task nxt of the queue once its phases are complete, or x = -1
// (queue empty, or stop); nxt becomes the queue index of the block's next
// task, fetched while this one runs
__device__ __forceinline__ int4 astep_take(const AStepArgs &a, int &nxt, unsigned *seen)
{
    const int4 stop = make_int4(-1, 0, 0, 0);
    if (ld_acquire(a.ctl + 1)) return stop;
    const int t = nxt;
    if (t >= a.ntask) return stop;
    const int4 tk = a.tasks[t];
    nxt = atomicAdd(a.ctl, 1);
    bool fresh = false;
    if (!astep_wait(a, (tk.w & 0xffff) - 1, seen, fresh) ||
        !astep_wait(a, (tk.w >> 16) - 1, seen, fresh)) {
        atomicExch(a.ctl + 1, 1);
        return stop;
    }
    if (fresh) __threadfence();
    return tk;
}

template <int P>
__global__ void __launch_bounds__(ASTEP_T, CCFMM_P2P_MINB) k_astep(const AStepArgs a)
{
    constexpr int KRP = red_padded(P);
    extern __shared__ __align__(16) unsigned char smraw[];
    __shared__ int4 s_task;
    __shared__ unsigned s_seen[ASEEN / 32];
    const int tid = threadIdx.x, w = tid >> 5;
    int nxt = 0;
    if (tid < ASEEN / 32) s_seen[tid] = 0u;
    if (tid == 0) nxt = atomicAdd(a.ctl, 1);
    __syncthreads();
    for (;;) {
        if (tid == 0) s_task = astep_take(a, nxt, s_seen);
        __syncthreads();
        const int4 tk = s_task;
        if (tk.x < 0) break;
        const int type = tk.x & 255;
        switch (type) {
        case AT_ROT:
            if (a.rotate)
                for (long long i = (long long)tk.y * ACHUNK + tid;
                     i < min(a.N, (long long)(tk.y + 1) * ACHUNK); i += ASTEP_T)
                    rotate_one(a.mom, i, a.prm);
            break;
        case AT_PERM:
            for (long long i = (long long)tk.y * ACHUNK + tid;
                 i < min(a.N, (long long)(tk.y + 1) * ACHUNK); i += ASTEP_T)
                permute_one<float>(i, a.mom, a.perm, a.A, a.B);
            break;
        case AT_P2M:
            for (int r = 0; r < ACELLS; r += P2M_W) {
                const int li = tk.y + r + w;
                const bool live = li < tk.z;
                const int c = live ? a.leaves[li] : 0;
                const int s0 = live ? a.p0[c] : 0, s1 = live ? s0 + a.np[c] : 0;
                p2m_run<float>(P, a.KP, live, s0, s1, a.A, a.B, a.Q + (long long)c * a.KP,
                               *reinterpret_cast<P2MScratch<float> *>(smraw));
                __syncthreads();
            }
            break;
        case AT_M2M:
            for (int idx = tk.y + w; idx < min(tk.z, tk.y + ACELLS); idx += AW) {
                am2m_cell<float>(P, a.KP, a.lvl_cells[idx], a.smp, a.lev, a.ch, a.geo, a.shift,
                                 a.Q, reinterpret_cast<AM2MWarp<float> *>(smraw)[w]);
                __syncwarp();
            }
            break;
        case AT_FOLD:
            for (int c = tk.y + w; c < min(a.nc, tk.y + ACELLS); c += AW) {
                afold_cell(P, a.KP, KRP, c, a.Q, a.Qr, reinterpret_cast<float *>(smraw) + w * AF_ROW);
                __syncwarp();
            }
            break;
        case AT_M2L_BIG:
            am2l_big_item<KRP>(P, a.it64[tk.y], a.pt, a.ps, a.rpow, a.D, a.ldD, a.itr, a.Qr,
                               a.VFr, smraw);
            break;
        case AT_M2L_SMALL:
            for (int g = tk.y; g < min(tk.z, tk.y + AGROUPS); ++g) {
                am2l_small_items<KRP>(P, a.it16, a.n16, g, a.pt, a.ps, a.rpow, a.D, a.ldD, a.itr,
                                      a.Qr, a.VFr, smraw);
                __syncthreads();
            }
            break;
        case AT_L2L:
            for (int idx = tk.y + w; idx < min(tk.z, tk.y + ACELLS); idx += AW) {
                al2l_cell<float, true>(P, a.KP, KRP, a.lvl_cells[idx], a.smp, a.lev, a.par, a.ic,
                                       a.geo, a.shift, a.harm, a.VFr, a.V,
                                       reinterpret_cast<AL2LWarp *>(smraw)[w]);
                __syncwarp();
            }
            break;
        case AT_P2P: {
            const int c = a.leaves[tk.y];
            const double4 cc = a.cen[c];
            const AdaEnts ents{a.p0, a.np, a.near_src, a.cen, cc.x, cc.y, cc.z, c};
            const int e0 = a.near_first[c];
            p2p_leaf<float, AdaEnts, false, ASTEP_T, P2P_CH>(P, a.p0[c], a.np[c], e0,
                                                             e0 + a.near_num[c], ents, nullptr,
                                                             a.A, a.B, a.H);
            break;
        }
        case AT_L2P:
            for (int li = tk.y + w; li < min(tk.z, tk.y + ACELLS); li += L2P_W) {
                al2p_leaf<float, P>(a.KP, a.leaves[li], a.p0, a.np, a.A, a.V, a.H,
                                    reinterpret_cast<float *>(smraw) + w * nterms(PMAX));
                __syncwarp();
            }
            break;
        case AT_UNPERM:
            for (long long i = (long long)tk.y * ACHUNK + tid;
                 i < min(a.N, (long long)(tk.y + 1) * ACHUNK); i += ASTEP_T)
                aunperm_one<float>(i, a.perm, a.H, a.Hd);
            break;
        case AT_ENERGY:
            aenergy_sample<ASTEP_T>(tk.y, a.offd, a.mom, a.Hd, a.E,
                                    reinterpret_cast<double *>(smraw));
            break;
        default: break;
        }
        // every thread's writes reach the GPU scope before the phase counter
        __threadfence();
        __syncthreads();
        if (tid == 0) atomicAdd(a.ctl + 2 + (tk.x >> 8), 1);
    }
}

// dynamic shared memory of k_astep<P>: the largest stage scratch
template <int P> size_t astep_smem(int KP, int ldD)
{
    constexpr int KRP = red_padded(P);
    size_t m = (size_t)P2P_CH * (sizeof(float4) + sizeof(float2)) + (size_t)P2P_NE * sizeof(float4) +
               (2 * P2P_NE + 4) * sizeof(int) + (size_t)KP * sizeof(float) + 64;
    m = std::max(m, sizeof(P2MScratch<float>));
    m = std::max(m, AW * sizeof(AM2MWarp<float>));
    m = std::max(m, AW * sizeof(AL2LWarp));
    m = std::max(m, (size_t)AW * AF_ROW * sizeof(float));
    m = std::max(m, am2l_big_smem<KRP>(ldD));
    m = std::max(m, am2l_small_smem<KRP>(ldD));
    m = std::max(m, (size_t)L2P_W * nterms(PMAX) * sizeof(float));
    m = std::max(m, (size_t)ASTEP_T * sizeof(double));
    return (m + 15) & ~(size_t)15;
}

// launch with as many blocks as fit the SMs (no more than tasks)
template <int P> cudaError_t launch_astep_p(const AStepArgs &a, cudaStream_t s)
{
    const size_t smem = astep_smem<P>(a.KP, a.ldD);
    cudaError_t e = cudaFuncSetAttribute(k_astep<P>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    int per = 0, dev = 0, nsm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_astep<P>, ASTEP_T, smem);
    if (e != cudaSuccess) return e;
    const int grid = std::max(1, std::min(a.ntask, std::max(1, per) * nsm));
    note_launch();
    k_astep<P><<<grid, ASTEP_T, smem, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_astep(int p, const AStepArgs &a, cudaStream_t s)
{
    switch (p) {
    case 2: return launch_astep_p<2>(a, s);
    case 3: return launch_astep_p<3>(a, s);
    case 4: return launch_astep_p<4>(a, s);
    case 5: return launch_astep_p<5>(a, s);
    case 6: return launch_astep_p<6>(a, s);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace ccfmm

// =================================================================== host
using namespace ccfmm;

namespace {

std::string g_aerr;

ccfmm_status afail(ccfmm_status st, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    set_last_error(buf);
    return st;
}

#define ACK(call)                                                                                \
    do {                                                                                         \
        cudaError_t e_ = (call);                                                                 \
        if (e_ != cudaSuccess) {                                                                 \
            cudaGetLastError();                                                                  \
            return afail(CCFMM_ERR_CUDA, "%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_),  \
                         __FILE__, __LINE__);                                                    \
        }                                                                                        \
    } while (0)
#define ATRY(x)                                                                                  \
    do {                                                                                         \
        ccfmm_status s_ = (x);                                                                   \
        if (s_ != CCFMM_OK) return s_;                                                           \
    } while (0)

struct ABuf {
    void *p = nullptr;
    size_t bytes = 0;
};

ccfmm_status aalloc(ABuf &b, size_t bytes)
{
    if (bytes == 0) bytes = 16;
    if (b.p && b.bytes >= bytes) return CCFMM_OK;
    if (b.p) cudaFree(b.p);
    b.p = nullptr;
    b.bytes = 0;
    cudaError_t e = cudaMalloc(&b.p, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        b.p = nullptr;
        return afail(CCFMM_ERR_ALLOC, "device allocation of %zu bytes failed: %s", bytes,
                     cudaGetErrorString(e));
    }
    b.bytes = bytes;
    return CCFMM_OK;
}

// grow keeping the first `used` bytes
ccfmm_status agrow(ABuf &b, size_t used, size_t need, cudaStream_t s)
{
    if (b.p && b.bytes >= need) return CCFMM_OK;
    ABuf nb;
    ATRY(aalloc(nb, std::max(need, 2 * b.bytes)));
    if (used) ACK(cudaMemcpyAsync(nb.p, b.p, used, cudaMemcpyDeviceToDevice, s));
    if (b.p) {
        ACK(cudaStreamSynchronize(s));
        cudaFree(b.p);
    }
    b = nb;
    return CCFMM_OK;
}

void afree(ABuf &b)
{
    if (b.p) cudaFree(b.p);
    b.p = nullptr;
    b.bytes = 0;
}

template <typename T> T *AP(ABuf &b) { return reinterpret_cast<T *>(b.p); }

// scratch of one build step, freed when it goes out of scope (on every
// return path); cudaFree waits for the kernels still using it
struct ATmp : ABuf {
    ATmp() = default;
    ATmp(const ATmp &) = delete;
    ATmp &operator=(const ATmp &) = delete;
    ~ATmp() { afree(*this); }
};

bool is_dev(const void *p)
{
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

unsigned nblk(long long n, int t) { return (unsigned)((n + t - 1) / t); }

}  // namespace

struct ccfmm_adaptive_s {
    int device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    int ns = 0;
    long long N = 0;
    int p = 0, K = 0, KP = 0, TD = 0, ldD = 0, maxdeg = 0;
    double theta = 0.0;
    bool dbl = false;
    std::vector<long long> off;
    // autotuner: per size class (floor(log2 N)) its smallest N and split
    std::vector<long long> tune_nmin;
    std::vector<double> tune_split;
    ABuf offd, pos, mom, geo, perm, A, B, H, Hd, E, flags, tmp;
    // cells
    int nc = 0, nleaf = 0, maxL = 0;
    ABuf lev, smp, p0, np, par, ch, ic, cen, leaves, lvl_cells;
    std::vector<int> lvl_off;
    // lists
    long long nfar = 0, nnear = 0;
    unsigned long long near_pairs = 0;
    ABuf near_first, near_num, near_src, far_t, far_s;
    // M2L groups
    int nd = 0, n64 = 0, n16 = 0;
    ABuf pt, ps, sep, rpow, D, it64, it16, fdense, fst, fq, fval, itab;
    ABuf Q, VF, V, shift;
    // harmonic reduction of the FP32 tensor-core M2L
    bool red = false;
    int KRP = 0;
    ABuf Qr, VFr, itr, harm;
    // ensemble step
    ABuf prm;
    RotateParams *hprm = nullptr;
    cudaGraphExec_t gexec[2] = {nullptr, nullptr};  // evaluation, rotation + evaluation
    // the far chain (P2M .. L2L) runs on s_far (highest priority) beside the
    // near field on the handle's stream; off with CCFMM_OVERLAP=0
    bool overlap = true;
    cudaStream_t s_far = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    long long kernels_per_eval = 0;
    double ms_build = 0.0;
    bool evaluated = false;
    // persistent step (k_astep): task queue, tasks per phase, control words
    // (head, err, done per phase) and a pinned copy of err
    bool persistent = false;
    int qntask = 0, qnphase = 0;
    long long qpoll = 1ll << 24;
    ABuf qtasks, qneed, qctl;
    int *hctl = nullptr;
};


namespace {

ccfmm_status read_flags(ccfmm_adaptive_t h)
{
    int f = 0;
    ACK(cudaMemcpyAsync(&f, h->flags.p, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    ACK(cudaStreamSynchronize(h->stream));
    if (f & FLAG_NONFINITE) return afail(CCFMM_ERR_ARG, "non-finite position or degenerate box");
    if (f & FLAG_OFFSET_RANGE)
        return afail(CCFMM_ERR_ARG, "adaptive tree too deep or box too elongated for its cell keys");
    if (f & FLAG_LIST_OVERFLOW) return afail(CCFMM_ERR_ARG, "adaptive list refinement deeper than its stack");
    return CCFMM_OK;
}

template <typename T> ccfmm_status to_host(ccfmm_adaptive_t h, T *dst, const void *src, size_t n)
{
    ACK(cudaMemcpyAsync(dst, src, sizeof(T) * n, cudaMemcpyDeviceToHost, h->stream));
    ACK(cudaStreamSynchronize(h->stream));
    return CCFMM_OK;
}

// 1-2: keys, sort, cells, leaves, levels
ccfmm_status build_tree(ccfmm_adaptive_t h, const double *ubox, const double *split,
                        double s_default, ABuf &stemp)
{
    const cudaStream_t s = h->stream;
    const long long n = h->N;
    const int ns = h->ns;
    ATmp dbox, dsplit;
    if (ubox) {
        ATRY(aalloc(dbox, 6 * sizeof(double)));
        ACK(cudaMemcpyAsync(dbox.p, ubox, 6 * sizeof(double), cudaMemcpyHostToDevice, s));
    }
    if (split) {
        ATRY(aalloc(dsplit, ns * sizeof(double)));
        ACK(cudaMemcpyAsync(dsplit.p, split, ns * sizeof(double), cudaMemcpyHostToDevice, s));
    }
    ATRY(aalloc(h->geo, sizeof(AGeom) * ns));
    note_launch();
    k_ageom<<<ns, 256, 0, s>>>(AP<double>(h->pos), AP<long long>(h->offd),
                               ubox ? AP<double>(dbox) : nullptr,
                               split ? AP<double>(dsplit) : nullptr, s_default, AP<AGeom>(h->geo),
                               AP<int>(h->flags));
    ACK(cudaGetLastError());
    ATmp klo, khi, idx, k2, v2, k3, v3, shi;
    for (ABuf *b : std::initializer_list<ABuf *>{&klo, &khi, &idx, &k2, &v2, &k3, &v3, &shi, &h->perm})
        ATRY(aalloc(*b, 4 * n));
    note_launch();
    k_akeys<<<nblk(n, 256), 256, 0, s>>>(AP<double>(h->pos), n, AP<long long>(h->offd), ns,
                                         AP<AGeom>(h->geo), AP<uint32_t>(klo), AP<uint32_t>(khi),
                                         AP<int>(idx), AP<int>(h->flags));
    ACK(cudaGetLastError());
    ATRY(read_flags(h));
    int sbits = 0;
    while ((1 << sbits) < ns) ++sbits;
    // stable LSD sort by (sample, key): the low word, then the high word
    radix_sort(AP<uint32_t>(klo), AP<int>(idx), AP<uint32_t>(k2), AP<int>(v2), AP<uint32_t>(k3),
               AP<int>(v3), n, 32, stemp.p, s);
    note_launch();
    k_gather_u32<<<nblk(n, 256), 256, 0, s>>>(AP<uint32_t>(khi), AP<int>(v2), n, AP<uint32_t>(k3));
    radix_sort(AP<uint32_t>(k3), AP<int>(v2), AP<uint32_t>(shi), AP<int>(h->perm),
               AP<uint32_t>(k2), AP<int>(v3), n, 8 + sbits, stemp.p, s);
    note_launch();
    k_gather_u32<<<nblk(n, 256), 256, 0, s>>>(AP<uint32_t>(klo), AP<int>(h->perm), n,
                                              AP<uint32_t>(k3));
    ABuf &slo = k3;
    ACK(cudaGetLastError());

    // cells: chain lengths, numbering, cells
    ATmp len, first, total;
    ATRY(aalloc(len, 4 * n));
    ATRY(aalloc(first, 4 * n));
    ATRY(aalloc(total, 64));
    CellOut none{};
    note_launch();
    k_chain<false><<<nblk(n, 256), 256, 0, s>>>(n, AP<long long>(h->offd), AP<AGeom>(h->geo),
                                                AP<uint32_t>(slo), AP<uint32_t>(shi),
                                                AP<int>(len), nullptr, none);
    scan_exclusive(AP<int>(len), AP<int>(first), n, AP<int>(total), stemp.p, s);
    ACK(cudaGetLastError());
    int nc = 0;
    ATRY(to_host(h, &nc, total.p, 1));
    h->nc = nc;
    for (ABuf *b : {&h->lev, &h->smp, &h->p0, &h->np, &h->par}) ATRY(aalloc(*b, 4 * (size_t)nc));
    ATRY(aalloc(h->ch, 8 * (size_t)nc));
    ATRY(aalloc(h->ic, sizeof(int4) * (size_t)nc));
    ATRY(aalloc(h->cen, sizeof(double4) * (size_t)nc));
    ACK(cudaMemsetAsync(h->ch.p, 0xff, 8 * (size_t)nc, s));
    CellOut co{AP<int>(h->lev), AP<int>(h->smp), AP<int>(h->p0), AP<int>(h->np),
               AP<int>(h->par), AP<int>(h->ch), AP<int4>(h->ic), AP<double4>(h->cen)};
    note_launch();
    k_chain<true><<<nblk(n, 256), 256, 0, s>>>(n, AP<long long>(h->offd), AP<AGeom>(h->geo),
                                               AP<uint32_t>(slo), AP<uint32_t>(shi), AP<int>(len),
                                               AP<int>(first), co);
    ACK(cudaGetLastError());

    // leaves, in cell order
    ATmp flag, rank;
    ATRY(aalloc(flag, 4 * (size_t)nc));
    ATRY(aalloc(rank, 4 * (size_t)nc));
    ATRY(aalloc(stemp, std::max(stemp.bytes, std::max(radix_temp_bytes(nc), scan_temp_bytes(nc)))));
    note_launch();
    k_leaf_flag<<<nblk(nc, 256), 256, 0, s>>>(nc, AP<int>(h->ch), AP<int>(flag));
    scan_exclusive(AP<int>(flag), AP<int>(rank), nc, AP<int>(total), stemp.p, s);
    ACK(cudaGetLastError());
    ATRY(to_host(h, &h->nleaf, total.p, 1));
    ATRY(aalloc(h->leaves, 4 * (size_t)h->nleaf));
    note_launch();
    k_leaf_list<<<nblk(nc, 256), 256, 0, s>>>(nc, AP<int>(flag), AP<int>(rank), AP<int>(h->leaves));
    // cells of each level, in cell order (a stable sort by level)
    ATmp cid, lk, lk2, lv2, hist;
    for (ABuf *b : std::initializer_list<ABuf *>{&cid, &lk, &lk2, &lv2, &h->lvl_cells})
        ATRY(aalloc(*b, 4 * (size_t)nc));
    ATRY(aalloc(hist, 4 * (AMAXL + 2)));
    ACK(cudaMemsetAsync(hist.p, 0, 4 * (AMAXL + 2), s));
    note_launch();
    k_iota<<<nblk(nc, 256), 256, 0, s>>>(nc, AP<int>(cid));
    note_launch();
    k_level_hist<<<nblk(nc, 256), 256, 0, s>>>(nc, AP<int>(h->lev), AP<int>(hist));
    radix_sort(AP<uint32_t>(h->lev), AP<int>(cid), AP<uint32_t>(lk), AP<int>(h->lvl_cells),
               AP<uint32_t>(lk2), AP<int>(lv2), nc, 8, stemp.p, s);
    ACK(cudaGetLastError());
    int hh[AMAXL + 2];
    ATRY(to_host(h, hh, hist.p, AMAXL + 2));
    h->lvl_off.assign(AMAXL + 2, 0);
    h->maxL = 0;
    for (int l = 0; l <= AMAXL; ++l) {
        h->lvl_off[l + 1] = h->lvl_off[l] + hh[l];
        if (hh[l]) h->maxL = l;
    }
    return CCFMM_OK;
}

// 3: the lists, level by level
ccfmm_status build_lists(ccfmm_adaptive_t h, ABuf &stemp)
{
    const cudaStream_t s = h->stream;
    const int nc = h->nc, ns = h->ns;
    int maxnl = 0;
    for (int l = 0; l <= h->maxL; ++l) maxnl = std::max(maxnl, h->lvl_off[l + 1] - h->lvl_off[l]);
    ATmp cand_a, cand_b, cfirst, cnum, cnt, off, total;
    ATRY(aalloc(cand_a, 4 * (size_t)std::max(ns, 1)));
    ATRY(aalloc(cfirst, 4 * (size_t)nc));
    ATRY(aalloc(cnum, 4 * (size_t)nc));
    ATRY(aalloc(cnt, 12 * (size_t)maxnl));
    ATRY(aalloc(off, 12 * (size_t)maxnl));
    ATRY(aalloc(total, 64));
    ATRY(aalloc(stemp, std::max(stemp.bytes, scan_temp_bytes(std::max(maxnl, 1)))));
    ATRY(aalloc(h->near_first, 4 * (size_t)nc));
    ATRY(aalloc(h->near_num, 4 * (size_t)nc));
    ACK(cudaMemsetAsync(h->near_first.p, 0, 4 * (size_t)nc, s));
    ACK(cudaMemsetAsync(h->near_num.p, 0, 4 * (size_t)nc, s));
    ABuf &ft = h->far_t, &fs = h->far_s, &nsrc = h->near_src;
    ATRY(aalloc(ft, 4 * (size_t)nc * 16));
    ATRY(aalloc(fs, 4 * (size_t)nc * 16));
    ATRY(aalloc(nsrc, 4 * (size_t)nc * 16));
    note_launch();
    k_root_cand<<<nblk(ns, 128), 128, 0, s>>>(ns, AP<int>(h->lvl_cells), AP<int>(cand_a),
                                             AP<int>(cfirst), AP<int>(cnum));
    ACK(cudaGetLastError());
    long long far_total = 0, near_total = 0;
    ABuf *cur = &cand_a, *nxt = &cand_b;
    const double thth = h->theta * h->theta;
    for (int l = 0; l <= h->maxL; ++l) {
        const int nl = h->lvl_off[l + 1] - h->lvl_off[l];
        if (nl == 0) continue;
        ListArgs a{};
        a.nl = nl;
        a.cells = AP<int>(h->lvl_cells) + h->lvl_off[l];
        a.geo = AP<AGeom>(h->geo);
        a.thth = thth;
        a.lev = AP<int>(h->lev);
        a.smp = AP<int>(h->smp);
        a.ch = AP<int>(h->ch);
        a.cen = AP<double4>(h->cen);
        a.cand = AP<int>(*cur);
        a.cand_first = AP<int>(cfirst);
        a.cand_num = AP<int>(cnum);
        a.cnt = AP<int>(cnt);
        a.flags = AP<int>(h->flags);
        note_launch();
        k_alist<false><<<nblk(nl, AW), 32 * AW, 0, s>>>(a);
        for (int k = 0; k < 3; ++k)
            scan_exclusive(AP<int>(cnt) + (size_t)k * nl, AP<int>(off) + (size_t)k * nl, nl,
                           AP<int>(total) + k, stemp.p, s);
        ACK(cudaGetLastError());
        int tot[3];
        ATRY(to_host(h, tot, total.p, 3));
        if ((long long)far_total + tot[1] > 0x7fffffffll || (long long)near_total + tot[2] > 0x7fffffffll)
            return afail(CCFMM_ERR_ARG, "adaptive interaction lists too large for 32-bit offsets");
        ATRY(aalloc(*nxt, 4 * (size_t)std::max(tot[0], 1)));
        ATRY(agrow(ft, 4 * (size_t)far_total, 4 * (size_t)(far_total + tot[1] + 1), s));
        ATRY(agrow(fs, 4 * (size_t)far_total, 4 * (size_t)(far_total + tot[1] + 1), s));
        ATRY(agrow(nsrc, 4 * (size_t)near_total, 4 * (size_t)(near_total + tot[2] + 1), s));
        a.off = AP<int>(off);
        a.far_base = far_total;
        a.near_base = near_total;
        a.cand_next = AP<int>(*nxt);
        a.cand_first_w = AP<int>(cfirst);
        a.cand_num_w = AP<int>(cnum);
        a.far_t = AP<int>(ft);
        a.far_s = AP<int>(fs);
        a.near_src = AP<int>(nsrc);
        a.near_first = AP<int>(h->near_first);
        a.near_num = AP<int>(h->near_num);
        note_launch();
        k_alist<true><<<nblk(nl, AW), 32 * AW, 0, s>>>(a);
        ACK(cudaGetLastError());
        far_total += tot[1];
        near_total += tot[2];
        std::swap(cur, nxt);
    }
    h->nfar = far_total;
    h->nnear = near_total;
    ATRY(read_flags(h));
    ACK(cudaMemsetAsync(total.p, 0, 8, s));
    note_launch();
    k_near_pairs<<<nblk(h->nleaf, 128), 128, 0, s>>>(
        h->nleaf, AP<int>(h->leaves), AP<int>(h->np), AP<int>(h->near_first), AP<int>(h->near_num),
        AP<int>(h->near_src), AP<unsigned long long>(total));
    ACK(cudaGetLastError());
    ATRY(to_host(h, &h->near_pairs, total.p, 1));
    return CCFMM_OK;
}

// 4: separations, D rows, M2L items
template <typename real> ccfmm_status build_m2l(ccfmm_adaptive_t h, ABuf &stemp)
{
    const cudaStream_t s = h->stream;
    const long long nf = h->nfar;
    const int O = 2 * h->p;
    h->TD = nterms(O);
    h->ldD = ((h->TD + 1 + 3) / 4) * 4;
    ATRY(aalloc(h->fdense, ftable_scratch_bytes(O)));
    ATRY(aalloc(h->fst, sizeof(int) * (h->TD + 1)));
    ATRY(aalloc(h->fq, sizeof(uint16_t) * h->TD * 160));
    ATRY(aalloc(h->fval, sizeof(double) * h->TD * 160));
    launch_ftable(O, AP<double>(h->fdense), AP<int>(h->fst), AP<uint16_t>(h->fq),
                  AP<double>(h->fval), s);
    ATRY(aalloc(h->itab, sizeof(uint16_t) * h->KP * h->KP));
    launch_itable(h->p, h->KP, h->maxdeg, AP<uint16_t>(h->itab), s);
    ATRY(aalloc(h->pt, 4 * (size_t)std::max(nf, 1ll)));
    ATRY(aalloc(h->ps, 4 * (size_t)std::max(nf, 1ll)));
    h->nd = h->n64 = h->n16 = 0;
    if (nf > 0) {
        ATmp K1, K2, K3, K4, V1, V2, V3, V4, khi, ksm, gflag, grank, total;
        for (ABuf *b : std::initializer_list<ABuf *>{&K1, &K2, &K3, &K4, &V1, &V2, &V3, &V4, &khi, &ksm, &gflag, &grank})
            ATRY(aalloc(*b, 4 * (size_t)nf));
        ATRY(aalloc(total, 64));
        ATRY(aalloc(stemp, std::max(stemp.bytes, std::max(radix_temp_bytes(nf), scan_temp_bytes(nf)))));
        note_launch();
        k_dkey<<<nblk(nf, 256), 256, 0, s>>>(nf, AP<int>(h->far_t), AP<int>(h->far_s),
                                             AP<int>(h->lev), AP<int>(h->smp), AP<int4>(h->ic),
                                             AP<AGeom>(h->geo), AP<uint32_t>(K1), AP<uint32_t>(khi),
                                             AP<uint32_t>(ksm), AP<int>(V1), AP<int>(h->flags));
        ACK(cudaGetLastError());
        ATRY(read_flags(h));
        int sbits = 0;
        while ((1 << sbits) < h->ns) ++sbits;
        radix_sort(AP<uint32_t>(K1), AP<int>(V1), AP<uint32_t>(K2), AP<int>(V2), AP<uint32_t>(K3),
                   AP<int>(V3), nf, 32, stemp.p, s);
        note_launch();
        k_gather_u32<<<nblk(nf, 256), 256, 0, s>>>(AP<uint32_t>(khi), AP<int>(V2), nf,
                                                   AP<uint32_t>(K3));
        radix_sort(AP<uint32_t>(K3), AP<int>(V2), AP<uint32_t>(K4), AP<int>(V4), AP<uint32_t>(K2),
                   AP<int>(V3), nf, 31, stemp.p, s);
        note_launch();
        k_gather_u32<<<nblk(nf, 256), 256, 0, s>>>(AP<uint32_t>(ksm), AP<int>(V4), nf,
                                                   AP<uint32_t>(K3));
        int *perm = AP<int>(V4);
        uint32_t *ssm = AP<uint32_t>(K3);
        if (sbits > 0) {
            radix_sort(AP<uint32_t>(K3), AP<int>(V4), AP<uint32_t>(K2), AP<int>(V2),
                       AP<uint32_t>(K4), AP<int>(V3), nf, sbits, stemp.p, s);
            perm = AP<int>(V2);
            ssm = AP<uint32_t>(K2);
        }
        note_launch();
        k_group_flags<<<nblk(nf, 256), 256, 0, s>>>(nf, perm, AP<uint32_t>(K1), AP<uint32_t>(khi),
                                                    ssm, AP<int>(h->far_t), AP<int>(h->far_s),
                                                    AP<int>(h->pt), AP<int>(h->ps), AP<int>(gflag));
        scan_exclusive(AP<int>(gflag), AP<int>(grank), nf, AP<int>(total), stemp.p, s);
        ACK(cudaGetLastError());
        ATRY(to_host(h, &h->nd, total.p, 1));
        const int nd = h->nd;
        ATmp gstart, c64, c16, o64, o16;
        for (ABuf *b : std::initializer_list<ABuf *>{&gstart, &c64, &c16, &o64, &o16})
            ATRY(aalloc(*b, 4 * (size_t)nd));
        ATRY(aalloc(h->sep, sizeof(double4) * (size_t)nd));
        ATRY(aalloc(h->rpow, sizeof(float) * (PMAX + 2) * (size_t)nd));
        note_launch();
        k_group_sep<<<nblk(nf, 256), 256, 0, s>>>(nf, h->p, AP<int>(gflag), AP<int>(grank),
                                                  AP<int>(h->pt), AP<int>(h->ps),
                                                  AP<double4>(h->cen), AP<int>(gstart),
                                                  AP<double4>(h->sep), AP<float>(h->rpow));
        note_launch();
        k_item_count<<<nblk(nd, 256), 256, 0, s>>>(nd, AP<int>(gstart), nf, AP<int>(c64),
                                                   AP<int>(c16));
        scan_exclusive(AP<int>(c64), AP<int>(o64), nd, AP<int>(total), stemp.p, s);
        scan_exclusive(AP<int>(c16), AP<int>(o16), nd, AP<int>(total) + 1, stemp.p, s);
        ACK(cudaGetLastError());
        int nit[2];
        ATRY(to_host(h, nit, total.p, 2));
        h->n64 = nit[0];
        h->n16 = nit[1];
        ATRY(aalloc(h->it64, sizeof(int4) * (size_t)std::max(h->n64, 1)));
        ATRY(aalloc(h->it16, sizeof(int4) * (size_t)std::max(h->n16, 1)));
        note_launch();
        k_item_fill<<<nblk(nd, 256), 256, 0, s>>>(nd, AP<int>(gstart), nf, AP<int>(o64),
                                                  AP<int>(o16), AP<int4>(h->it64),
                                                  AP<int4>(h->it16));
        ATRY(aalloc(h->D, sizeof(real) * (size_t)std::max(nd, 1) * h->ldD));
        launch_dtables<real>(h->p, AP<int>(h->fst), AP<uint16_t>(h->fq), AP<double>(h->fval),
                             AP<double4>(h->sep), nd, AP<real>(h->D), h->ldD, s);
        ACK(cudaGetLastError());
        ACK(cudaStreamSynchronize(s));
    }
    ATRY(aalloc(h->shift, sizeof(ShiftTab)));
    note_launch();
    k_shift_tab<<<1, KPMAX, 0, s>>>(h->p, AP<ShiftTab>(h->shift));
    h->red = sizeof(real) == 4 && h->maxdeg >= 2 * h->p && am2l_mma_ok(h->p);
    ATRY(aalloc(h->harm, sizeof(HarmTab)));
    note_launch();
    k_harm_tab<<<1, KPMAX, 0, s>>>(h->p, AP<HarmTab>(h->harm));
    if (h->red) {
        h->KRP = red_padded(h->p);
        ATRY(aalloc(h->itr, sizeof(uint16_t) * h->KRP * h->KRP));
        launch_itable_red(h->p, h->KP, h->KRP, AP<uint16_t>(h->itab), AP<uint16_t>(h->itr), s);
        ATRY(aalloc(h->Qr, sizeof(float) * (size_t)h->nc * h->KRP));
        ATRY(aalloc(h->VFr, sizeof(float) * (size_t)h->nc * h->KRP));
    }
    const size_t cells = (size_t)h->nc * h->KP;
    ATRY(aalloc(h->Q, sizeof(real) * cells));
    ATRY(aalloc(h->VF, sizeof(real) * cells));
    ATRY(aalloc(h->V, sizeof(double) * cells));
    ATRY(aalloc(h->A, sizeof(typename vec4<real>::t) * (size_t)h->N));
    ATRY(aalloc(h->B, sizeof(typename vec2<real>::t) * (size_t)h->N));
    ATRY(aalloc(h->H, sizeof(typename vec4<real>::t) * (size_t)h->N));
    ATRY(aalloc(h->Hd, sizeof(double) * 3 * (size_t)h->N));
    ATRY(aalloc(h->E, sizeof(double) * (size_t)h->ns));
    note_launch();
    k_apoints<real><<<nblk(h->nleaf, AW), 32 * AW, 0, s>>>(
        h->nleaf, AP<int>(h->leaves), AP<int>(h->p0), AP<int>(h->np), AP<double4>(h->cen),
        AP<int>(h->perm), AP<double>(h->pos), AP<typename vec4<real>::t>(h->A));
    ACK(cudaGetLastError());
    return CCFMM_OK;
}

// one evaluation (with the ensemble rotation first when rotate).  With the
// overlap on, the near field (without the smooth field) runs on the handle's
// stream while P2M, M2M, M2L and L2L run on the high-priority stream; the
// smooth field is added after the join.
void enqueue_persistent(ccfmm_adaptive_t h, bool rotate)
{
    const cudaStream_t s = h->stream;
    cudaMemsetAsync(h->VFr.p, 0, sizeof(float) * (size_t)h->nc * h->KRP, s);
    cudaMemsetAsync(h->qctl.p, 0, sizeof(int) * (2 + (size_t)h->qnphase), s);
    AStepArgs a;
    a.tasks = AP<int4>(h->qtasks);
    a.ntask = h->qntask;
    a.ctl = AP<int>(h->qctl);
    a.need = AP<int>(h->qneed);
    a.poll_limit = h->qpoll;
    a.rotate = rotate ? 1 : 0;
    a.p = h->p;
    a.KP = h->KP;
    a.KRP = h->KRP;
    a.ldD = h->ldD;
    a.n16 = h->n16;
    a.nc = h->nc;
    a.N = h->N;
    a.mom = AP<double>(h->mom);
    a.prm = AP<RotateParams>(h->prm);
    a.perm = AP<int>(h->perm);
    a.A = AP<float4>(h->A);
    a.H = AP<float4>(h->H);
    a.B = AP<float2>(h->B);
    a.Hd = AP<double>(h->Hd);
    a.E = AP<double>(h->E);
    a.V = AP<double>(h->V);
    a.offd = AP<long long>(h->offd);
    a.leaves = AP<int>(h->leaves);
    a.p0 = AP<int>(h->p0);
    a.np = AP<int>(h->np);
    a.near_first = AP<int>(h->near_first);
    a.near_num = AP<int>(h->near_num);
    a.near_src = AP<int>(h->near_src);
    a.cen = AP<double4>(h->cen);
    a.Q = AP<float>(h->Q);
    a.Qr = AP<float>(h->Qr);
    a.VFr = AP<float>(h->VFr);
    a.lvl_cells = AP<int>(h->lvl_cells);
    a.smp = AP<int>(h->smp);
    a.lev = AP<int>(h->lev);
    a.ch = AP<int>(h->ch);
    a.par = AP<int>(h->par);
    a.ic = AP<int4>(h->ic);
    a.geo = AP<AGeom>(h->geo);
    a.shift = AP<ShiftTab>(h->shift);
    a.harm = AP<HarmTab>(h->harm);
    a.it64 = AP<int4>(h->it64);
    a.it16 = AP<int4>(h->it16);
    a.pt = AP<int>(h->pt);
    a.ps = AP<int>(h->ps);
    a.rpow = AP<float>(h->rpow);
    a.D = AP<float>(h->D);
    a.itr = AP<uint16_t>(h->itr);
    launch_astep(h->p, a, s);
    h->kernels_per_eval = 1;
}

template <typename real> void enqueue_eval(ccfmm_adaptive_t h, bool rotate)
{
    typedef typename vec4<real>::t R4;
    typedef typename vec2<real>::t R2;
    const cudaStream_t s = h->stream;
    const cudaStream_t sf = h->overlap ? h->s_far : s;
    long long k = 0;
    if (rotate) {
        launch_rotate(AP<double>(h->mom), h->N, AP<RotateParams>(h->prm), s);
        ++k;
    }
    launch_permute_moments<real>(AP<double>(h->mom), AP<int>(h->perm), h->N, AP<R4>(h->A),
                                 AP<R2>(h->B), s);
    ++k;
    if (h->overlap) {
        cudaEventRecord(h->ev_fork, s);
        cudaStreamWaitEvent(sf, h->ev_fork, 0);
        launch_ap2p<real>(h->p, h->KP, h->nleaf, AP<int>(h->leaves), AP<int>(h->p0),
                          AP<int>(h->np), AP<int>(h->near_first), AP<int>(h->near_num),
                          AP<int>(h->near_src), AP<double4>(h->cen), AP<R4>(h->A), AP<R2>(h->B),
                          nullptr, AP<R4>(h->H), s);
        ++k;
    }
    launch_ap2m<real>(h->p, h->KP, h->nleaf, AP<int>(h->leaves), AP<int>(h->p0), AP<int>(h->np),
                      AP<R4>(h->A), AP<R2>(h->B), AP<real>(h->Q), sf);
    ++k;
    for (int l = h->maxL - 1; l >= 0; --l) {
        const int ncl = h->lvl_off[l + 1] - h->lvl_off[l];
        if (ncl == 0) continue;
        note_launch();
        k_am2m<real><<<nblk(ncl, AW), 32 * AW, 0, sf>>>(
            h->p, h->KP, AP<int>(h->lvl_cells) + h->lvl_off[l], ncl, AP<int>(h->smp),
            AP<int>(h->lev), AP<int>(h->ch), AP<AGeom>(h->geo), AP<ShiftTab>(h->shift),
            AP<real>(h->Q));
        ++k;
    }
    if (h->red) {
        launch_afold(h->p, h->KP, h->KRP, h->nc, AP<float>(h->Q), AP<float>(h->Qr), sf);
        ++k;
        cudaMemsetAsync(h->VFr.p, 0, sizeof(float) * (size_t)h->nc * h->KRP, sf);
        launch_am2l_red(h->p, h->KRP, AP<int4>(h->it64), h->n64, 64, AP<int>(h->pt),
                        AP<int>(h->ps), AP<float>(h->rpow), AP<float>(h->D), h->ldD,
                        AP<uint16_t>(h->itr), AP<float>(h->Qr), AP<float>(h->VFr), sf);
        launch_am2l_red(h->p, h->KRP, AP<int4>(h->it16), h->n16, 16, AP<int>(h->pt),
                        AP<int>(h->ps), AP<float>(h->rpow), AP<float>(h->D), h->ldD,
                        AP<uint16_t>(h->itr), AP<float>(h->Qr), AP<float>(h->VFr), sf);
    } else {
        cudaMemsetAsync(h->VF.p, 0, sizeof(real) * (size_t)h->nc * h->KP, sf);
        launch_am2l<real>(h->p, h->KP, AP<int4>(h->it64), h->n64, 64, AP<int>(h->pt),
                          AP<int>(h->ps), AP<double4>(h->sep), AP<float>(h->rpow), AP<real>(h->D),
                          h->ldD, AP<uint16_t>(h->itab), h->maxdeg, AP<real>(h->Q),
                          AP<real>(h->VF), sf);
        launch_am2l<real>(h->p, h->KP, AP<int4>(h->it16), h->n16, 16, AP<int>(h->pt),
                          AP<int>(h->ps), AP<double4>(h->sep), AP<float>(h->rpow), AP<real>(h->D),
                          h->ldD, AP<uint16_t>(h->itab), h->maxdeg, AP<real>(h->Q),
                          AP<real>(h->VF), sf);
    }
    k += (h->n64 > 0) + (h->n16 > 0);
    for (int l = 0; l <= h->maxL; ++l) {
        const int ncl = h->lvl_off[l + 1] - h->lvl_off[l];
        if (ncl == 0) continue;
        note_launch();
        if (h->red)
            k_al2l<float, true><<<nblk(ncl, AW), 32 * AW, 0, sf>>>(
                h->p, h->KP, h->KRP, AP<int>(h->lvl_cells) + h->lvl_off[l], ncl, AP<int>(h->smp),
                AP<int>(h->lev), AP<int>(h->par), AP<int4>(h->ic), AP<AGeom>(h->geo),
                AP<ShiftTab>(h->shift), AP<HarmTab>(h->harm), AP<float>(h->VFr), AP<double>(h->V));
        else
            k_al2l<real, false><<<nblk(ncl, AW), 32 * AW, 0, sf>>>(
                h->p, h->KP, h->KP, AP<int>(h->lvl_cells) + h->lvl_off[l], ncl, AP<int>(h->smp),
                AP<int>(h->lev), AP<int>(h->par), AP<int4>(h->ic), AP<AGeom>(h->geo),
                AP<ShiftTab>(h->shift), AP<HarmTab>(h->harm), AP<real>(h->VF), AP<double>(h->V));
        ++k;
    }
    if (h->overlap) {
        cudaEventRecord(h->ev_join, sf);
        cudaStreamWaitEvent(s, h->ev_join, 0);
        launch_al2p<real>(h->p, h->KP, h->nleaf, AP<int>(h->leaves), AP<int>(h->p0),
                          AP<int>(h->np), AP<R4>(h->A), AP<double>(h->V), AP<R4>(h->H), s);
    } else {
        launch_ap2p<real>(h->p, h->KP, h->nleaf, AP<int>(h->leaves), AP<int>(h->p0),
                          AP<int>(h->np), AP<int>(h->near_first), AP<int>(h->near_num),
                          AP<int>(h->near_src), AP<double4>(h->cen), AP<R4>(h->A), AP<R2>(h->B),
                          AP<double>(h->V), AP<R4>(h->H), s);
    }
    ++k;
    note_launch(2);
    k_aunperm<real><<<nblk(h->N, 256), 256, 0, s>>>(h->N, AP<int>(h->perm), AP<R4>(h->H),
                                                    AP<double>(h->Hd));
    k_aenergy<<<h->ns, 256, 0, s>>>(AP<long long>(h->offd), AP<double>(h->mom), AP<double>(h->Hd),
                                    AP<double>(h->E));
    k += 2;
    h->kernels_per_eval = k - (rotate ? 1 : 0);
}

// The task queue of the persistent step (k_astep), in the order the blocks
// take it: the rotation, the moment permutation, then the far chain's phases
// (P2M; M2M level by level from the deepest; the fold; the M2L items; L2L
// level by level from the roots), each waiting for the one before it, with
// an equal share of the near-field leaves after each phase (they wait only
// for the permutation and keep the SMs busy while a level completes); then
// L2P (waits for the last L2L level and the whole near field), the unpermute
// and the energies.  CCFMM_ASTEP_STALL=1 (tests of the time-out path) asks
// one task more of the M2L phase than it has and lets every wait give up
// after 2^12 polls.
// Shape of a forest for the persistent step's task queue.
struct AQShape {
    long long N;
    int ns, nleaf, nc, maxL, n64, n16;
    const int *lvl_off;  // maxL + 2 offsets of each level's cells in the level-ordered list
};

// The task queue of the persistent step (k_astep) for a forest of shape q:
// t in queue order, need[ph] = tasks of phase ph, ph_m2l = the M2L phase.
void build_queue(const AQShape &q, std::vector<int4> &t, std::vector<int> &need, int &ph_m2l)
{
    t.clear();
    need.clear();
    auto phase = [&]() {
        need.push_back(0);
        return (int)need.size() - 1;
    };
    auto add = [&](int type, int ph, long long y, long long z, int w1, int w2) {
        t.push_back(make_int4(type | (ph << 8), (int)y, (int)z, (w1 + 1) | ((w2 + 1) << 16)));
        ++need[ph];
    };
    const long long nch = (q.N + ACHUNK - 1) / ACHUNK;
    const int ph_rot = phase();
    for (long long i = 0; i < nch; ++i) add(AT_ROT, ph_rot, i, 0, -1, -1);
    const int ph_perm = phase();
    for (long long i = 0; i < nch; ++i) add(AT_PERM, ph_perm, i, 0, ph_rot, -1);
    // far-chain phases: (type, y, z) of each task
    std::vector<std::vector<int3>> far;
    auto level_tasks = [&](int type, int l) {
        const int a = q.lvl_off[l], b = q.lvl_off[l + 1];
        if (b <= a) return;
        far.emplace_back();
        for (int i = a; i < b; i += ACELLS) far.back().push_back(make_int3(type, i, b));
    };
    far.emplace_back();
    for (int li = 0; li < q.nleaf; li += ACELLS) far.back().push_back(make_int3(AT_P2M, li, q.nleaf));
    for (int l = q.maxL - 1; l >= 0; --l) level_tasks(AT_M2M, l);
    far.emplace_back();
    for (int c = 0; c < q.nc; c += ACELLS) far.back().push_back(make_int3(AT_FOLD, c, q.nc));
    const size_t m2l_phase = far.size();
    far.emplace_back();
    for (int i = 0; i < q.n64; ++i) far.back().push_back(make_int3(AT_M2L_BIG, i, 0));
    const int ng = (q.n16 + 3) / 4;
    for (int g = 0; g < ng; g += AGROUPS) far.back().push_back(make_int3(AT_M2L_SMALL, g, ng));
    for (int l = 0; l <= q.maxL; ++l) level_tasks(AT_L2L, l);
    const int ph_p2p = phase();
    int prev = ph_perm;
    ph_m2l = -1;
    long long next = 0;
    const long long nf = (long long)far.size();
    for (long long k = 0; k < nf; ++k) {
        const int ph = phase();
        if ((size_t)k == m2l_phase) ph_m2l = ph;
        for (const int3 &x : far[k]) add(x.x, ph, x.y, x.z, prev, -1);
        prev = ph;
        for (const long long upto = (long long)q.nleaf * (k + 1) / (nf + 1); next < upto; ++next)
            add(AT_P2P, ph_p2p, next, 0, ph_perm, -1);
    }
    for (; next < q.nleaf; ++next) add(AT_P2P, ph_p2p, next, 0, ph_perm, -1);
    const int ph_l2p = phase();
    for (int li = 0; li < q.nleaf; li += ACELLS) add(AT_L2P, ph_l2p, li, q.nleaf, prev, ph_p2p);
    const int ph_un = phase();
    for (long long i = 0; i < nch; ++i) add(AT_UNPERM, ph_un, i, 0, ph_l2p, -1);
    const int ph_e = phase();
    for (int i = 0; i < q.ns; ++i) add(AT_ENERGY, ph_e, i, 0, ph_un, -1);
}

ccfmm_status enable_persistent(ccfmm_adaptive_t h)
{
    if (h->dbl || !h->red || h->p < 2 || h->p > 6)
        return afail(CCFMM_ERR_ARG, "the persistent step needs the FP32 path with the "
                                    "tensor-core M2L (p in 2..6)");
    std::vector<int4> t;
    std::vector<int> need;
    int ph_m2l = -1;
    build_queue(AQShape{h->N, h->ns, h->nleaf, h->nc, h->maxL, h->n64, h->n16, h->lvl_off.data()},
                t, need, ph_m2l);
    if ((long long)t.size() > INT32_MAX / 2 || need.size() > 0xfffe)
        return afail(CCFMM_ERR_ARG, "forest too large for the persistent step's task queue");
    const char *e = getenv("CCFMM_ASTEP_STALL");
    if (e && atoi(e) != 0 && ph_m2l >= 0) {
        ++need[ph_m2l];
        h->qpoll = 1ll << 12;
    }
    ATRY(aalloc(h->qtasks, sizeof(int4) * t.size()));
    ATRY(aalloc(h->qneed, sizeof(int) * need.size()));
    ATRY(aalloc(h->qctl, sizeof(int) * (2 + need.size())));
    if (!h->hctl && cudaMallocHost(&h->hctl, sizeof(int)) != cudaSuccess) {
        cudaGetLastError();
        h->hctl = nullptr;
        return afail(CCFMM_ERR_ALLOC, "pinned allocation failed");
    }
    ACK(cudaMemcpy(h->qtasks.p, t.data(), sizeof(int4) * t.size(), cudaMemcpyHostToDevice));
    ACK(cudaMemcpy(h->qneed.p, need.data(), sizeof(int) * need.size(), cudaMemcpyHostToDevice));
    h->qntask = (int)t.size();
    h->qnphase = (int)need.size();
    h->kernels_per_eval = 1;
    for (int i = 0; i < 2; ++i)
        if (h->gexec[i]) {
            cudaGraphExecDestroy(h->gexec[i]);
            h->gexec[i] = nullptr;
        }
    h->persistent = true;
    return CCFMM_OK;
}

ccfmm_status run(ccfmm_adaptive_t h, int rotate, double *H_out, double *E_out)
{
    const cudaStream_t s = h->stream;
    if (!h->gexec[rotate]) {
        cudaGraph_t g = nullptr;
        ACK(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
        if (h->persistent)
            enqueue_persistent(h, rotate != 0);
        else if (h->dbl)
            enqueue_eval<double>(h, rotate != 0);
        else
            enqueue_eval<float>(h, rotate != 0);
        cudaError_t e = cudaStreamEndCapture(s, &g);
        if (e != cudaSuccess) {
            cudaGetLastError();
            if (g) cudaGraphDestroy(g);
            return afail(CCFMM_ERR_CUDA, "graph capture failed: %s", cudaGetErrorString(e));
        }
        e = cudaGraphInstantiate(&h->gexec[rotate], g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) {
            cudaGetLastError();
            h->gexec[rotate] = nullptr;
            return afail(CCFMM_ERR_CUDA, "graph instantiation failed: %s", cudaGetErrorString(e));
        }
    }
    else
        note_launch((int)(h->kernels_per_eval + (h->persistent ? 0 : rotate)));
    ACK(cudaGraphLaunch(h->gexec[rotate], s));
    if (H_out)
        ACK(cudaMemcpyAsync(H_out, h->Hd.p, sizeof(double) * 3 * (size_t)h->N,
                            is_dev(H_out) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s));
    if (E_out)
        ACK(cudaMemcpyAsync(E_out, h->E.p, sizeof(double) * (size_t)h->ns,
                            is_dev(E_out) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s));
    if (h->persistent)
        ACK(cudaMemcpyAsync(h->hctl, AP<int>(h->qctl) + 1, sizeof(int), cudaMemcpyDeviceToHost, s));
    ACK(cudaStreamSynchronize(s));
    if (h->persistent && *h->hctl)
        return afail(CCFMM_ERR_TIMEOUT, "persistent step: a bounded wait between its stages gave up");
    h->evaluated = true;
    return CCFMM_OK;
}

}  // namespace

// ================================================================== C-ABI
extern "C" {

ccfmm_status fmm_adaptive_queue(int64_t N, int32_t nsamples, int32_t nleaf, int32_t ncells,
                                int32_t max_level, const int32_t *level_offsets, int32_t n_big,
                                int32_t n_small, int32_t *tasks, int64_t capacity,
                                int64_t *ntasks, int32_t *need, int32_t need_capacity,
                                int32_t *nphases, int32_t *tiles)
{
    set_last_error("");
    if (!ntasks || !nphases || !level_offsets) return afail(CCFMM_ERR_ARG, "NULL argument");
    if (N < 1 || nsamples < 1 || nleaf < 1 || ncells < nleaf || max_level < 0 ||
        max_level > AMAXL || n_big < 0 || n_small < 0 || capacity < 0 || need_capacity < 0)
        return afail(CCFMM_ERR_ARG, "bad forest shape");
    if (level_offsets[0] != 0 || level_offsets[max_level + 1] != ncells)
        return afail(CCFMM_ERR_ARG, "level offsets must run from 0 to ncells");
    for (int l = 0; l <= max_level; ++l)
        if (level_offsets[l + 1] < level_offsets[l])
            return afail(CCFMM_ERR_ARG, "level offsets must not decrease");
    std::vector<int4> t;
    std::vector<int> need_v;
    int ph_m2l = -1;
    build_queue(AQShape{N, nsamples, nleaf, ncells, max_level, n_big, n_small, level_offsets},
                t, need_v, ph_m2l);
    *ntasks = (int64_t)t.size();
    *nphases = (int32_t)need_v.size();
    if (tasks)
        for (size_t i = 0; i < t.size() && (int64_t)i < capacity; ++i) {
            tasks[4 * i] = t[i].x;
            tasks[4 * i + 1] = t[i].y;
            tasks[4 * i + 2] = t[i].z;
            tasks[4 * i + 3] = t[i].w;
        }
    if (need)
        for (size_t i = 0; i < need_v.size() && (int64_t)i < need_capacity; ++i) need[i] = need_v[i];
    if (tiles) {
        tiles[0] = ACHUNK;
        tiles[1] = ACELLS;
        tiles[2] = AGROUPS;
    }
    return CCFMM_OK;
}

void fmm_adaptive_destroy(ccfmm_adaptive_t h)
{
    if (!h) return;
    cudaSetDevice(h->device);
    if (h->stream) cudaStreamSynchronize(h->stream);
    for (int i = 0; i < 2; ++i)
        if (h->gexec[i]) cudaGraphExecDestroy(h->gexec[i]);
    ABuf *bufs[] = {&h->offd, &h->pos, &h->mom, &h->geo, &h->perm, &h->A, &h->B, &h->H, &h->Hd,
                    &h->E, &h->flags, &h->tmp, &h->lev, &h->smp, &h->p0, &h->np, &h->par, &h->ch,
                    &h->ic, &h->cen, &h->leaves, &h->lvl_cells, &h->near_first, &h->near_num,
                    &h->near_src, &h->far_t, &h->far_s, &h->pt, &h->ps, &h->sep, &h->rpow, &h->D, &h->it64,
                    &h->it16, &h->fdense, &h->fst, &h->fq, &h->fval, &h->itab, &h->Q, &h->VF,
                    &h->V, &h->shift, &h->Qr, &h->VFr, &h->itr, &h->harm, &h->prm,
                    &h->qtasks, &h->qneed, &h->qctl};
    for (ABuf *b : bufs) afree(*b);
    if (h->hprm) cudaFreeHost(h->hprm);
    if (h->hctl) cudaFreeHost(h->hctl);
    if (h->ev_fork) cudaEventDestroy(h->ev_fork);
    if (h->ev_join) cudaEventDestroy(h->ev_join);
    if (h->s_far) cudaStreamDestroy(h->s_far);
    if (h->own_stream && h->stream) cudaStreamDestroy(h->stream);
    delete h;
}

static ccfmm_status adaptive_create(const double *positions, const double *moments,
                                    const int64_t *offsets, int nsamples, int p, double theta,
                                    const double *split, const double *box, ccfmm_prec prec,
                                    void *stream, ccfmm_adaptive_t *out)
{
    set_last_error("");
    if (!out) return afail(CCFMM_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (!positions || !moments || !offsets) return afail(CCFMM_ERR_ARG, "NULL array");
    if (nsamples < 1 || nsamples > (1 << 20)) return afail(CCFMM_ERR_ARG, "bad nsamples");
    if (p < 1 || p > PMAX) return afail(CCFMM_ERR_ARG, "p must be in 1..%d", PMAX);
    if (!(theta > 0.0 && theta < 1.0)) return afail(CCFMM_ERR_ARG, "theta must be in (0, 1)");
    if (prec != CCFMM_MIXED && prec != CCFMM_FP64) return afail(CCFMM_ERR_ARG, "bad precision");
    if (box && nsamples != 1) return afail(CCFMM_ERR_ARG, "a box is accepted for one sample only");
    if (offsets[0] != 0) return afail(CCFMM_ERR_ARG, "offsets[0] must be 0");
    for (int i = 0; i < nsamples; ++i)
        if (offsets[i + 1] <= offsets[i]) return afail(CCFMM_ERR_ARG, "every sample needs a dipole");
    const long long N = offsets[nsamples];
    if (N > 0x7fffffffll / 2) return afail(CCFMM_ERR_ARG, "too many dipoles");
    if (split)
        for (int i = 0; i < nsamples; ++i)
            if (!(split[i] >= 1.0)) return afail(CCFMM_ERR_ARG, "split thresholds must be >= 1");
    if (box)
        for (int a = 0; a < 3; ++a)
            if (!(box[3 + a] > box[a])) return afail(CCFMM_ERR_ARG, "empty box");
    ccfmm_adaptive_t h = new ccfmm_adaptive_s();
    cudaGetDevice(&h->device);
    auto bail = [&](ccfmm_status st) {
        std::string msg = ccfmm_last_error();
        fmm_adaptive_destroy(h);
        set_last_error(msg.c_str());
        return st;
    };
    if (stream) {
        h->stream = (cudaStream_t)stream;
    } else {
        if (cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking) != cudaSuccess) {
            cudaGetLastError();
            delete h;
            return afail(CCFMM_ERR_CUDA, "stream creation failed");
        }
        h->own_stream = true;
    }
    {
        const char *e = getenv("CCFMM_OVERLAP");
        h->overlap = !(e && strcmp(e, "0") == 0);
        int least = 0, greatest = 0;
        if (cudaDeviceGetStreamPriorityRange(&least, &greatest) != cudaSuccess ||
            cudaStreamCreateWithPriority(&h->s_far, cudaStreamNonBlocking, greatest) != cudaSuccess ||
            cudaEventCreateWithFlags(&h->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&h->ev_join, cudaEventDisableTiming) != cudaSuccess) {
            cudaGetLastError();
            afail(CCFMM_ERR_CUDA, "stream or event creation failed");
            return bail(CCFMM_ERR_CUDA);
        }
    }
    h->ns = nsamples;
    h->N = N;
    h->p = p;
    h->K = nterms(p) - 1;
    h->KP = padded_k(p);
    h->maxdeg = 2 * p;
    h->theta = theta;
    h->dbl = prec == CCFMM_FP64;
    h->off.assign(offsets, offsets + nsamples + 1);
    const auto t0 = std::chrono::steady_clock::now();
    ccfmm_status st;
#define BTRY(x)                                                                                  \
    do {                                                                                         \
        st = (x);                                                                                \
        if (st != CCFMM_OK) return bail(st);                                                     \
    } while (0)
    BTRY(aalloc(h->offd, sizeof(long long) * (nsamples + 1)));
    BTRY(aalloc(h->pos, sizeof(double) * 3 * N));
    BTRY(aalloc(h->mom, sizeof(double) * 3 * N));
    BTRY(aalloc(h->flags, 16));
    BTRY(aalloc(h->prm, sizeof(RotateParams)));
    if (cudaMallocHost(&h->hprm, sizeof(RotateParams)) != cudaSuccess) {
        cudaGetLastError();
        h->hprm = nullptr;
        afail(CCFMM_ERR_ALLOC, "pinned allocation failed");
        return bail(CCFMM_ERR_ALLOC);
    }
    const cudaStream_t s = h->stream;
    if (cudaMemcpyAsync(h->offd.p, h->off.data(), sizeof(long long) * (nsamples + 1),
                        cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaMemcpyAsync(h->pos.p, positions, sizeof(double) * 3 * N,
                        is_dev(positions) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                        s) != cudaSuccess ||
        cudaMemcpyAsync(h->mom.p, moments, sizeof(double) * 3 * N,
                        is_dev(moments) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                        s) != cudaSuccess ||
        cudaMemsetAsync(h->flags.p, 0, 16, s) != cudaSuccess) {
        cudaGetLastError();
        afail(CCFMM_ERR_CUDA, "input upload failed");
        return bail(CCFMM_ERR_CUDA);
    }
    const double s_default = p > 3 ? 0.74 * (double)p * (double)p : 8.0;
    ATmp stemp;
    st = aalloc(stemp, std::max(radix_temp_bytes(N), scan_temp_bytes(N)));
    if (st == CCFMM_OK) st = build_tree(h, box, split, s_default, stemp);
    if (st == CCFMM_OK) st = build_lists(h, stemp);
    if (st == CCFMM_OK) st = h->dbl ? build_m2l<double>(h, stemp) : build_m2l<float>(h, stemp);
    if (st == CCFMM_OK && cudaStreamSynchronize(s) != cudaSuccess) {
        cudaGetLastError();
        st = afail(CCFMM_ERR_CUDA, "adaptive build failed");
    }
    afree(stemp);
    if (st != CCFMM_OK) return bail(st);
#undef BTRY
    h->ms_build = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    *out = h;
    return CCFMM_OK;
}

ccfmm_status fmm_adaptive_create(const double *positions, const double *moments,
                                 const int64_t *offsets, int nsamples, int p, double theta,
                                 const double *split, const double *box, ccfmm_prec prec,
                                 void *stream, ccfmm_adaptive_t *out)
{
    return adaptive_create(positions, moments, offsets, nsamples, p, theta, split, box, prec,
                           stream, out);
}

// Autotuner of the split threshold: samples are grouped by floor(log2 N);
// for each class, up to 16 of its samples (spread over its sizes) form a
// trial forest for every candidate s = s0 x {1, sqrt2, 2, 2 sqrt2, 4}
// (s0 = the given split, or Eq. so), timed over `trials` evaluations after
// one warm-up; the fastest mean wins, and the final forest takes each
// sample's class threshold.
static ccfmm_status adaptive_create_tuned(const double *positions, const double *moments,
                                         const int64_t *offsets, int nsamples, int p,
                                         double theta, const double *split, const double *box,
                                         ccfmm_prec prec, const ccfmm_adaptive_opts *opts,
                                         void *stream, ccfmm_adaptive_t *out)
{
    set_last_error("");
    if (!out || !positions || !moments || !offsets || nsamples < 1)
        return afail(CCFMM_ERR_ARG, "bad argument");
    if (p < 1 || p > PMAX) return afail(CCFMM_ERR_ARG, "p must be in 1..%d", PMAX);
    for (int i = 0; i < nsamples; ++i)
        if (offsets[i + 1] <= offsets[i]) return afail(CCFMM_ERR_ARG, "every sample needs a dipole");
    const int trials = opts->trials > 0 ? opts->trials : 3;
    const double s0 = p > 3 ? 0.74 * (double)p * (double)p : 8.0;
    const double mult[5] = {1.0, 1.4142135623730951, 2.0, 2.8284271247461903, 4.0};
    std::vector<int> cls(nsamples);
    int ncls = 0;
    for (int i = 0; i < nsamples; ++i) {
        long long n = offsets[i + 1] - offsets[i];
        int c = 0;
        while ((2ll << c) <= n) ++c;
        cls[i] = c;
        ncls = std::max(ncls, c + 1);
    }
    std::vector<double> best(ncls, 0.0);
    std::vector<long long> nmin(ncls, -1);
    for (int c = 0; c < ncls; ++c) {
        std::vector<int> mem;
        for (int i = 0; i < nsamples; ++i)
            if (cls[i] == c) mem.push_back(i);
        if (mem.empty()) continue;
        std::sort(mem.begin(), mem.end(), [&](int a, int b) {
            return offsets[a + 1] - offsets[a] < offsets[b + 1] - offsets[b];
        });
        nmin[c] = offsets[mem[0] + 1] - offsets[mem[0]];
        std::vector<int> pick;
        const int take = std::min<int>((int)mem.size(), 16);
        for (int j = 0; j < take; ++j) pick.push_back(mem[(size_t)j * mem.size() / take]);
        std::vector<int64_t> toff(1, 0);
        for (int i : pick) toff.push_back(toff.back() + offsets[i + 1] - offsets[i]);
        double *tpos = nullptr, *tmom = nullptr;
        if (cudaMalloc(&tpos, sizeof(double) * 3 * toff.back()) != cudaSuccess ||
            cudaMalloc(&tmom, sizeof(double) * 3 * toff.back()) != cudaSuccess) {
            cudaGetLastError();
            cudaFree(tpos);
            return afail(CCFMM_ERR_ALLOC, "autotuner allocation failed");
        }
        for (size_t j = 0; j < pick.size(); ++j) {
            const size_t nb = sizeof(double) * 3 * (offsets[pick[j] + 1] - offsets[pick[j]]);
            cudaMemcpy(tpos + 3 * toff[j], positions + 3 * offsets[pick[j]], nb, cudaMemcpyDefault);
            cudaMemcpy(tmom + 3 * toff[j], moments + 3 * offsets[pick[j]], nb, cudaMemcpyDefault);
        }
        const double base = split ? split[mem[mem.size() / 2]] : s0;
        double tbest = 1e300;
        for (double m : mult) {
            const double sv = base * m;
            std::vector<double> sp(pick.size(), sv);
            ccfmm_adaptive_t t = nullptr;
            ccfmm_status st = adaptive_create(tpos, tmom, toff.data(), (int)pick.size(), p, theta,
                                              sp.data(), nullptr, prec, stream, &t);
            if (st != CCFMM_OK) {
                cudaFree(tpos);
                cudaFree(tmom);
                return st;
            }
            st = run(t, 0, nullptr, nullptr);
            const auto a0 = std::chrono::steady_clock::now();
            for (int r = 0; r < trials && st == CCFMM_OK; ++r) st = run(t, 0, nullptr, nullptr);
            const double ms =
                std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - a0).count() / trials;
            fmm_adaptive_destroy(t);
            if (st != CCFMM_OK) {
                cudaFree(tpos);
                cudaFree(tmom);
                return st;
            }
            if (ms < tbest) {
                tbest = ms;
                best[c] = sv;
            }
        }
        cudaFree(tpos);
        cudaFree(tmom);
    }
    std::vector<double> sp(nsamples);
    for (int i = 0; i < nsamples; ++i) sp[i] = best[cls[i]];
    ccfmm_status st = adaptive_create(positions, moments, offsets, nsamples, p, theta, sp.data(),
                                      box, prec, stream, out);
    if (st != CCFMM_OK) return st;
    for (int c = 0; c < ncls; ++c)
        if (nmin[c] >= 0) {
            (*out)->tune_nmin.push_back(nmin[c]);
            (*out)->tune_split.push_back(best[c]);
        }
    return CCFMM_OK;
}

ccfmm_status fmm_adaptive_create_ex(const double *positions, const double *moments,
                                    const int64_t *offsets, int nsamples, int p, double theta,
                                    const double *split, const double *box, ccfmm_prec prec,
                                    const ccfmm_adaptive_opts *opts, void *stream,
                                    ccfmm_adaptive_t *out)
{
    ccfmm_status st =
        (opts && opts->autotune)
            ? adaptive_create_tuned(positions, moments, offsets, nsamples, p, theta, split, box,
                                    prec, opts, stream, out)
            : adaptive_create(positions, moments, offsets, nsamples, p, theta, split, box, prec,
                              stream, out);
    if (st != CCFMM_OK || !opts || !opts->persistent) return st;
    st = enable_persistent(*out);
    if (st != CCFMM_OK) {
        const std::string msg = ccfmm_last_error();
        fmm_adaptive_destroy(*out);
        *out = nullptr;
        set_last_error(msg.c_str());
    }
    return st;
}

ccfmm_status fmm_adaptive_tuning(ccfmm_adaptive_t h, int32_t *nclasses, int64_t *class_nmin,
                                 double *class_split, int32_t capacity)
{
    set_last_error("");
    if (!h || !nclasses) return afail(CCFMM_ERR_ARG, "NULL argument");
    *nclasses = (int32_t)h->tune_nmin.size();
    for (int i = 0; i < (int)h->tune_nmin.size() && i < capacity; ++i) {
        if (class_nmin) class_nmin[i] = h->tune_nmin[i];
        if (class_split) class_split[i] = h->tune_split[i];
    }
    return CCFMM_OK;
}

ccfmm_status fmm_adaptive_evaluate(ccfmm_adaptive_t h, double *H_out, double *E_out)
{
    set_last_error("");
    if (!h) return afail(CCFMM_ERR_ARG, "handle is NULL");
    ACK(cudaSetDevice(h->device));
    return run(h, 0, H_out, E_out);
}

ccfmm_status fmm_adaptive_step(ccfmm_adaptive_t h, uint64_t seed, uint64_t step,
                               double max_angle, double *H_out, double *E_out)
{
    set_last_error("");
    if (!h) return afail(CCFMM_ERR_ARG, "handle is NULL");
    if (!(max_angle >= 0.0) || isinf(max_angle)) return afail(CCFMM_ERR_ARG, "bad max_angle");
    ACK(cudaSetDevice(h->device));
    ACK(cudaStreamSynchronize(h->stream));
    h->hprm->seed = seed;
    h->hprm->step = step;
    h->hprm->max_angle = max_angle;
    ACK(cudaMemcpyAsync(h->prm.p, h->hprm, sizeof(RotateParams), cudaMemcpyHostToDevice, h->stream));
    return run(h, 1, H_out, E_out);
}

ccfmm_status fmm_adaptive_set_moments(ccfmm_adaptive_t h, const double *moments)
{
    set_last_error("");
    if (!h || !moments) return afail(CCFMM_ERR_ARG, "NULL argument");
    ACK(cudaSetDevice(h->device));
    ACK(cudaStreamSynchronize(h->stream));
    ACK(cudaMemcpyAsync(h->mom.p, moments, sizeof(double) * 3 * (size_t)h->N,
                        is_dev(moments) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                        h->stream));
    ACK(cudaStreamSynchronize(h->stream));
    return CCFMM_OK;
}

ccfmm_status fmm_adaptive_get_moments(ccfmm_adaptive_t h, double *out)
{
    set_last_error("");
    if (!h || !out) return afail(CCFMM_ERR_ARG, "NULL argument");
    ACK(cudaSetDevice(h->device));
    ACK(cudaMemcpyAsync(out, h->mom.p, sizeof(double) * 3 * (size_t)h->N,
                        is_dev(out) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, h->stream));
    ACK(cudaStreamSynchronize(h->stream));
    return CCFMM_OK;
}

ccfmm_status fmm_adaptive_info(ccfmm_adaptive_t h, ccfmm_adaptive_stats *out)
{
    set_last_error("");
    if (!h || !out) return afail(CCFMM_ERR_ARG, "NULL argument");
    memset(out, 0, sizeof(*out));
    out->n = h->N;
    out->nsamples = h->ns;
    out->p = h->p;
    out->theta = h->theta;
    out->ncells = h->nc;
    out->nleaves = h->nleaf;
    out->max_level = h->maxL;
    out->far_pairs = h->nfar;
    out->near_entries = h->nnear;
    out->near_pairs = (int64_t)h->near_pairs;
    out->d_rows = h->nd;
    out->m2l_items = (int64_t)h->n64 + h->n16;
    out->kernels_per_eval = h->kernels_per_eval;
    out->ms_build = h->ms_build;
    return CCFMM_OK;
}

ccfmm_status fmm_adaptive_cells(ccfmm_adaptive_t h, int64_t *out)
{
    set_last_error("");
    if (!h || !out) return afail(CCFMM_ERR_ARG, "NULL argument");
    ACK(cudaSetDevice(h->device));
    const size_t nc = (size_t)h->nc;
    std::vector<int> lev(nc), par(nc), ch(2 * nc), p0(nc), np(nc), smp(nc);
    ATRY(to_host(h, lev.data(), h->lev.p, nc));
    ATRY(to_host(h, par.data(), h->par.p, nc));
    ATRY(to_host(h, ch.data(), h->ch.p, 2 * nc));
    ATRY(to_host(h, p0.data(), h->p0.p, nc));
    ATRY(to_host(h, np.data(), h->np.p, nc));
    ATRY(to_host(h, smp.data(), h->smp.p, nc));
    for (size_t c = 0; c < nc; ++c) {
        int64_t *r = out + 8 * c;
        r[0] = lev[c];
        r[1] = par[c];
        r[2] = ch[2 * c];
        r[3] = ch[2 * c + 1];
        r[4] = p0[c];
        r[5] = np[c];
        r[6] = (ch[2 * c] < 0 && ch[2 * c + 1] < 0) ? 1 : 0;
        r[7] = smp[c];
    }
    return CCFMM_OK;
}

ccfmm_status fmm_adaptive_perm(ccfmm_adaptive_t h, int64_t *out)
{
    set_last_error("");
    if (!h || !out) return afail(CCFMM_ERR_ARG, "NULL argument");
    ACK(cudaSetDevice(h->device));
    std::vector<int> v((size_t)h->N);
    ATRY(to_host(h, v.data(), h->perm.p, (size_t)h->N));
    for (long long i = 0; i < h->N; ++i) out[i] = v[i];
    return CCFMM_OK;
}

ccfmm_status fmm_adaptive_pairs(ccfmm_adaptive_t h, int kind, int64_t *out, int64_t capacity,
                                int64_t *count)
{
    set_last_error("");
    if (!h || !count || (kind != 0 && kind != 1)) return afail(CCFMM_ERR_ARG, "bad argument");
    ACK(cudaSetDevice(h->device));
    const long long n = kind ? h->nfar : h->nnear;
    *count = n;
    if (!out) return CCFMM_OK;
    if (capacity < n) return afail(CCFMM_ERR_ARG, "capacity %lld < %lld pairs", (long long)capacity, n);
    if (kind) {
        std::vector<int> t((size_t)n), s((size_t)n);
        ATRY(to_host(h, t.data(), h->pt.p, (size_t)n));
        ATRY(to_host(h, s.data(), h->ps.p, (size_t)n));
        for (long long k = 0; k < n; ++k) {
            out[2 * k] = t[k];
            out[2 * k + 1] = s[k];
        }
        return CCFMM_OK;
    }
    const size_t nc = (size_t)h->nc;
    std::vector<int> nf(nc), nn(nc), src((size_t)n);
    ATRY(to_host(h, nf.data(), h->near_first.p, nc));
    ATRY(to_host(h, nn.data(), h->near_num.p, nc));
    ATRY(to_host(h, src.data(), h->near_src.p, (size_t)n));
    long long k = 0;
    for (size_t c = 0; c < nc; ++c)
        for (int e = nf[c]; e < nf[c] + nn[c]; ++e) {
            out[2 * k] = (int64_t)c;
            out[2 * k + 1] = src[e];
            ++k;
        }
    return CCFMM_OK;
}

ccfmm_status fmm_adaptive_expansions(ccfmm_adaptive_t h, double *Q_out, double *V_out)
{
    set_last_error("");
    if (!h) return afail(CCFMM_ERR_ARG, "handle is NULL");
    if (!h->evaluated) return afail(CCFMM_ERR_STATE, "no evaluation yet");
    ACK(cudaSetDevice(h->device));
    const size_t nc = (size_t)h->nc, KP = (size_t)h->KP, K = (size_t)h->K;
    if (Q_out) {
        std::vector<double> q(nc * KP);
        if (h->dbl) {
            ATRY(to_host(h, q.data(), h->Q.p, nc * KP));
        } else {
            std::vector<float> f(nc * KP);
            ATRY(to_host(h, f.data(), h->Q.p, nc * KP));
            for (size_t i = 0; i < f.size(); ++i) q[i] = f[i];
        }
        for (size_t c = 0; c < nc; ++c)
            for (size_t j = 0; j < K; ++j) Q_out[c * K + j] = q[c * KP + j];
    }
    if (V_out) {
        std::vector<double> v(nc * KP);
        ATRY(to_host(h, v.data(), h->V.p, nc * KP));
        for (size_t c = 0; c < nc; ++c)
            for (size_t j = 0; j < K; ++j) V_out[c * K + j] = v[c * KP + j];
    }
    return CCFMM_OK;
}

}  // extern "C"
