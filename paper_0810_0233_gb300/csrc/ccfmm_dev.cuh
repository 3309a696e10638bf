// ccfmm_dev.cuh -- internal declarations shared by the libccfmm translation
// units (kernels and the host orchestrator).  Not part of the C-ABI.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace ccfmm {

// Depth limit of the complete tree: leaf keys are LCAP-bit integers and the
// dense per-level arrays hold 2^l cells.
constexpr int LCAP = 24;
constexpr int PMAX = 8;
// Targets per M2L tile (same level, same parity along the last split).
constexpr int TT = 128;

// ---------------------------------------------------------------------------
// Multi-indices n = (nx, ny, nz).  The library orders them by total order k,
// then inside an order by nz ascending, then ny ascending (nx = k - ny - nz).
// Coefficient arrays Q and V store the multi-indices 1 .. T(p)-1 (Q_0 = 0
// for dipoles, V_0 never reaches the field) in columns 0 .. K-1, K = T(p)-1,
// padded with zeros to KP columns.
// ---------------------------------------------------------------------------
__host__ __device__ constexpr int nterms(int k) { return k < 0 ? 0 : (k + 1) * (k + 2) * (k + 3) / 6; }
__host__ __device__ inline int midx(int nx, int ny, int nz)
{
    int k = nx + ny + nz;
    return nterms(k - 1) + nz * (2 * k + 3 - nz) / 2 + ny;
}
__host__ __device__ inline void midx_inv(int t, int &nx, int &ny, int &nz)
{
    int k = 0;
    while (nterms(k) <= t) ++k;
    int r = t - nterms(k - 1);
    nz = 0;
    while (r >= k + 1 - nz) {
        r -= k + 1 - nz;
        ++nz;
    }
    ny = r;
    nx = k - ny - nz;
}
inline int padded_k(int p) { return ((nterms(p) - 1 + 7) / 8) * 8; }
// M2L truncation: the term (n, k) of Eq. taylorcalc is kept when
// |n|+|k| <= maxdeg (2p: every stored pair, the square truncation).  The
// coefficient columns are ordered by degree, so the columns k that can meet
// column n form a prefix; its length, 0 for padding columns n >= K.
__host__ __device__ inline int m2l_kend(int p, int maxdeg, int n)
{
    const int K = nterms(p) - 1;
    if (n >= K) return 0;
    int d = 1;
    while (nterms(d) <= n + 1) ++d;  // degree of multi-index n + 1
    const int r = maxdeg - d;
    if (r < 1) return 0;
    return r >= p ? K : nterms(r) - 1;
}

// Harmonic reduction of the M2L contraction (the D tensors satisfy Laplace's
// equation): per order k the 2k + 1 multi-indices with n_z <= 1, the first
// 2k + 1 of the order in the library's order; reduced column r of order k
// (k^2 - 1 <= r < (k+1)^2 - 1) is full column T(k-1) - 1 + r - (k^2 - 1).
__host__ __device__ constexpr int red_count(int p) { return (p + 1) * (p + 1) - 1; }
__host__ __device__ constexpr int red_padded(int p) { return ((red_count(p) + 7) / 8) * 8; }
__host__ __device__ inline int red_order(int r)
{
    int k = 1;
    while ((k + 1) * (k + 1) - 1 <= r) ++k;
    return k;
}
__host__ __device__ inline int red_full(int r)
{
    const int k = red_order(r);
    return nterms(k - 1) - 1 + r - (k * k - 1);
}

template <typename T> struct vec4;
template <> struct vec4<float> { typedef float4 t; };
template <> struct vec4<double> { typedef double4 t; };
template <typename T> struct vec2;
template <> struct vec2<float> { typedef float2 t; };
template <> struct vec2<double> { typedef double2 t; };

// Tree geometry, in device memory.  Level l cells have widths w[l]; h[l] is
// the cell "radius" (half the diagonal, Sec. II), the scale of the M2L
// operands at that level.
struct Geom {
    double lo[3], ext[3];
    int axis[LCAP + 1];          // axis[l]: axis halved to make level l (l >= 1)
    int nsplit[LCAP + 1][3];     // splits of each axis in the first l levels
    double w[LCAP + 1][3];
    double h[LCAP + 1];
    int L;                       // chosen depth (set once known)
};

// Flag bits written by kernels into the handle's device status word.
enum : int {
    FLAG_NONFINITE = 1,
    FLAG_OUTSIDE_BOX = 2,
    FLAG_OFFSET_RANGE = 4,
    FLAG_LIST_OVERFLOW = 8,
    FLAG_TILE_OVERFLOW = 16,
    FLAG_TIMEOUT = 32
};

// Per-level table classifying an integer cell offset o = (coords of field
// cell) - (coords of partner), for offsets inside the cube |o_a| <= R[a]:
// value >= 0 : a far offset, its global D-table id;
// NEAR (-2)  : a near offset (self included);
// NONE (-1)  : not reachable from a near parent pair.
struct OffsetCube {
    int R[3];
    long long base;   // start of this level's table in the concatenated array
};
constexpr int OFF_NEAR = -2;
constexpr int OFF_NONE = -1;

struct NearEnt {   // leaf-level / per-level near entry
    int src;       // partner key at the same level
    int ox, oy, oz;
};
struct FarEnt {    // far entry of one cell
    int src;       // partner key
    int gid;       // global far-offset id (D table row)
};
struct Tile {      // M2L work unit
    int level;
    int first;     // targets are keys 2*(first+i) + parity, 0 <= i < nt
    int parity;
    int nt;
    int ent_start; // entries [ent_start, ent_start + ent_count)
    int ent_count;
    int nbits;     // far offsets of this level (bitmap width)
    int gid_base;  // first global offset id of this level
    const int *keys;  // device: target i is the level's cell keys[i] (the
                      // non-empty cells of one parity, in key order)
};

// Batched launches (ensemble step): one launch covers a stage of every
// member; bstart[m] .. bstart[m+1] are member m's blocks.  Returns m and
// sets local to the block's index within its member.
__device__ __forceinline__ int batch_member(const int *bstart, int nm, int blk, int &local)
{
    int lo = 0, hi = nm;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (__ldg(bstart + mid) <= blk) lo = mid; else hi = mid;
    }
    local = blk - __ldg(bstart + lo);
    return lo;
}

// Count of kernel launches issued by the library in this process.
void note_launch(int n = 1);
// Message returned by ccfmm_last_error() on this thread.
void set_last_error(const char *msg);

// Parameters of the ensemble rotation step, read by the kernel from device
// memory so that a captured graph serves every step.
struct RotateParams {
    unsigned long long seed, step;
    double max_angle;
};
void launch_rotate(double *mom, long long n, const RotateParams *prm, cudaStream_t s);

// ------------------------------------------------------------------ prims.cu
size_t scan_temp_bytes(long long n);
// exclusive scan of n int32 values; total (if not null) written to device
void scan_exclusive(const int *in, int *out, long long n, int *d_total, void *temp,
                    cudaStream_t s);
// two exclusive scans of the same length in one launch set; scratch: twice
// what scan_exclusive needs for n
void scan_exclusive2(const int *in0, int *out0, int *total0, const int *in1, int *out1,
                     int *total1, long long n, void *temp, cudaStream_t s);
size_t radix_temp_bytes(long long n);
// stable sort of (key, value) by the low `bits` bits of key; results in
// (k_out, v_out)
void radix_sort(const uint32_t *k_in, const int *v_in, uint32_t *k_out, int *v_out,
                uint32_t *k_tmp, int *v_tmp, long long n, int bits, void *temp, cudaStream_t s);

// ------------------------------------------------------------------ tree.cu
void launch_bbox(const double *pos, long long n, const double *user_box, double *d_geom_box,
                 double *partial, int *d_flags, cudaStream_t s);
void launch_geom(const double *d_box6, Geom *d_geom, cudaStream_t s);
void launch_keys(const double *pos, long long n, const Geom *d_geom, uint32_t *keys, int *idx,
                 int *d_flags, int check_box, cudaStream_t s);
void launch_depth_hist(const uint32_t *keys_sorted, long long n, int *d_hist, cudaStream_t s);
void launch_leaf_start(const uint32_t *keys_sorted, long long n, int L, int *leaf_start,
                       cudaStream_t s);
template <typename real>
void launch_sort_points(const double *pos, const double *mom, const int *perm,
                        const uint32_t *keys_sorted, long long n, const Geom *d_geom, int L,
                        typename vec4<real>::t *A, typename vec2<real>::t *B, cudaStream_t s);
template <typename real>
void launch_permute_moments(const double *mom, const int *perm, long long n,
                            typename vec4<real>::t *A, typename vec2<real>::t *B,
                            cudaStream_t s);
// non-empty cells per level (d_ne); with flags != nullptr also flags[hid] =
// 1 for every non-empty cell, 0 otherwise (flags[0] = 0)
void launch_level_counts(const int *leaf_start, int L, int *d_ne, int *flags, int *oflags,
                         int *d_ne_odd, cudaStream_t s);
// the M2L tiles' target cells: for every level l >= 2 the non-empty cells of
// each parity in key order, segment (l, parity) at seg[2 l + parity]
void launch_tile_keys(int L, const int *flags, const int *rank, const int *rank_odd,
                      const int *seg, int *tkeys, cudaStream_t s);
void launch_check_finite(const double *x, long long n, int *d_flags, cudaStream_t s);

// ------------------------------------------------------------------ lists.cu
// one level of the interaction lists in fixed slots (see lists.cu): rank =
// exclusive prefix of the non-empty flags over all heap ids; nl[hid] = (first
// near entry, count); near_total / far_total receive the level's totals
void launch_list_level(int level, const int *leaf_start, int L, const int *rank, int2 *nl,
                       const NearEnt *near_prev, const int *cube, OffsetCube cube_info, int axis,
                       int NB, NearEnt *near_out, long long far_base, int FB, FarEnt *far_out,
                       int *far_off, int *far_num, int *near_total, int *far_total, int *d_flags,
                       cudaStream_t s);
// per tile: the number of distinct far offsets; its offset bitmap and the
// prefix of the bitmap words' popcounts are stored (nwmax = (max_bits + 31)
// / 32 words a tile) for the fill
void launch_tile_count(const Tile *tiles, int ntiles, const int *far_off, const int *far_num,
                       const FarEnt *far, int max_bits, unsigned *gbm, unsigned *gwp, int *counts,
                       cudaStream_t s);
// entries get the D table of their offset class (dmap[class]); ent_src must
// hold -1 in every slot beforehand
void launch_tile_fill(Tile *tiles, int ntiles, const int *ent_start, const int *far_off,
                      const int *far_num, const FarEnt *far, int max_bits, const unsigned *gbm,
                      const unsigned *gwp, const int *dmap, int *ent_u, int *ent_src,
                      cudaStream_t s);

// ------------------------------------------------------------------ expand.cu
size_t ftable_scratch_bytes(int order);
void launch_ftable(int order, double *dense_scratch, int *f_start, uint16_t *f_q, double *f_val,
                   cudaStream_t s);
template <typename real>
// one D table per scaled separation sep[i] = (c_x, c_y, c_z) / h
void launch_dtables(int p, const int *f_start, const uint16_t *f_q, const double *f_val,
                    const double4 *sep, int nd, real *D, int ldD, cudaStream_t s);
void launch_itable(int p, int KP, int maxdeg, uint16_t *it, cudaStream_t s);
template <typename real>
void launch_p2m(int p, int KP, int L, const int *leaf_start, const typename vec4<real>::t *A,
                const typename vec2<real>::t *B, real *Q, cudaStream_t s);
// M2M over all levels (L-1 .. 0) and L2L over all levels (2 .. L), three
// levels per launch
template <typename real>
void launch_m2m_all(int p, int KP, int L, const Geom *d_geom, real *Q, cudaStream_t s);
void launch_l2l_all(int p, int KP, int L, const Geom *d_geom, const int *leaf_start, double *V,
                    cudaStream_t s);

// ------------------------------------------------------------------ m2l.cu
// FP32 M2L work item: a run of at most M2L_EC consecutive entries of a tile
constexpr int M2L_EC = 64;
struct M2LItem {
    int tile;
    int e0, e1;
};
bool m2l_f32_supported(int KP, int ldD);
void launch_m2l_f32(int p, int KP, const Tile *tiles, int ntiles, const M2LItem *items,
                    int nitems, const int *tile_item0, const int *tile_nitems, const int *ent_u,
                    const int *ent_src, const float *Q, const float *D, int ldD,
                    const uint16_t *it, int maxdeg, const Geom *g, float *Ps, double *V,
                    cudaStream_t s);
void launch_m2l_reduce(int p, int KP, const Tile *tiles, int ntiles, const int *tile_item0,
                       const int *tile_nitems, const float *Ps, const Geom *g, double *V,
                       cudaStream_t s);
// tensor-core (tcgen05, 3xTF32) M2L for KP in {40, 56, 88, 120}
constexpr bool M2L_TC_DEFAULT = true;
bool m2l_tc_supported(int KP);
size_t m2l_tc_op_bytes(int KP);  // operator bytes per far offset class
int m2l_tc_kt(int KP);           // padded K (row length of the split moments)
void launch_m2l_tc_ops(int p, int KP, int L, int n_off, const Geom *g, const float *D, int ldD,
                       const uint16_t *it, float *gk, float *Bop, cudaStream_t s);
// tensor map of the split moments for the TMA gather (map: 128 bytes,
// 64-byte aligned); false when the driver cannot encode it
bool m2l_tc_qmap(void *map, const float *Qs, long long ncell, int KP);
void launch_m2l_tc(int p, int KP, const Tile *tiles, int ntiles, const M2LItem *items, int nitems,
                   const int *tile_item0, const int *tile_nitems, const int *ent_u,
                   const int *ent_src, const float *Q, long long ncell, const float *gk,
                   float *Qs, const void *qmap, bool a_tmem, const float *Bop, const Geom *g,
                   float *Ps, double *V, int *flags, cudaStream_t s);
template <typename real>
void launch_m2l(int p, int KP, const Tile *tiles, int ntiles, const int *ent_u,
                const int *ent_src, const real *Q, const real *D, int ldD, const uint16_t *it,
                int maxdeg, const Geom *d_geom, double *V, cudaStream_t s);

// ------------------------------------------------------------------ p2p.cu
template <typename real>
void launch_p2p(int p, int KP, int L, const int *leaf_start, const int2 *near_nl,
                const NearEnt *near, const Geom *d_geom, const typename vec4<real>::t *A,
                const typename vec2<real>::t *B, const double *V, typename vec4<real>::t *H,
                cudaStream_t s);
// symmetric near field (CCFMM_P2P=sym): zeroes H, adds the near field with
// global reductions; the smooth field is added by launch_l2p
bool p2p_symmetric();
void launch_p2p_sym(int L, const int *leaf_start, const int2 *near_nl, const NearEnt *near,
                    const Geom *d_geom, const float4 *A, const float2 *B, float4 *H,
                    long long N, cudaStream_t s);
// V == nullptr: near field only; launch_l2p then adds the smooth field
template <typename real>
void launch_l2p(int p, int KP, int L, const int *leaf_start, const typename vec4<real>::t *A,
                const double *V, typename vec4<real>::t *H, cudaStream_t s);
template <typename real>
void launch_finish(const typename vec4<real>::t *H, const int *perm, const double *mom,
                   long long n, double *H_out, double *partial, double *d_E, cudaStream_t s);
void launch_direct(const double *pos, const double *mom, long long n, const long long *tgt,
                   long long nt, double *H_out, cudaStream_t s);
void launch_p2p_pair_count(int L, const int *leaf_start, const int2 *near_nl,
                           const NearEnt *near, unsigned long long *d_count, cudaStream_t s);

// ------------------------------------------------ batched ensemble stages
// One launch per stage covers every member of an ensemble (FP32 path,
// tensor-core M2L): the arguments of each member's launch in device
// memory, and bstart (nm + 1 block offsets) mapping blocks to members.
struct PermuteArgs {
    const double *mom;
    const int *perm;
    long long n;
    float4 *A;
    float2 *B;
    double *V;        // zeroed by the same launch
    long long nV;     // doubles of V
};
struct P2MArgs {
    int p, KP, L;
    const int *leaf_start;
    const float4 *A;
    const float2 *B;
    float *Q;
};
struct M2MArgs {   // one round: levels l0 + D - 1 .. l0 from l0 + D
    int p, KP, l0, D;
    const Geom *g;
    float *Q;
};
struct QSplitArgs {
    int p;
    long long ncell;
    const float *Q, *gk;
    float *Qs;
};
struct M2LTCArgs {
    const M2LItem *items;
    const int *ent_u, *ent_src;
    const float *Qs;
    long long qplane;
    const unsigned char *Bop;
    float *Ps;
    int *flags;
};
struct ReduceArgs {
    int p, KP;
    const Tile *tiles;
    const int *tile_item0, *tile_nitems;
    const float *Ps;
    const Geom *g;
    double *V;
};
struct L2LArgs {   // one round: levels l0 + 1 .. l0 + D from l0
    int p, KP, l0, D, L;
    const Geom *g;
    const int *leaf_start;
    double *V;
};
struct P2PArgs {   // near field with the fused smooth field
    int p, KP, L;
    const int *leaf_start;
    const int2 *near_nl;
    const NearEnt *near;
    const Geom *g;
    const float4 *A;
    const float2 *B;
    const double *V;
    float4 *H;
};
struct FinishArgs {
    const float4 *H;
    const int *perm;
    const double *mom;
    long long n;
    double *Hout, *partial, *E;
};
int permute_blocks(long long n);
int p2m_blocks(int L);
int q_split_blocks(int KP, long long ncell);
int finish_blocks(long long n);
void launch_permute_batch(const PermuteArgs *a, const int *bstart, int nm, int nblocks,
                          cudaStream_t s);
void launch_p2m_batch(const P2MArgs *a, const int *bstart, int nm, int nblocks, cudaStream_t s);
void launch_m2m_batch(const M2MArgs *a, const int *bstart, int nm, int nblocks, cudaStream_t s);
void launch_l2l_batch(const L2LArgs *a, const int *bstart, int nm, int nblocks, cudaStream_t s);
void launch_q_split_batch(int KP, const QSplitArgs *a, const int *bstart, int nm, int nblocks,
                          cudaStream_t s);
void launch_m2l_tc_batch(int KP, const M2LTCArgs *a, const int *bstart, int nm, int nblocks,
                         long long spin, int stall, cudaStream_t s);
void launch_reduce_batch(int p, const ReduceArgs *a, const int *bstart, int nm, int nblocks,
                         cudaStream_t s);
// the tensor-core path's reduce (harmonic reduction: reduced partial sums,
// then the full V); KPF the full coefficient width
void launch_reduce_h_batch(int p, int KPF, const ReduceArgs *a, const int *bstart, int nm,
                           int nblocks, cudaStream_t s);
void launch_p2p_batch(const P2PArgs *a, const int *bstart, int nm, int nblocks, int KP,
                      cudaStream_t s);
void launch_finish_batch(const FinishArgs *a, const int *bstart, int nm, int nblocks,
                         cudaStream_t s);
// smooth field added to the near field (P2PArgs with V set), every member
int l2p_blocks(int L);
void launch_l2p_batch(int p, const P2PArgs *a, const int *bstart, int nm, int nblocks,
                      cudaStream_t s);
// ------------------------------------------------ adaptive-depth tree
// P2M of every leaf cell (any level) about its centre
template <typename real>
void launch_ap2m(int p, int KP, int nleaf, const int *leaves, const int *p0, const int *np,
                 const typename vec4<real>::t *A, const typename vec2<real>::t *B, real *Q,
                 cudaStream_t s);
// M2L grouped by D row: items (first pair, count, D row) over the sorted
// pair arrays pt/ps; accumulates into VF with atomics.  ap = 64: groups of
// more than 16 pairs, 16: the others.  rpow: per D row rho^-d, d = 0 .. p+1
// (PMAX + 2 floats a row; FP32 tensor-core form), or null.
template <typename real>
void launch_am2l(int p, int KP, const int4 *items, int nitems, int ap, const int *pt,
                 const int *ps, const double4 *sep, const float *rpow, const real *D, int ldD,
                 const uint16_t *it, int maxdeg, const real *Q, real *VF, cudaStream_t s);
// adaptive M2L over the harmonic reduction (FP32, p <= 6, tensor cores):
// moments folded into reduced rows (KRP = red_padded(p) floats), the reduced
// index table from the full one, and the contraction into a reduced
// accumulator VFr[cell][KRP]
bool am2l_mma_ok(int p);
void launch_afold(int p, int KPF, int KRP, int nc, const float *Q, float *Qr, cudaStream_t s);
void launch_itable_red(int p, int KPF, int KRP, const uint16_t *it, uint16_t *itr,
                       cudaStream_t s);
void launch_am2l_red(int p, int KRP, const int4 *items, int nitems, int ap, const int *pt,
                     const int *ps, const float *rpow, const float *D, int ldD,
                     const uint16_t *itr, const float *Qr, float *VFr, cudaStream_t s);
// smooth field of every leaf cell added to H (after launch_ap2p with V null)
template <typename real>
void launch_al2p(int p, int KP, int nleaf, const int *leaves, const int *p0, const int *np,
                 const typename vec4<real>::t *A, const double *V, typename vec4<real>::t *H,
                 cudaStream_t s);
// near field of every leaf cell, with the smooth field fused when V is not null
template <typename real>
void launch_ap2p(int p, int KP, int nleaf, const int *leaves, const int *p0, const int *np,
                 const int *near_first, const int *near_num, const int *near_src,
                 const double4 *cen, const typename vec4<real>::t *A,
                 const typename vec2<real>::t *B, const double *V, typename vec4<real>::t *H,
                 cudaStream_t s);

// the M2M and L2L rounds of a tree of depth L: (l0, D) per round
int m2m_rounds(int L, int *l0, int *D);
int l2l_rounds(int L, int *l0, int *D);

}  // namespace ccfmm
