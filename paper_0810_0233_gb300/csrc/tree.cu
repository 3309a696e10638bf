// tree.cu -- recursive-bisection tree on the GPU (Sec. II; Sec. IV rule of
// thumb): bounding box and split sequence, LCAP-bit bisection keys, the
// non-empty-leaf histogram that selects the depth, leaf ranges, and the
// sorted dipole arrays (coordinates relative to the leaf centre).
#include "ccfmm_dev.cuh"
#include "stages.cuh"

#include <math.h>

namespace ccfmm {

constexpr int BB_T = 256, BB_BLOCKS = 1024;

__global__ void __launch_bounds__(BB_T) k_bbox_partial(const double *pos, long long n,
                                                       double *partial, int *flags)
{
    double mn[3] = {INFINITY, INFINITY, INFINITY}, mx[3] = {-INFINITY, -INFINITY, -INFINITY};
    int bad = 0;
    for (long long i = (long long)blockIdx.x * BB_T + threadIdx.x; i < n;
         i += (long long)gridDim.x * BB_T) {
        for (int a = 0; a < 3; ++a) {
            double x = pos[3 * i + a];
            if (!isfinite(x)) bad = 1;
            mn[a] = fmin(mn[a], x);
            mx[a] = fmax(mx[a], x);
        }
    }
    __shared__ double sm[6][BB_T / 32];
    int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int a = 0; a < 3; ++a) {
        for (int o = 16; o; o >>= 1) {
            mn[a] = fmin(mn[a], __shfl_xor_sync(0xffffffffu, mn[a], o));
            mx[a] = fmax(mx[a], __shfl_xor_sync(0xffffffffu, mx[a], o));
        }
        if (lane == 0) {
            sm[a][warp] = mn[a];
            sm[3 + a][warp] = mx[a];
        }
    }
    bad = __any_sync(0xffffffffu, bad);
    if (bad && lane == 0) atomicOr(flags, FLAG_NONFINITE);
    __syncthreads();
    if (threadIdx.x < 6) {
        double v = sm[threadIdx.x][0];
        for (int w = 1; w < BB_T / 32; ++w)
            v = threadIdx.x < 3 ? fmin(v, sm[threadIdx.x][w]) : fmax(v, sm[threadIdx.x][w]);
        partial[6 * blockIdx.x + threadIdx.x] = v;
    }
}

__global__ void __launch_bounds__(256) k_bbox_final(const double *partial, int nparts,
                                                    const double *user_box, double *box6, int *flags)
{
    __shared__ double sm[6][256];
    double v[6] = {INFINITY, INFINITY, INFINITY, -INFINITY, -INFINITY, -INFINITY};
    for (int b = threadIdx.x; b < nparts; b += 256)
        for (int a = 0; a < 3; ++a) {
            v[a] = fmin(v[a], partial[6 * b + a]);
            v[3 + a] = fmax(v[3 + a], partial[6 * b + 3 + a]);
        }
    for (int a = 0; a < 6; ++a) sm[a][threadIdx.x] = v[a];
    __syncthreads();
    for (int w = 128; w; w >>= 1) {
        if (threadIdx.x < w)
            for (int a = 0; a < 6; ++a)
                sm[a][threadIdx.x] = a < 3 ? fmin(sm[a][threadIdx.x], sm[a][threadIdx.x + w])
                                           : fmax(sm[a][threadIdx.x], sm[a][threadIdx.x + w]);
        __syncthreads();
    }
    if (threadIdx.x != 0) return;
    double mn[3], mx[3];
    for (int a = 0; a < 3; ++a) {
        mn[a] = sm[a][0];
        mx[a] = sm[3 + a][0];
    }
    if (user_box) {
        for (int a = 0; a < 3; ++a) {
            if (mn[a] < user_box[a] || mx[a] > user_box[3 + a]) atomicOr(flags, FLAG_OUTSIDE_BOX);
            box6[a] = user_box[a];
            box6[3 + a] = user_box[3 + a];
        }
    } else {
        // bounding box widened by 2^-20 of its largest extent on every side
        double m = 0.0;
        for (int a = 0; a < 3; ++a)
            if (mx[a] - mn[a] > m) m = mx[a] - mn[a];
        if (m == 0.0) m = 1.0;
        double pad = m * 9.5367431640625e-07;  // 2^-20
        for (int a = 0; a < 3; ++a) {
            box6[a] = mn[a] - pad;
            box6[3 + a] = mx[a] + pad;
        }
    }
}

// split sequence: at every level halve the currently widest axis, ties x<y<z
// Box, split sequence and cell sizes of every level.  One thread; the
// running widths and split counts stay in registers (the stores to g are
// never read back here, so no step waits on a global-memory round trip).
// The split sequence (one thread: halve the widest axis, ties x < y < z),
// then the widths and radii of every level (one thread per level).
__global__ void k_geom(const double *box6, Geom *g)
{
    __shared__ int s_ns[LCAP + 1][3];
    const int t = threadIdx.x;
    double ext[3];
    for (int a = 0; a < 3; ++a) ext[a] = box6[3 + a] - box6[a];
    if (t == 0) {
        int ns[3] = {0, 0, 0};
        double w[3] = {ext[0], ext[1], ext[2]};
        for (int a = 0; a < 3; ++a) {
            g->lo[a] = box6[a];
            g->ext[a] = ext[a];
            s_ns[0][a] = 0;
        }
        g->axis[0] = -1;
        for (int l = 1; l <= LCAP; ++l) {
            int a = 0;
            if (w[1] > w[a]) a = 1;
            if (w[2] > w[a]) a = 2;
            g->axis[l] = a;
            ns[a] += 1;
            w[a] = ldexp(ext[a], -ns[a]);
            for (int b = 0; b < 3; ++b) s_ns[l][b] = ns[b];
        }
        g->L = -1;
    }
    __syncthreads();
    for (int l = t; l <= LCAP; l += blockDim.x) {
        double w[3];
        for (int b = 0; b < 3; ++b) {
            w[b] = ldexp(ext[b], -s_ns[l][b]);
            g->nsplit[l][b] = s_ns[l][b];
            g->w[l][b] = w[b];
        }
        g->h[l] = 0.5 * sqrt(w[0] * w[0] + w[1] * w[1] + w[2] * w[2]);
    }
}

void launch_bbox(const double *pos, long long n, const double *user_box, double *d_box6,
                 double *partial, int *d_flags, cudaStream_t s)
{
    int nb = (int)((n + BB_T - 1) / BB_T);
    if (nb > BB_BLOCKS) nb = BB_BLOCKS;
    if (nb < 1) nb = 1;
    note_launch();
    k_bbox_partial<<<nb, BB_T, 0, s>>>(pos, n, partial, d_flags);
    note_launch();
    k_bbox_final<<<1, 256, 0, s>>>(partial, nb, user_box, d_box6, d_flags);
}

void launch_geom(const double *d_box6, Geom *d_geom, cudaStream_t s)
{
    note_launch();
    k_geom<<<1, 32, 0, s>>>(d_box6, d_geom);
}

// LCAP-bit key of each point: leaf coordinate per axis at depth LCAP,
// c_a = min(floor((x_a - lo_a) * n_a / ext_a), n_a - 1), with the bits of the
// axes interleaved in split order (level 1 = most significant bit).
__global__ void k_keys(const double *pos, long long n, const Geom *g, uint32_t *keys, int *idx,
                       int *flags, int check_box)
{
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    long long c[3];
    int nb[3];
    for (int a = 0; a < 3; ++a) {
        nb[a] = g->nsplit[LCAP][a];
        long long na = 1ll << nb[a];
        double t = (pos[3 * i + a] - g->lo[a]) * (double)na / g->ext[a];
        long long ca = (long long)floor(t);
        if (check_box && (t < 0.0 || t > (double)na)) atomicOr(flags, FLAG_OUTSIDE_BOX);
        if (ca > na - 1) ca = na - 1;
        if (ca < 0) ca = 0;
        c[a] = ca;
    }
    // level j takes the next bit (from the top) of the coordinate along the
    // axis split at j: bit nsplit[LCAP][a] - nsplit[j][a] of c[a]
    uint32_t key = 0;
#pragma unroll
    for (int j = 1; j <= LCAP; ++j) {
        const int a = g->axis[j];
        const long long ca = a == 0 ? c[0] : (a == 1 ? c[1] : c[2]);
        const int sh = (a == 0 ? nb[0] : (a == 1 ? nb[1] : nb[2])) - g->nsplit[j][a];
        key = (key << 1) | (uint32_t)((ca >> sh) & 1);
    }
    keys[i] = key;
    idx[i] = (int)i;
}

void launch_keys(const double *pos, long long n, const Geom *d_geom, uint32_t *keys, int *idx,
                 int *d_flags, int check_box, cudaStream_t s)
{
    if (n <= 0) return;
    note_launch();
    k_keys<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(pos, n, d_geom, keys, idx, d_flags,
                                                       check_box);
}

// hist[L] = number of adjacent sorted keys whose depth-L prefixes first differ
// at level L; nonempty leaves at depth L = 1 + sum_{L' <= L} hist[L'].
__global__ void k_depth_hist(const uint32_t *keys, long long n, int *hist)
{
    __shared__ int h[LCAP + 1];
    if (threadIdx.x <= LCAP) h[threadIdx.x] = 0;
    __syncthreads();
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x + 1; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        uint32_t x = keys[i] ^ keys[i - 1];
        if (x) {
            int hb = 31 - __clz(x);
            atomicAdd(&h[LCAP - hb], 1);
        }
    }
    __syncthreads();
    if (threadIdx.x <= LCAP && h[threadIdx.x]) atomicAdd(&hist[threadIdx.x], h[threadIdx.x]);
}

void launch_depth_hist(const uint32_t *keys_sorted, long long n, int *d_hist, cudaStream_t s)
{
    cudaMemsetAsync(d_hist, 0, sizeof(int) * (LCAP + 1), s);
    long long nb = (n + 255) / 256;
    if (nb > 4096) nb = 4096;
    if (nb < 1) nb = 1;
    note_launch();
    k_depth_hist<<<(unsigned)nb, 256, 0, s>>>(keys_sorted, n, d_hist);
}

// leaf_start[k] = first sorted index with leaf key >= k, k = 0 .. 2^L
__global__ void k_leaf_start(const uint32_t *keys, long long n, int L, int *leaf_start)
{
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i > n) return;
    int sh = LCAP - L;
    long long prev = (i == 0) ? -1 : (long long)(keys[i - 1] >> sh);
    long long cur = (i == n) ? (1ll << L) : (long long)(keys[i] >> sh);
    for (long long k = prev + 1; k <= cur; ++k) leaf_start[k] = (int)i;
}

void launch_leaf_start(const uint32_t *keys_sorted, long long n, int L, int *leaf_start,
                       cudaStream_t s)
{
    note_launch();
    k_leaf_start<<<(unsigned)((n + 1 + 255) / 256), 256, 0, s>>>(keys_sorted, n, L, leaf_start);
}

__device__ __forceinline__ void leaf_coords(const Geom *g, int L, uint32_t k, int ic[3])
{
    ic[0] = ic[1] = ic[2] = 0;
    for (int j = 1; j <= L; ++j) {
        int bit = (int)((k >> (L - j)) & 1u);
        int a = g->axis[j];
        ic[a] = 2 * ic[a] + bit;
    }
}

template <typename real>
__global__ void k_sort_points(const double *pos, const double *mom, const int *perm,
                              const uint32_t *keys, long long n, const Geom *g, int L,
                              typename vec4<real>::t *A, typename vec2<real>::t *B)
{
    long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    int i = perm[s];
    uint32_t k = keys[s] >> (LCAP - L);
    int ic[3];
    leaf_coords(g, L, k, ic);
    double l[3];
    for (int a = 0; a < 3; ++a) {
        double c = g->lo[a] + ((double)ic[a] + 0.5) * g->w[L][a];
        l[a] = pos[3 * (long long)i + a] - c;
    }
    typename vec4<real>::t av;
    av.x = (real)l[0];
    av.y = (real)l[1];
    av.z = (real)l[2];
    av.w = (real)mom[3 * (long long)i];
    typename vec2<real>::t bv;
    bv.x = (real)mom[3 * (long long)i + 1];
    bv.y = (real)mom[3 * (long long)i + 2];
    A[s] = av;
    B[s] = bv;
}

template <typename real>
void launch_sort_points(const double *pos, const double *mom, const int *perm,
                        const uint32_t *keys_sorted, long long n, const Geom *d_geom, int L,
                        typename vec4<real>::t *A, typename vec2<real>::t *B, cudaStream_t s)
{
    if (n <= 0) return;
    note_launch();
    k_sort_points<real><<<(unsigned)((n + 255) / 256), 256, 0, s>>>(pos, mom, perm, keys_sorted,
                                                                    n, d_geom, L, A, B);
}

template <typename real>
__global__ void k_permute_moments(const double *mom, const int *perm, long long n,
                                  typename vec4<real>::t *A, typename vec2<real>::t *B)
{
    const long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (s < n) permute_one<real>(s, mom, perm, A, B);
}

template <typename real>
void launch_permute_moments(const double *mom, const int *perm, long long n,
                            typename vec4<real>::t *A, typename vec2<real>::t *B, cudaStream_t s)
{
    if (n <= 0) return;
    note_launch();
    k_permute_moments<real><<<(unsigned)((n + 255) / 256), 256, 0, s>>>(mom, perm, n, A, B);
}

// every member's moments into its sorted arrays, and its Taylor
// coefficients zeroed, in one launch (ensemble step)
__global__ void k_permute_batch(const PermuteArgs *a, const int *bstart, int nm)
{
    int blk;
    const int m = batch_member(bstart, nm, blockIdx.x, blk);
    const PermuteArgs &x = a[m];
    const long long s = (long long)blk * 256 + threadIdx.x;
    if (s < x.n) {
        const long long i = x.perm[s];
        x.A[s].w = (float)x.mom[3 * i];
        x.B[s] = make_float2((float)x.mom[3 * i + 1], (float)x.mom[3 * i + 2]);
    }
    const long long nth = (long long)(bstart[m + 1] - bstart[m]) * 256;
    for (long long j = s; j < x.nV; j += nth) x.V[j] = 0.0;
}

int permute_blocks(long long n) { return (int)((n + 255) / 256); }

void launch_permute_batch(const PermuteArgs *a, const int *bstart, int nm, int nblocks,
                          cudaStream_t s)
{
    if (nblocks <= 0) return;
    note_launch();
    k_permute_batch<<<(unsigned)nblocks, 256, 0, s>>>(a, bstart, nm);
}

// non-empty cells per level (levels 0..L), from the leaf ranges
__global__ void k_level_counts(const int *leaf_start, int L, int *ne, int *flags, int *oflags,
                               int *ne_odd)
{
    __shared__ int h[LCAP + 1], ho[LCAP + 1];
    if (threadIdx.x <= LCAP) h[threadIdx.x] = ho[threadIdx.x] = 0;
    __syncthreads();
    long long ncell = (1ll << (L + 1)) - 1;
    for (long long id = (long long)blockIdx.x * blockDim.x + threadIdx.x; id < ncell;
         id += (long long)gridDim.x * blockDim.x) {
        long long hid = id + 1;
        int l = 63 - __clzll(hid);
        long long key = hid - (1ll << l);
        int sh = L - l;
        const bool full = leaf_start[(key + 1) << sh] > leaf_start[key << sh];
        const bool odd = full && (key & 1);
        if (full) atomicAdd(&h[l], 1);
        if (odd) atomicAdd(&ho[l], 1);
        if (flags) flags[hid] = full ? 1 : 0;
        if (oflags) oflags[hid] = odd ? 1 : 0;
    }
    if (flags && blockIdx.x == 0 && threadIdx.x == 0) flags[0] = 0;
    if (oflags && blockIdx.x == 0 && threadIdx.x == 0) oflags[0] = 0;
    __syncthreads();
    if (threadIdx.x <= LCAP && h[threadIdx.x]) atomicAdd(&ne[threadIdx.x], h[threadIdx.x]);
    if (ne_odd && threadIdx.x <= LCAP && ho[threadIdx.x])
        atomicAdd(&ne_odd[threadIdx.x], ho[threadIdx.x]);
}

void launch_level_counts(const int *leaf_start, int L, int *d_ne, int *flags, int *oflags,
                         int *d_ne_odd, cudaStream_t s)
{
    cudaMemsetAsync(d_ne, 0, sizeof(int) * (LCAP + 1), s);
    if (d_ne_odd) cudaMemsetAsync(d_ne_odd, 0, sizeof(int) * (LCAP + 1), s);
    long long ncell = (1ll << (L + 1)) - 1;
    long long nb = (ncell + 255) / 256;
    if (nb > 4096) nb = 4096;
    note_launch();
    k_level_counts<<<(unsigned)nb, 256, 0, s>>>(leaf_start, L, d_ne, flags, oflags, d_ne_odd);
}

// target cells of the M2L tiles: the non-empty cells of each level l >= 2
// and parity, in key order, at seg[2 l + parity]
__global__ void k_tile_keys(int L, const int *flags, const int *rank, const int *rank_odd,
                            const int *seg, int *tkeys)
{
    const long long ncell = 1ll << (L + 1);
    for (long long hid = 4 + (long long)blockIdx.x * blockDim.x + threadIdx.x; hid < ncell;
         hid += (long long)gridDim.x * blockDim.x) {
        if (!flags[hid]) continue;
        const int l = 63 - __clzll(hid);
        const long long l0 = 1ll << l;
        const int key = (int)(hid - l0);
        const int rl = rank[hid] - rank[l0], ro = rank_odd[hid] - rank_odd[l0];
        const int par = key & 1;
        tkeys[seg[2 * l + par] + (par ? ro : rl - ro)] = key;
    }
}

void launch_tile_keys(int L, const int *flags, const int *rank, const int *rank_odd,
                      const int *seg, int *tkeys, cudaStream_t s)
{
    if (L < 2) return;
    const long long n = (1ll << (L + 1)) - 4;
    long long nb = (n + 255) / 256;
    if (nb > 4096) nb = 4096;
    note_launch();
    k_tile_keys<<<(unsigned)nb, 256, 0, s>>>(L, flags, rank, rank_odd, seg, tkeys);
}

__global__ void k_check_finite(const double *x, long long n, int *flags)
{
    int bad = 0;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        if (!isfinite(x[i])) bad = 1;
    if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(flags, FLAG_NONFINITE);
}

void launch_check_finite(const double *x, long long n, int *d_flags, cudaStream_t s)
{
    long long nb = (n + 255) / 256;
    if (nb > 2048) nb = 2048;
    if (nb < 1) nb = 1;
    note_launch();
    k_check_finite<<<(unsigned)nb, 256, 0, s>>>(x, n, d_flags);
}

template void launch_sort_points<float>(const double *, const double *, const int *,
                                        const uint32_t *, long long, const Geom *, int, float4 *,
                                        float2 *, cudaStream_t);
template void launch_sort_points<double>(const double *, const double *, const int *,
                                         const uint32_t *, long long, const Geom *, int,
                                         double4 *, double2 *, cudaStream_t);
template void launch_permute_moments<float>(const double *, const int *, long long, float4 *,
                                            float2 *, cudaStream_t);
template void launch_permute_moments<double>(const double *, const int *, long long, double4 *,
                                             double2 *, cudaStream_t);

}  // namespace ccfmm
