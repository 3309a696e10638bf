// lists.cu -- interaction lists (Sec. II step 1; Appendix createPartners) on
// the GPU, level by level, and the M2L work tiles.
//
// createPartners, restated per level: the near pairs of level l (self pairs
// included) expand into child pairs; a child pair (c, a), c != a, is near if
// its opening angle 2r/d exceeds alpha_m, else it is a far pair (a Partners
// entry of c, used by M2L at level l+1).  A self pair (P, P) expands into the
// sibling pairs, i.e. the step "put one child into the other child's
// Partners list".  At the leaf level near pairs are the nearPartners lists
// (self included).  Empty cells are skipped: they hold no dipoles, so their
// moments are zero and they need no field.
//
// All level-l cells are congruent, so near/far depends only on the integer
// offset o = coords(field cell) - coords(partner); the host classifies every
// offset that a near parent pair can produce (OffsetCube) and the kernels
// look the class up.
#include "ccfmm_dev.cuh"

namespace ccfmm {

__device__ __forceinline__ int cell_count(const int *leaf_start, int L, int l, long long key)
{
    int sh = L - l;
    return leaf_start[(key + 1) << sh] - leaf_start[key << sh];
}

__device__ __forceinline__ int cube_class(const int *cube, const OffsetCube &ci, const int o[3],
                                          int *flags)
{
    if (abs(o[0]) > ci.R[0] || abs(o[1]) > ci.R[1] || abs(o[2]) > ci.R[2]) {
        atomicOr(flags, FLAG_OFFSET_RANGE);
        return OFF_NONE;
    }
    long long idx = ci.base + ((long long)(o[2] + ci.R[2]) * (2 * ci.R[1] + 1) + (o[1] + ci.R[1])) *
                                  (2 * ci.R[0] + 1) + (o[0] + ci.R[0]);
    int v = cube[idx];
    if (v == OFF_NONE) atomicOr(flags, FLAG_OFFSET_RANGE);
    return v;
}

__device__ __forceinline__ int warp_excl(int v, int lane, int *total)
{
    int x = v;
    for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    *total = __shfl_sync(0xffffffffu, x, 31);
    return x - v;
}

// One level in one pass, warp per cell c.  Lists live in fixed slots: the
// r-th non-empty cell of the level (r = rank[hid] - rank[2^lv], rank = the
// exclusive prefix of the non-empty flags over all heap ids) owns NB near and
// FB far entries, NB / FB = the level's near / far offset classes, which
// bound the partners a cell can have (each offset at most once).  The cell's
// near list is nl[hid] = (first slot entry, count); its far list far_off /
// far_num.  No count pass or scan is needed; the level totals go to
// near_total / far_total for the statistics.  The order of a cell's entries,
// (parent entry, child bit), is the same as the oracle's recursion visits
// them and does not depend on the launch.
__global__ void k_list_level(int lv, const int *leaf_start, int L, const int *rank, int2 *nl,
                             const NearEnt *near_prev, const int *cube, OffsetCube ci, int axis,
                             int NB, NearEnt *near_out, long long far_base, int FB,
                             FarEnt *far_out, int *far_off, int *far_num, int *near_total,
                             int *far_total, int *flags)
{
    const long long c = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    const long long nc = 1ll << lv;
    if (c >= nc) return;
    const long long hid = nc + c;
    if (cell_count(leaf_start, L, lv, c) == 0) {
        if (lane == 0) {
            nl[hid] = make_int2(0, 0);
            far_off[hid] = 0;
            far_num[hid] = 0;
        }
        return;
    }
    const long long r = rank[hid] - rank[nc];
    const long long nbase0 = r * NB, fbase0 = far_base + r * FB;
    const int2 pl = nl[hid >> 1];
    const int bc = (int)(c & 1);
    const int e0 = pl.x, e1 = pl.x + pl.y;
    long long nbase = nbase0, fbase = fbase0;
    const long long nend = nbase0 + NB, fend = fbase0 + FB;
    for (int eb = e0; eb < e1; eb += 32) {
        const int e = eb + lane;
        NearEnt out_n[2];
        FarEnt out_f[2];
        int nn = 0, nf = 0;
        if (e < e1) {
            const NearEnt ne = near_prev[e];
            for (int ba = 0; ba < 2; ++ba) {
                const long long a = 2ll * ne.src + ba;
                if (cell_count(leaf_start, L, lv, a) == 0) continue;
                int o[3] = {ne.ox, ne.oy, ne.oz};
                o[axis] = 2 * o[axis] + bc - ba;
                const int cls = cube_class(cube, ci, o, flags);
                if (cls == OFF_NEAR) {
                    out_n[nn].src = (int)a;
                    out_n[nn].ox = o[0];
                    out_n[nn].oy = o[1];
                    out_n[nn].oz = o[2];
                    ++nn;
                } else if (cls >= 0) {
                    out_f[nf].src = (int)a;
                    out_f[nf].gid = cls;
                    ++nf;
                }
            }
        }
        int tn, tf;
        const int pn = warp_excl(nn, lane, &tn);
        const int pf = warp_excl(nf, lane, &tf);
        for (int j = 0; j < nn; ++j) {
            const long long at = nbase + pn + j;
            if (at < nend)
                near_out[at] = out_n[j];
            else
                atomicOr(flags, FLAG_LIST_OVERFLOW);
        }
        for (int j = 0; j < nf; ++j) {
            const long long at = fbase + pf + j;
            if (at < fend)
                far_out[at] = out_f[j];
            else
                atomicOr(flags, FLAG_LIST_OVERFLOW);
        }
        nbase += tn;
        fbase += tf;
    }
    if (lane == 0) {
        const int tn = (int)min(nbase - nbase0, (long long)NB);
        const int tf = (int)min(fbase - fbase0, (long long)FB);
        nl[hid] = make_int2((int)nbase0, tn);
        far_off[hid] = (int)fbase0;
        far_num[hid] = tf;
        atomicAdd(near_total, tn);
        atomicAdd(far_total, tf);
    }
}

void launch_list_level(int level, const int *leaf_start, int L, const int *rank, int2 *nl,
                       const NearEnt *near_prev, const int *cube, OffsetCube cube_info, int axis,
                       int NB, NearEnt *near_out, long long far_base, int FB, FarEnt *far_out,
                       int *far_off, int *far_num, int *near_total, int *far_total, int *d_flags,
                       cudaStream_t s)
{
    const long long threads = (1ll << level) * 32;
    note_launch();
    k_list_level<<<(unsigned)((threads + 255) / 256), 256, 0, s>>>(
        level, leaf_start, L, rank, nl, near_prev, cube, cube_info, axis, NB, near_out, far_base,
        FB, far_out, far_off, far_num, near_total, far_total, d_flags);
}

// ---------------------------------------------------------------------------
// M2L tiles: for each tile (up to TT same-parity targets of one level) the
// distinct far offsets present among its targets, and for each such offset
// the partner of every target (heap id, or -1).
// ---------------------------------------------------------------------------
constexpr int TL_T = 256;

__device__ __forceinline__ void tile_bitmap(const Tile &t, const int *far_off, const int *far_num,
                                            const FarEnt *far, unsigned *bm, int nwords)
{
    for (int w = threadIdx.x; w < nwords; w += blockDim.x) bm[w] = 0u;
    __syncthreads();
    int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    for (int i = warp; i < t.nt; i += nw) {
        long long hid = (1ll << t.level) + t.keys[i];
        int e0 = far_off[hid], n = far_num[hid];
        for (int e = lane; e < n; e += 32) {
            int u = far[e0 + e].gid - t.gid_base;
            atomicOr(&bm[u >> 5], 1u << (u & 31));
        }
    }
    __syncthreads();
}

__global__ void __launch_bounds__(TL_T) k_tile_count(const Tile *tiles, const int *far_off,
                                                     const int *far_num, const FarEnt *far,
                                                     int *counts)
{
    extern __shared__ unsigned bm[];
    __shared__ int red[TL_T / 32];
    Tile t = tiles[blockIdx.x];
    int nwords = (t.nbits + 31) / 32;
    tile_bitmap(t, far_off, far_num, far, bm, nwords);
    int c = 0;
    for (int w = threadIdx.x; w < nwords; w += blockDim.x) c += __popc(bm[w]);
    for (int o = 16; o; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = c;
    __syncthreads();
    if (threadIdx.x == 0) {
        int s = 0;
        for (int w = 0; w < TL_T / 32; ++w) s += red[w];
        counts[blockIdx.x] = s;
    }
}

__global__ void __launch_bounds__(TL_T) k_tile_fill(const Tile *tiles, const int *ent_start,
                                                    const int *far_off, const int *far_num,
                                                    const FarEnt *far, const int *dmap, int *ent_u,
                                                    int *ent_src)
{
    extern __shared__ unsigned bm[];
    __shared__ int sm[32];
    Tile t = tiles[blockIdx.x];
    int nwords = (t.nbits + 31) / 32;
    unsigned *wpre = bm + nwords;
    tile_bitmap(t, far_off, far_num, far, bm, nwords);
    // exclusive prefix of the popcounts over the bitmap words
    int per = (nwords + TL_T - 1) / TL_T;
    int w0 = threadIdx.x * per;
    int local = 0;
    for (int w = w0; w < w0 + per && w < nwords; ++w) local += __popc(bm[w]);
    int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int x = local;
    for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) sm[warp] = x;
    __syncthreads();
    if (warp == 0) {
        int v = lane < TL_T / 32 ? sm[lane] : 0;
        for (int o = 1; o < 32; o <<= 1) {
            int y = __shfl_up_sync(0xffffffffu, v, o);
            if (lane >= o) v += y;
        }
        sm[lane] = v;
    }
    __syncthreads();
    int run = (warp ? sm[warp - 1] : 0) + x - local;
    for (int w = w0; w < w0 + per && w < nwords; ++w) {
        wpre[w] = (unsigned)run;
        run += __popc(bm[w]);
    }
    __syncthreads();
    int start = ent_start[blockIdx.x];
    int count = ent_start[blockIdx.x + 1] - start;
    for (int w = threadIdx.x; w < nwords; w += blockDim.x) {
        unsigned b = bm[w];
        int r = (int)wpre[w];
        while (b) {
            int bit = __ffs(b) - 1;
            ent_u[start + r] = dmap[t.gid_base + w * 32 + bit];  // D table of the class
            ++r;
            b &= b - 1;
        }
    }
    for (long long j = threadIdx.x; j < (long long)count * TT; j += blockDim.x)
        ent_src[(long long)start * TT + j] = -1;
    __syncthreads();
    int nw = blockDim.x >> 5;
    for (int i = warp; i < t.nt; i += nw) {
        long long hid = (1ll << t.level) + t.keys[i];
        int e0 = far_off[hid], n = far_num[hid];
        for (int e = lane; e < n; e += 32) {
            FarEnt fe = far[e0 + e];
            int u = fe.gid - t.gid_base;
            int pos = (int)wpre[u >> 5] + __popc(bm[u >> 5] & ((1u << (u & 31)) - 1u));
            ent_src[((long long)start + pos) * TT + i] = (1 << t.level) + fe.src;
        }
    }
}

void launch_tile_count(const Tile *tiles, int ntiles, const int *far_off, const int *far_num,
                       const FarEnt *far, int max_bits, int *counts, cudaStream_t s)
{
    if (ntiles <= 0) return;
    size_t smem = (size_t)((max_bits + 31) / 32) * sizeof(unsigned);
    if (smem > 48 * 1024)
        cudaFuncSetAttribute(k_tile_count, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    note_launch();
    k_tile_count<<<ntiles, TL_T, smem, s>>>(tiles, far_off, far_num, far, counts);
}

void launch_tile_fill(Tile *tiles, int ntiles, const int *ent_start, const int *far_off,
                      const int *far_num, const FarEnt *far, int max_bits, const int *dmap, int *ent_u,
                      int *ent_src, cudaStream_t s)
{
    if (ntiles <= 0) return;
    size_t smem = 2 * (size_t)((max_bits + 31) / 32) * sizeof(unsigned);
    if (smem > 48 * 1024)
        cudaFuncSetAttribute(k_tile_fill, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    note_launch();
    k_tile_fill<<<ntiles, TL_T, smem, s>>>(tiles, ent_start, far_off, far_num, far, dmap, ent_u, ent_src);
}

}  // namespace ccfmm
