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
__global__ void __launch_bounds__(256) k_list_level(
    int lv, const int *leaf_start, int L, const int *rank, int2 *nl, const NearEnt *near_prev,
    const int *cube, OffsetCube ci, int axis, int NB, NearEnt *near_out, long long far_base,
    int FB, FarEnt *far_out, int *far_off, int *far_num, int *near_total, int *far_total,
    int *flags)
{
    __shared__ int s_tot[2];
    if (threadIdx.x < 2) s_tot[threadIdx.x] = 0;
    __syncthreads();
    const long long c = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    const long long nc = 1ll << lv;
    const long long hid = nc + c;
    if (c < nc && cell_count(leaf_start, L, lv, c) == 0) {
        if (lane == 0) {
            nl[hid] = make_int2(0, 0);
            far_off[hid] = 0;
            far_num[hid] = 0;
        }
    } else if (c < nc) {
        const long long r = rank[hid] - rank[nc];
        const long long nbase0 = r * NB, fbase0 = far_base + r * FB;
        const int2 pl = nl[hid >> 1];
        const int bc = (int)(c & 1);
        const int e0 = pl.x, e1 = pl.x + pl.y;
        long long nbase = nbase0, fbase = fbase0;
        const long long nend = nbase0 + NB, fend = fbase0 + FB;
        for (int eb = e0; eb < e1; eb += 32) {
            const int e = eb + lane;
            // up to two near and two far results per lane, in registers
            NearEnt n0{}, n1{};
            FarEnt f0{}, f1{};
            int nn = 0, nf = 0;
            if (e < e1) {
                const NearEnt ne = near_prev[e];
#pragma unroll
                for (int ba = 0; ba < 2; ++ba) {
                    const long long a = 2ll * ne.src + ba;
                    if (cell_count(leaf_start, L, lv, a) == 0) continue;
                    int o[3] = {ne.ox, ne.oy, ne.oz};
                    const int d = bc - ba;
                    o[0] = axis == 0 ? 2 * o[0] + d : o[0];
                    o[1] = axis == 1 ? 2 * o[1] + d : o[1];
                    o[2] = axis == 2 ? 2 * o[2] + d : o[2];
                    const int cls = cube_class(cube, ci, o, flags);
                    if (cls == OFF_NEAR) {
                        const NearEnt x{(int)a, o[0], o[1], o[2]};
                        if (nn == 0) n0 = x; else n1 = x;
                        ++nn;
                    } else if (cls >= 0) {
                        const FarEnt x{(int)a, cls};
                        if (nf == 0) f0 = x; else f1 = x;
                        ++nf;
                    }
                }
            }
            int tn, tf;
            const int pn = warp_excl(nn, lane, &tn);
            const int pf = warp_excl(nf, lane, &tf);
            if (nn > 0) {
                const long long at = nbase + pn;
                if (at + nn <= nend) {
                    near_out[at] = n0;
                    if (nn > 1) near_out[at + 1] = n1;
                } else {
                    atomicOr(flags, FLAG_LIST_OVERFLOW);
                }
            }
            if (nf > 0) {
                const long long at = fbase + pf;
                if (at + nf <= fend) {
                    far_out[at] = f0;
                    if (nf > 1) far_out[at + 1] = f1;
                } else {
                    atomicOr(flags, FLAG_LIST_OVERFLOW);
                }
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
            atomicAdd(&s_tot[0], tn);
            atomicAdd(&s_tot[1], tf);
        }
    }
    // one global addition per block for the level totals
    __syncthreads();
    if (threadIdx.x == 0) {
        if (s_tot[0]) atomicAdd(near_total, s_tot[0]);
        if (s_tot[1]) atomicAdd(far_total, s_tot[1]);
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

// counts[tile] = distinct far offsets among the tile's targets; the tile's
// offset bitmap and the exclusive prefix of its words' popcounts go to
// gbm / gwp (nwmax words a tile) for the fill
__global__ void __launch_bounds__(TL_T) k_tile_count(const Tile *tiles, const int *far_off,
                                                     const int *far_num, const FarEnt *far,
                                                     int nwmax, unsigned *gbm, unsigned *gwp,
                                                     int *counts)
{
    extern __shared__ unsigned bm[];
    __shared__ int sm[32];
    Tile t = tiles[blockIdx.x];
    const int nwords = (t.nbits + 31) / 32;
    tile_bitmap(t, far_off, far_num, far, bm, nwords);
    const int per = (nwords + TL_T - 1) / TL_T;
    const int w0 = threadIdx.x * per;
    int local = 0;
    for (int w = w0; w < w0 + per && w < nwords; ++w) local += __popc(bm[w]);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
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
    unsigned *obm = gbm + (long long)blockIdx.x * nwmax, *owp = gwp + (long long)blockIdx.x * nwmax;
    for (int w = w0; w < w0 + per && w < nwords; ++w) {
        obm[w] = bm[w];
        owp[w] = (unsigned)run;
        run += __popc(bm[w]);
    }
    if (threadIdx.x == 0) counts[blockIdx.x] = sm[TL_T / 32 - 1];
}

// Entries of every tile from its stored bitmap: entry j of the tile is its
// j-th present offset (D table ent_u) with the partner of each target
// (ent_src, -1 beforehand); blockIdx.y takes targets 32 y .. 32 y + 31
constexpr int TF_SPLIT = TT / 32;
__global__ void __launch_bounds__(TL_T) k_tile_fill(const Tile *tiles, const int *ent_start,
                                                    const int *far_off, const int *far_num,
                                                    const FarEnt *far, int nwmax,
                                                    const unsigned *gbm, const unsigned *gwp,
                                                    const int *dmap, int *ent_u, int *ent_src)
{
    const Tile t = tiles[blockIdx.x];
    const unsigned *bm = gbm + (long long)blockIdx.x * nwmax;
    const unsigned *wpre = gwp + (long long)blockIdx.x * nwmax;
    const int start = ent_start[blockIdx.x];
    if (blockIdx.y == 0) {
        const int nwords = (t.nbits + 31) / 32;
        for (int w = threadIdx.x; w < nwords; w += blockDim.x) {
            unsigned b = bm[w];
            int r = (int)wpre[w];
            while (b) {
                const int bit = __ffs(b) - 1;
                ent_u[start + r] = dmap[t.gid_base + w * 32 + bit];  // D table of the class
                ++r;
                b &= b - 1;
            }
        }
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int i1 = min(t.nt, 32 * ((int)blockIdx.y + 1));
    for (int i = 32 * blockIdx.y + warp; i < i1; i += nw) {
        const long long hid = (1ll << t.level) + t.keys[i];
        const int e0 = far_off[hid], n = far_num[hid];
        for (int e = lane; e < n; e += 32) {
            const FarEnt fe = far[e0 + e];
            const int u = fe.gid - t.gid_base;
            const int pos = (int)__ldg(wpre + (u >> 5)) +
                            __popc(__ldg(bm + (u >> 5)) & ((1u << (u & 31)) - 1u));
            ent_src[((long long)start + pos) * TT + i] = (1 << t.level) + fe.src;
        }
    }
}

void launch_tile_count(const Tile *tiles, int ntiles, const int *far_off, const int *far_num,
                       const FarEnt *far, int max_bits, unsigned *gbm, unsigned *gwp, int *counts,
                       cudaStream_t s)
{
    if (ntiles <= 0) return;
    const int nwmax = (max_bits + 31) / 32;
    size_t smem = (size_t)nwmax * sizeof(unsigned);
    if (smem > 48 * 1024)
        cudaFuncSetAttribute(k_tile_count, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    note_launch();
    k_tile_count<<<ntiles, TL_T, smem, s>>>(tiles, far_off, far_num, far, nwmax, gbm, gwp, counts);
}

void launch_tile_fill(Tile *tiles, int ntiles, const int *ent_start, const int *far_off,
                      const int *far_num, const FarEnt *far, int max_bits, const unsigned *gbm,
                      const unsigned *gwp, const int *dmap, int *ent_u, int *ent_src,
                      cudaStream_t s)
{
    if (ntiles <= 0) return;
    note_launch();
    k_tile_fill<<<dim3((unsigned)ntiles, TF_SPLIT), TL_T, 0, s>>>(
        tiles, ent_start, far_off, far_num, far, (max_bits + 31) / 32, gbm, gwp, dmap, ent_u,
        ent_src);
}

}  // namespace ccfmm
