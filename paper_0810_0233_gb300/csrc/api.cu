// api.cu -- the C-ABI of libccfmm (include/ccfmm.h): handle, validation,
// device memory, the build (tree, lists, D tables) and the evaluation graph
// of kernels, with a small number of host synchronisation points during the
// build (depth choice, per-level sizes, list totals).
#include "../../include/ccfmm.h"
#include "ccfmm_dev.cuh"

#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <array>
#include <chrono>
#include <map>
#include <string>
#include <unordered_map>
#include <vector>

using namespace ccfmm;


// ---------------------------------------------------------------- launches
#include <atomic>
static std::atomic<long long> g_launches(0);
void ccfmm::note_launch(int n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

// ---------------------------------------------------------------- errors
static thread_local std::string g_err;

void ccfmm::set_last_error(const char *msg) { g_err = msg; }

static ccfmm_status fail(ccfmm_status st, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_err = buf;
    return st;
}

#define CK(call)                                                                                 \
    do {                                                                                         \
        cudaError_t e_ = (call);                                                                 \
        if (e_ != cudaSuccess) {                                                                 \
            cudaGetLastError();                                                                  \
            return fail(CCFMM_ERR_CUDA, "%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_),   \
                        __FILE__, __LINE__);                                                     \
        }                                                                                        \
    } while (0)
#define TRY(x)                                                                                   \
    do {                                                                                         \
        ccfmm_status s_ = (x);                                                                   \
        if (s_ != CCFMM_OK) return s_;                                                           \
    } while (0)
#define KCHECK() CK(cudaGetLastError())

// test hook: CCFMM_FAIL_ALLOC=k makes the k-th device allocation of the
// process fail (k >= 1), to exercise the error path without a GPU fault.
static long long g_alloc_count = 0;
static long long fail_alloc_at()
{
    static long long v = -2;
    if (v == -2) {
        const char *e = getenv("CCFMM_FAIL_ALLOC");
        v = e ? atoll(e) : -1;
    }
    return v;
}

struct DevBuf {
    void *p = nullptr;
    size_t bytes = 0;
};

static ccfmm_status ensure(DevBuf &b, size_t bytes)
{
    if (bytes == 0) bytes = 16;
    if (b.p && b.bytes >= bytes) return CCFMM_OK;
    if (b.p) cudaFree(b.p);
    b.p = nullptr;
    b.bytes = 0;
    ++g_alloc_count;
    if (fail_alloc_at() > 0 && g_alloc_count == fail_alloc_at())
        return fail(CCFMM_ERR_ALLOC, "device allocation of %zu bytes failed (injected)", bytes);
    cudaError_t e = cudaMalloc(&b.p, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        b.p = nullptr;
        return fail(CCFMM_ERR_ALLOC, "device allocation of %zu bytes failed: %s", bytes,
                    cudaGetErrorString(e));
    }
    b.bytes = bytes;
    return CCFMM_OK;
}

template <typename T> static T *P(DevBuf &b) { return reinterpret_cast<T *>(b.p); }

// small block of device values read back at the build's sync points
struct Readback {
    int flags;
    int hist[LCAP + 1];
    int ne[LCAP + 1];
    int ne_odd[LCAP + 1];  // non-empty cells with an odd key, per level
    int near_total[LCAP + 1];
    int far_total[LCAP + 1];
    int ent_total;
    int pad;
    unsigned long long pairs;
    double box6[6];
    double E;
    // raised by evaluation kernels (bounded waits); kept across builds until
    // a synchronising call has reported it.  Last member: the build clears
    // everything before it.
    int eflags;
    int pad2;
};

struct LevelPlan {
    std::vector<int> nearv, farv;  // packed offsets
    int R[3] = {0, 0, 0};
    long long cube_base = 0;
    long long near_bound = 0, far_bound = 0, far_base = 0;
    int gid_base = 0;
};

// build events, then a ring of per-evaluation stage events so that stage
// times of evaluations inside a caller's timed region can be read afterwards
enum { EV_B0, EV_BS1, EV_BS2, EV_BS3, EV_BS4, EV_B1, EV_NB };
// evaluation events: far chain E0..L2L, near field P2P0..P2P1, then the join
// (both done), L2P and the unpermute (FIN)
enum { EV_E0, EV_P2M, EV_M2M, EV_M2L, EV_L2L, EV_JOIN, EV_L2P, EV_FIN, EV_P2P0, EV_P2P1, EV_NE };
constexpr int EV_RING = 32;

struct ccfmm_s {
    int device = 0;
    cudaStream_t stream = nullptr;
    long long N = 0;
    int p = 0;
    double theta = 0.0, leaf_req = 0.0, leaf_target = 0.0;
    ccfmm_prec prec = CCFMM_MIXED;
    bool has_box = false;
    double box_user[6] = {0, 0, 0, 0, 0, 0};
    int K = 0, KP = 0, TD = 0, ldD = 0;
    int maxdeg = 0;  // M2L terms with |n|+|k| <= maxdeg (2p: square truncation)
    size_t rsz = 4;  // sizeof(real)

    Geom geom;
    int L = 0;
    bool capped = false;
    std::vector<LevelPlan> plan;
    int n_off = 0, ntiles = 0, max_bits = 0;
    int n_d = 0;  // distinct scaled separations (D tables) over all far offset classes
    long long near_leaf_total = 0, far_total = 0, ent_total = 0;
    double ms_plan_host = 0.0;  // host time of the last make_plan
    bool built = false, evaluated = false, ftable_ready = false;
    bool tc_ops_ready = false;  // tensor-core M2L operators of the current build
    bool pairs_counted = false; // near-pair count of the current build taken
    long long pairs = 0;
    bool rb_fresh = true;       // device readback block not yet initialised
    bool leaf_perm_valid = false;

    DevBuf pos, mom, keys, keys2, keys3, idx, idx2, idx3, sorttemp, scantemp;
    DevBuf geomd, box6, userbox, partial, rb;
    DevBuf leaf_start, A, B, H;
    DevBuf cube, nl, neA, neB, cflag, crank, oflag, orank, tkeys, tseg;
    DevBuf far, far_off, far_num, tiles, tcount, tstart, ent_u, ent_src, tbm, twp;
    DevBuf offs, fst, fq, fval, fdense, D, itab, Q, V;
    DevBuf Hout, epart, items, titem0, tnitems, Ps;
    DevBuf Qs, Bop, gkt;  // tensor-core M2L: split moments, operators, level scales
    // tensor map of Qs for the TMA row gather, encoded for (qmap_for, qmap_ncell)
    alignas(64) unsigned char qmap[128];
    const void *qmap_for = nullptr;
    long long qmap_ncell = 0;
    bool qmap_ok = false;
    DevBuf dmap, dsep;    // far offset class -> D table; scaled separation of each D table
    // host sources of the build's asynchronous uploads, kept until the next
    // build (which starts after the previous one has synchronised)
    std::vector<int> h_cube, h_dmap, h_i0, h_ni;
    std::vector<int4> h_offs;
    std::vector<double4> h_dsep;
    std::vector<M2LItem> h_items;
    std::vector<Tile> h_tiles;
    int h_ns0[2] = {0, 1};
    int h_seg[2 * (LCAP + 1)];  // tile key segments per (level, parity)
    NearEnt h_e0 = {0, 0, 0, 0};
    int nitems = 0;
    // batch members: energy input and output redirected, no stage events
    int item_len = M2L_EC;  // entries per M2L work item (the batch autotuner may change it)
    const double *mom_energy = nullptr;
    double *E_dst = nullptr;
    bool quiet = false;
    Readback *hrb = nullptr;  // pinned
    int2 *near_nl = nullptr;  // leaf near lists: (first entry, count) per leaf
    size_t near_leaf_bytes = 0;
    NearEnt *near_leaf = nullptr;
    cudaEvent_t evb[EV_NB];
    cudaEvent_t eve[EV_RING][EV_NE];
    long long n_eval = 0, n_eval_reset = 0;
    bool ev_ok = false;
    // near/far overlap: the far chain runs on s_far (highest priority) while
    // the near field runs on the handle's stream
    cudaStream_t s_far = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    ccfmm_stats st;
};

static bool is_device_ptr(const void *p)
{
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

static ccfmm_status copy_in(ccfmm_t h, DevBuf &dst, const double *src, long long n)
{
    TRY(ensure(dst, sizeof(double) * (size_t)n));
    cudaMemcpyKind k = is_device_ptr(src) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    CK(cudaMemcpyAsync(dst.p, src, sizeof(double) * (size_t)n, k, h->stream));
    return CCFMM_OK;
}

double ccfmm_leaf_size_rule(int p) { return p > 3 ? 0.74 * (double)p * (double)p : 8.0; }

// ------------------------------------------------------------ offset plan
// near iff alpha = 2r/d > theta, r = |w|/2: |w|^2 > theta^2 d^2 (1 + 1e-12);
// the factor makes a computed tie alpha == theta count as far.
static bool near_offset(const int o[3], const double w[3], double theta)
{
    double W2 = w[0] * w[0] + w[1] * w[1] + w[2] * w[2];
    double d2 = 0.0;
    for (int a = 0; a < 3; ++a) {
        double x = (double)o[a] * w[a];
        d2 += x * x;
    }
    return W2 > theta * theta * d2 * (1.0 + 1e-12);
}

static inline int packo(int x, int y, int z)
{
    return ((x + 512) & 1023) | (((y + 512) & 1023) << 10) | (((z + 512) & 1023) << 20);
}
static inline void unpacko(int v, int o[3])
{
    o[0] = (v & 1023) - 512;
    o[1] = ((v >> 10) & 1023) - 512;
    o[2] = ((v >> 20) & 1023) - 512;
}

// Offsets a near parent pair can produce at each level, classified near/far
// (createPartners restated on integer offsets of congruent cells).
static ccfmm_status make_plan(ccfmm_t h)
{
    int L = h->L;
    h->plan.assign(L + 1, LevelPlan());
    h->plan[0].nearv.push_back(packo(0, 0, 0));
    long long cube_total = 0;
    int gid = 0;
    for (int l = 1; l <= L; ++l) {
        int s = h->geom.axis[l];
        std::vector<int> cand;
        cand.reserve(h->plan[l - 1].nearv.size() * 3);
        for (int v : h->plan[l - 1].nearv) {
            int O[3];
            unpacko(v, O);
            for (int d = -1; d <= 1; ++d) {
                int o[3] = {O[0], O[1], O[2]};
                o[s] = 2 * O[s] + d;
                for (int a = 0; a < 3; ++a) {
                    long long nmax = (1ll << h->geom.nsplit[l][a]) - 1;
                    if (o[a] > nmax || o[a] < -nmax) goto skip;
                }
                if (abs(o[0]) > 511 || abs(o[1]) > 511 || abs(o[2]) > 511)
                    return fail(CCFMM_ERR_ARG, "theta %g too small for this tree: partner offsets "
                                "exceed 511 cells", h->theta);
                cand.push_back(packo(o[0], o[1], o[2]));
            skip:;
            }
        }
        std::sort(cand.begin(), cand.end());
        cand.erase(std::unique(cand.begin(), cand.end()), cand.end());
        LevelPlan &lp = h->plan[l];
        for (int v : cand) {
            int o[3];
            unpacko(v, o);
            bool self = o[0] == 0 && o[1] == 0 && o[2] == 0;
            if (self || near_offset(o, h->geom.w[l], h->theta))
                lp.nearv.push_back(v);
            else
                lp.farv.push_back(v);
            for (int a = 0; a < 3; ++a) lp.R[a] = std::max(lp.R[a], abs(o[a]));
        }
        lp.cube_base = cube_total;
        cube_total += (long long)(2 * lp.R[0] + 1) * (2 * lp.R[1] + 1) * (2 * lp.R[2] + 1);
        lp.gid_base = gid;
        gid += (int)lp.farv.size();
        if ((long long)lp.farv.size() > (1 << 18))
            return fail(CCFMM_ERR_ARG, "theta %g too small: %zu far offsets at level %d",
                        h->theta, lp.farv.size(), l);
    }
    if (cube_total > (1ll << 28)) return fail(CCFMM_ERR_ARG, "theta %g too small", h->theta);
    h->n_off = gid;
    // concatenated cube tables
    std::vector<int> &cube = h->h_cube;
    std::vector<int4> &offs = h->h_offs;
    cube.assign((size_t)std::max(cube_total, 1ll), OFF_NONE);
    offs.assign((size_t)std::max(gid, 1), make_int4(0, 0, 0, 0));
    for (int l = 1; l <= L; ++l) {
        LevelPlan &lp = h->plan[l];
        auto at = [&](const int o[3]) {
            return lp.cube_base + ((long long)(o[2] + lp.R[2]) * (2 * lp.R[1] + 1) + (o[1] + lp.R[1])) *
                                      (2 * lp.R[0] + 1) + (o[0] + lp.R[0]);
        };
        for (int v : lp.nearv) {
            int o[3];
            unpacko(v, o);
            cube[at(o)] = OFF_NEAR;
        }
        for (size_t u = 0; u < lp.farv.size(); ++u) {
            int o[3];
            unpacko(lp.farv[u], o);
            cube[at(o)] = lp.gid_base + (int)u;
            offs[lp.gid_base + u] = make_int4(o[0], o[1], o[2], l);
        }
    }
    // D tables depend on the separation in units of the level's cell radius
    // only, c/h = (o_x w_x, o_y w_y, o_z w_z) / h; levels of the same cell
    // shape (every third level of a cubic box) share them.  One table per
    // distinct scaled separation (exact FP64 equality).
    std::vector<int> &dmap = h->h_dmap;
    std::vector<double4> &dsep = h->h_dsep;
    dmap.assign((size_t)std::max(gid, 1), 0);
    dsep.clear();
    {
        // levels grouped by their exact scaled cell shape w/h; inside a group
        // an open-addressing table maps the packed integer offset to a D
        // table, which is reused only when its separation is bitwise equal
        size_t cap = 64;
        while (cap < 4 * (size_t)std::max(gid, 1)) cap <<= 1;
        std::vector<std::array<double, 3>> shapes;
        std::vector<std::vector<std::pair<int, int>>> tabs;  // (packed offset, D table)
        for (int l = 1; l <= L; ++l) {
            const LevelPlan &lp = h->plan[l];
            if (lp.farv.empty()) continue;
            const double hl = h->geom.h[l];
            const std::array<double, 3> shp = {h->geom.w[l][0] / hl, h->geom.w[l][1] / hl,
                                               h->geom.w[l][2] / hl};
            size_t gi = 0;
            while (gi < shapes.size() && memcmp(&shapes[gi], &shp, sizeof(shp)) != 0) ++gi;
            if (gi == shapes.size()) {
                shapes.push_back(shp);
                tabs.emplace_back(cap, std::make_pair(-1, -1));
            }
            std::vector<std::pair<int, int>> &tab = tabs[gi];
            for (size_t u = 0; u < lp.farv.size(); ++u) {
                const int key = lp.farv[u];
                int o[3];
                unpacko(key, o);
                const double v[3] = {(double)o[0] * h->geom.w[l][0] / hl,
                                     (double)o[1] * h->geom.w[l][1] / hl,
                                     (double)o[2] * h->geom.w[l][2] / hl};
                size_t k = ((uint32_t)key * 2654435761u) & (cap - 1);
                while (tab[k].first != -1 && tab[k].first != key) k = (k + 1) & (cap - 1);
                int d = tab[k].first == key ? tab[k].second : -1;
                if (d >= 0) {
                    const double4 &e = dsep[d];
                    const double w3[3] = {e.x, e.y, e.z};
                    if (memcmp(w3, v, sizeof(v)) != 0) d = -1;
                }
                if (d < 0) {
                    d = (int)dsep.size();
                    dsep.push_back(make_double4(v[0], v[1], v[2], 0.0));
                    tab[k] = std::make_pair(key, d);
                }
                dmap[lp.gid_base + u] = d;
            }
        }
    }
    h->n_d = (int)dsep.size();
    TRY(ensure(h->cube, sizeof(int) * cube.size()));
    CK(cudaMemcpyAsync(h->cube.p, cube.data(), sizeof(int) * cube.size(), cudaMemcpyHostToDevice,
                       h->stream));
    TRY(ensure(h->offs, sizeof(int4) * offs.size()));
    CK(cudaMemcpyAsync(h->offs.p, offs.data(), sizeof(int4) * offs.size(), cudaMemcpyHostToDevice,
                       h->stream));
    TRY(ensure(h->dmap, sizeof(int) * dmap.size()));
    CK(cudaMemcpyAsync(h->dmap.p, dmap.data(), sizeof(int) * dmap.size(), cudaMemcpyHostToDevice,
                       h->stream));
    TRY(ensure(h->dsep, sizeof(double4) * std::max<size_t>(dsep.size(), 1)));
    if (!dsep.empty())
        CK(cudaMemcpyAsync(h->dsep.p, dsep.data(), sizeof(double4) * dsep.size(),
                           cudaMemcpyHostToDevice, h->stream));
    return CCFMM_OK;
}

// ------------------------------------------------------------ build
static ccfmm_status check_flags(ccfmm_t h, int flags)
{
    if (flags & FLAG_NONFINITE) return fail(CCFMM_ERR_ARG, "non-finite position or moment");
    if (flags & FLAG_OUTSIDE_BOX) return fail(CCFMM_ERR_ARG, "a position lies outside the box");
    if (flags & FLAG_OFFSET_RANGE)
        return fail(CCFMM_ERR_STATE, "internal: partner offset outside the planned range");
    if (flags & FLAG_LIST_OVERFLOW) return fail(CCFMM_ERR_STATE, "internal: list overflow");
    if (flags & FLAG_TIMEOUT) return fail(CCFMM_ERR_TIMEOUT, "a bounded device wait gave up");
    (void)h;
    return CCFMM_OK;
}

static ccfmm_status overlap_prepare(ccfmm_t h);

static ccfmm_status build(ccfmm_t h, const double *positions, const double *moments)
{
    cudaStream_t s = h->stream;
    long long N = h->N;
    h->built = h->evaluated = false;
    if (h->ev_ok) CK(cudaEventRecord(h->evb[EV_B0], s));
    TRY(copy_in(h, h->pos, positions, 3 * N));
    TRY(copy_in(h, h->mom, moments, 3 * N));
    TRY(ensure(h->rb, sizeof(Readback)));
    TRY(ensure(h->geomd, sizeof(Geom)));
    TRY(ensure(h->box6, 6 * sizeof(double)));
    TRY(ensure(h->partial, 6 * sizeof(double) * 1024));
    Readback *drb = P<Readback>(h->rb);
    if (h->rb_fresh) {
        CK(cudaMemsetAsync(drb, 0, sizeof(Readback), s));
        h->rb_fresh = false;
    } else {
        CK(cudaMemsetAsync(drb, 0, offsetof(Readback, eflags), s));
    }
    const double *ubox = nullptr;
    if (h->has_box) {
        TRY(ensure(h->userbox, 6 * sizeof(double)));
        CK(cudaMemcpyAsync(h->userbox.p, h->box_user, 6 * sizeof(double), cudaMemcpyHostToDevice, s));
        ubox = P<double>(h->userbox);
    }
    launch_check_finite(P<double>(h->mom), 3 * N, &drb->flags, s);
    launch_bbox(P<double>(h->pos), N, ubox, P<double>(h->box6), P<double>(h->partial), &drb->flags, s);
    launch_geom(P<double>(h->box6), P<Geom>(h->geomd), s);
    // keys and sort
    TRY(ensure(h->keys, sizeof(uint32_t) * N));
    TRY(ensure(h->keys2, sizeof(uint32_t) * N));
    TRY(ensure(h->keys3, sizeof(uint32_t) * N));
    TRY(ensure(h->idx, sizeof(int) * N));
    TRY(ensure(h->idx2, sizeof(int) * N));
    TRY(ensure(h->idx3, sizeof(int) * N));
    TRY(ensure(h->sorttemp, radix_temp_bytes(N)));
    launch_keys(P<double>(h->pos), N, P<Geom>(h->geomd), P<uint32_t>(h->keys), P<int>(h->idx2),
                &drb->flags, h->has_box ? 1 : 0, s);
    // sorted keys -> keys2, permutation (sorted -> input index) -> idx
    radix_sort(P<uint32_t>(h->keys), P<int>(h->idx2), P<uint32_t>(h->keys2), P<int>(h->idx),
               P<uint32_t>(h->keys3), P<int>(h->idx3), N, LCAP, h->sorttemp.p, s);
    launch_depth_hist(P<uint32_t>(h->keys2), N, drb->hist, s);
    KCHECK();
    if (h->ev_ok) CK(cudaEventRecord(h->evb[EV_BS1], s));
    // sync 1: flags, box, depth histogram, geometry
    CK(cudaMemcpyAsync(h->hrb, drb, sizeof(Readback), cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(&h->geom, h->geomd.p, sizeof(Geom), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (h->hrb->eflags) {
        // reported once: an evaluation since the last synchronising call
        // gave up on a bounded wait
        CK(cudaMemsetAsync(&drb->eflags, 0, sizeof(int), s));
        CK(cudaStreamSynchronize(s));
        TRY(check_flags(h, h->hrb->eflags));
    }
    TRY(check_flags(h, h->hrb->flags));

    // depth: L minimising |N / nonempty_L - s| (ties to the smaller L);
    // N / nonempty_L never increases, so the scan stops once it is <= s
    {
        double best = INFINITY;
        int bestL = 0;
        long long ne = 1;
        bool stopped = false;
        for (int l = 0; l <= LCAP; ++l) {
            ne += h->hrb->hist[l];
            double avg = (double)N / (double)ne;
            double dev = fabs(avg - h->leaf_target);
            if (dev < best) {
                best = dev;
                bestL = l;
            }
            if (avg <= h->leaf_target) {
                stopped = true;
                break;
            }
        }
        h->L = bestL;
        h->capped = !stopped;
        h->geom.L = bestL;
    }
    const int L = h->L;
    const long long nleaf = 1ll << L, ncellp = 1ll << (L + 1);

    TRY(ensure(h->leaf_start, sizeof(int) * (nleaf + 1)));
    launch_leaf_start(P<uint32_t>(h->keys2), N, L, P<int>(h->leaf_start), s);
    const size_t rs = h->rsz;
    TRY(ensure(h->A, 4 * rs * N));
    TRY(ensure(h->B, 2 * rs * N));
    TRY(ensure(h->H, 4 * rs * N));
    if (h->prec == CCFMM_MIXED)
        launch_sort_points<float>(P<double>(h->pos), P<double>(h->mom), P<int>(h->idx),
                                  P<uint32_t>(h->keys2), N, P<Geom>(h->geomd), L, P<float4>(h->A),
                                  P<float2>(h->B), s);
    else
        launch_sort_points<double>(P<double>(h->pos), P<double>(h->mom), P<int>(h->idx),
                                   P<uint32_t>(h->keys2), N, P<Geom>(h->geomd), L,
                                   P<double4>(h->A), P<double2>(h->B), s);
    TRY(ensure(h->cflag, sizeof(int) * ncellp));
    TRY(ensure(h->oflag, sizeof(int) * ncellp));
    launch_level_counts(P<int>(h->leaf_start), L, drb->ne, P<int>(h->cflag), P<int>(h->oflag),
                        drb->ne_odd, s);
    KCHECK();
    if (h->ev_ok) CK(cudaEventRecord(h->evb[EV_BS2], s));
    // the plan needs only the depth and the geometry: the host builds it
    // while the kernels above run (its uploads queue behind them)
    const auto tp0 = std::chrono::steady_clock::now();
    TRY(make_plan(h));
    h->ms_plan_host =
        std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - tp0).count();
    // F table and derivative tensors of every (level, far offset), FP64.
    // They need only the plan, so they run on the far stream beside the
    // list construction and join the handle's stream before the build ends.
    // (ensemble members keep them on their own stream: their builds already
    // run side by side on the ensemble's branch streams)
    const bool side = !h->quiet;
    if (side) {
        TRY(overlap_prepare(h));
        CK(cudaEventRecord(h->ev_fork, s));
        CK(cudaStreamWaitEvent(h->s_far, h->ev_fork, 0));
    }
    const cudaStream_t sd = side ? h->s_far : s;
    int O = 2 * h->p;
    h->TD = nterms(O);
    h->ldD = ((h->TD + 1 + 3) / 4) * 4;
    if (!h->ftable_ready) {
        // the F table depends on p only: built once per handle
        TRY(ensure(h->fdense, ftable_scratch_bytes(O)));
        TRY(ensure(h->fst, sizeof(int) * (h->TD + 1)));
        TRY(ensure(h->fq, sizeof(uint16_t) * h->TD * 160));
        TRY(ensure(h->fval, sizeof(double) * h->TD * 160));
        launch_ftable(O, P<double>(h->fdense), P<int>(h->fst), P<uint16_t>(h->fq),
                      P<double>(h->fval), sd);
        TRY(ensure(h->itab, sizeof(uint16_t) * h->KP * h->KP));
        launch_itable(h->p, h->KP, h->maxdeg, P<uint16_t>(h->itab), sd);
        h->ftable_ready = true;
    }
    TRY(ensure(h->D, rs * (size_t)std::max(h->n_d, 1) * h->ldD));
    if (h->prec == CCFMM_MIXED)
        launch_dtables<float>(h->p, P<int>(h->fst), P<uint16_t>(h->fq), P<double>(h->fval),
                              P<double4>(h->dsep), h->n_d, P<float>(h->D), h->ldD, sd);
    else
        launch_dtables<double>(h->p, P<int>(h->fst), P<uint16_t>(h->fq), P<double>(h->fval),
                               P<double4>(h->dsep), h->n_d, P<double>(h->D), h->ldD, sd);
    KCHECK();
    if (side) CK(cudaEventRecord(h->ev_join, sd));
    // sync 2: non-empty cells per level
    CK(cudaMemcpyAsync(h->hrb, drb, sizeof(Readback), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    h->leaf_perm_valid = true;

    long long near_max = 1, far_sum = 0;
    for (int l = 0; l <= L; ++l) {
        LevelPlan &lp = h->plan[l];
        lp.near_bound = (long long)h->hrb->ne[l] * (long long)lp.nearv.size();
        lp.far_bound = (long long)h->hrb->ne[l] * (long long)lp.farv.size();
        lp.far_base = far_sum;
        far_sum += lp.far_bound;
        near_max = std::max(near_max, lp.near_bound);
    }
    if (near_max >= (1ll << 31) || far_sum >= (1ll << 31))
        return fail(CCFMM_ERR_ARG, "interaction lists too large for 32-bit offsets");
    TRY(ensure(h->nl, sizeof(int2) * ncellp));
    TRY(ensure(h->neA, sizeof(NearEnt) * near_max));
    TRY(ensure(h->neB, sizeof(NearEnt) * near_max));
    TRY(ensure(h->crank, sizeof(int) * (ncellp + 1)));
    TRY(ensure(h->far, sizeof(FarEnt) * std::max(far_sum, 1ll)));
    TRY(ensure(h->far_off, sizeof(int) * ncellp));
    TRY(ensure(h->far_num, sizeof(int) * ncellp));
    TRY(ensure(h->scantemp, scan_temp_bytes(std::max(ncellp, 4096ll) * 256)));
    CK(cudaMemsetAsync(h->far_num.p, 0, sizeof(int) * ncellp, s));
    CK(cudaMemsetAsync(h->far_off.p, 0, sizeof(int) * ncellp, s));
    // rank of every non-empty cell among all heap ids; a level's list slots
    // are indexed by rank within the level
    scan_exclusive(P<int>(h->cflag), P<int>(h->crank), ncellp, P<int>(h->crank) + ncellp,
                   h->scantemp.p, s);
    // the M2L tiles' target cells: non-empty cells per level and parity
    {
        long long tot = 0;
        for (int l = 0; l <= LCAP; ++l) {
            const int odd = l <= L ? h->hrb->ne_odd[l] : 0;
            const int even = l <= L ? h->hrb->ne[l] - odd : 0;
            h->h_seg[2 * l] = (int)tot;
            tot += l >= 2 ? even : 0;
            h->h_seg[2 * l + 1] = (int)tot;
            tot += l >= 2 ? odd : 0;
        }
        TRY(ensure(h->orank, sizeof(int) * (ncellp + 1)));
        TRY(ensure(h->tkeys, sizeof(int) * (size_t)std::max(tot, 1ll)));
        TRY(ensure(h->tseg, sizeof(h->h_seg)));
        scan_exclusive(P<int>(h->oflag), P<int>(h->orank), ncellp, P<int>(h->orank) + ncellp,
                       h->scantemp.p, s);
        CK(cudaMemcpyAsync(h->tseg.p, h->h_seg, sizeof(h->h_seg), cudaMemcpyHostToDevice, s));
        launch_tile_keys(L, P<int>(h->cflag), P<int>(h->crank), P<int>(h->orank), P<int>(h->tseg),
                         P<int>(h->tkeys), s);
    }
    // level 0: the root is near itself (one entry, offset 0)
    CK(cudaMemcpyAsync(P<int2>(h->nl) + 1, h->h_ns0, sizeof(h->h_ns0), cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(h->neA.p, &h->h_e0, sizeof(h->h_e0), cudaMemcpyHostToDevice, s));
    DevBuf *nePrev = &h->neA, *neCur = &h->neB;
    for (int l = 1; l <= L; ++l) {
        LevelPlan &lp = h->plan[l];
        OffsetCube ci;
        ci.R[0] = lp.R[0];
        ci.R[1] = lp.R[1];
        ci.R[2] = lp.R[2];
        ci.base = lp.cube_base;
        launch_list_level(l, P<int>(h->leaf_start), L, P<int>(h->crank), P<int2>(h->nl),
                          P<NearEnt>(*nePrev), P<int>(h->cube), ci, h->geom.axis[l],
                          (int)lp.nearv.size(), P<NearEnt>(*neCur), lp.far_base,
                          (int)lp.farv.size(), P<FarEnt>(h->far), P<int>(h->far_off),
                          P<int>(h->far_num), &drb->near_total[l], &drb->far_total[l],
                          &drb->flags, s);
        std::swap(nePrev, neCur);
    }
    KCHECK();
    h->near_nl = P<int2>(h->nl) + nleaf;
    h->near_leaf = P<NearEnt>(*nePrev);
    h->near_leaf_bytes = sizeof(NearEnt) * (size_t)std::max(1ll, h->plan[L].near_bound);

    // M2L tiles: TT same-parity cells of one level
    std::vector<Tile> &tiles = h->h_tiles;
    tiles.clear();
    h->max_bits = 32;
    // tiles: TT consecutive non-empty cells of one level and parity (empty
    // cells have no far partners and no field to receive)
    for (int l = 2; l <= L; ++l) {
        LevelPlan &lp = h->plan[l];
        if (lp.farv.empty()) continue;
        for (int par = 0; par < 2; ++par) {
            const int cnt = par ? h->hrb->ne_odd[l] : h->hrb->ne[l] - h->hrb->ne_odd[l];
            for (int f = 0; f < cnt; f += TT) {
                Tile t;
                t.level = l;
                t.first = f;
                t.parity = par;
                t.nt = std::min(TT, cnt - f);
                t.ent_start = t.ent_count = 0;
                t.nbits = (int)lp.farv.size();
                t.gid_base = lp.gid_base;
                t.keys = P<int>(h->tkeys) + h->h_seg[2 * l + par] + f;
                tiles.push_back(t);
            }
        }
        h->max_bits = std::max(h->max_bits, (int)lp.farv.size());
    }
    h->ntiles = (int)tiles.size();
    TRY(ensure(h->tiles, sizeof(Tile) * std::max<size_t>(tiles.size(), 1)));
    TRY(ensure(h->tcount, sizeof(int) * (tiles.size() + 1)));
    TRY(ensure(h->tstart, sizeof(int) * (tiles.size() + 1)));
    if (h->ntiles) {
        CK(cudaMemcpyAsync(h->tiles.p, tiles.data(), sizeof(Tile) * tiles.size(),
                           cudaMemcpyHostToDevice, s));
        const size_t tw = (size_t)h->ntiles * ((h->max_bits + 31) / 32);
        TRY(ensure(h->tbm, sizeof(unsigned) * tw));
        TRY(ensure(h->twp, sizeof(unsigned) * tw));
        launch_tile_count(P<Tile>(h->tiles), h->ntiles, P<int>(h->far_off), P<int>(h->far_num),
                          P<FarEnt>(h->far), h->max_bits, P<unsigned>(h->tbm),
                          P<unsigned>(h->twp), P<int>(h->tcount), s);
        scan_exclusive(P<int>(h->tcount), P<int>(h->tstart), h->ntiles, &drb->ent_total,
                       h->scantemp.p, s);
        CK(cudaMemcpyAsync(P<int>(h->tstart) + h->ntiles, &drb->ent_total, sizeof(int),
                           cudaMemcpyDeviceToDevice, s));
    }
    KCHECK();
    if (h->ev_ok) CK(cudaEventRecord(h->evb[EV_BS3], s));
    // sync 3: list totals and M2L work size
    CK(cudaMemcpyAsync(h->hrb, drb, sizeof(Readback), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    TRY(check_flags(h, h->hrb->flags));
    h->near_leaf_total = L == 0 ? 1 : h->hrb->near_total[L];
    h->far_total = 0;
    for (int l = 1; l <= L; ++l) h->far_total += h->hrb->far_total[l];
    h->ent_total = h->ntiles ? h->hrb->ent_total : 0;
    // FP32 M2L work items: runs of at most M2L_EC entries of one tile
    if (h->ntiles) {
        std::vector<int> ts(h->ntiles + 1);
        CK(cudaMemcpyAsync(ts.data(), h->tstart.p, sizeof(int) * (h->ntiles + 1),
                           cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        std::vector<M2LItem> &items = h->h_items;
        std::vector<int> &i0 = h->h_i0, &ni = h->h_ni;
        items.clear();
        i0.assign(h->ntiles, 0);
        ni.assign(h->ntiles, 0);
        for (int t = 0; t < h->ntiles; ++t) {
            i0[t] = (int)items.size();
            for (int e = ts[t]; e < ts[t + 1]; e += h->item_len) {
                M2LItem it;
                it.tile = t;
                it.e0 = e;
                it.e1 = std::min(e + h->item_len, ts[t + 1]);
                items.push_back(it);
            }
            ni[t] = (int)items.size() - i0[t];
        }
        h->nitems = (int)items.size();
        // entry ranges of the tiles, known on the host from the scan
        for (int t = 0; t < h->ntiles; ++t) {
            tiles[t].ent_start = ts[t];
            tiles[t].ent_count = ts[t + 1] - ts[t];
        }
        // uploads ordered on the handle's stream (which may be a non-blocking
        // stream); their host sources belong to the handle
        TRY(ensure(h->items, sizeof(M2LItem) * std::max<size_t>(items.size(), 1)));
        TRY(ensure(h->titem0, sizeof(int) * h->ntiles));
        TRY(ensure(h->tnitems, sizeof(int) * h->ntiles));
        CK(cudaMemcpyAsync(h->tiles.p, tiles.data(), sizeof(Tile) * tiles.size(),
                           cudaMemcpyHostToDevice, s));
        if (!items.empty())
            CK(cudaMemcpyAsync(h->items.p, items.data(), sizeof(M2LItem) * items.size(),
                               cudaMemcpyHostToDevice, s));
        CK(cudaMemcpyAsync(h->titem0.p, i0.data(), sizeof(int) * h->ntiles, cudaMemcpyHostToDevice,
                           s));
        CK(cudaMemcpyAsync(h->tnitems.p, ni.data(), sizeof(int) * h->ntiles,
                           cudaMemcpyHostToDevice, s));
        if (h->prec == CCFMM_MIXED)
            TRY(ensure(h->Ps, sizeof(float) * (size_t)std::max(h->nitems, 1) * TT * h->KP));
    }
    if (h->ev_ok) CK(cudaEventRecord(h->evb[EV_BS4], s));
    TRY(ensure(h->ent_u, sizeof(int) * std::max(h->ent_total, 1ll)));
    TRY(ensure(h->ent_src, sizeof(int) * (size_t)TT * std::max(h->ent_total, 1ll)));
    // every partner slot starts as -1 (no partner): one memset at full bandwidth
    if (h->ent_total > 0)
        CK(cudaMemsetAsync(h->ent_src.p, 0xff, sizeof(int) * (size_t)TT * h->ent_total, s));
    if (h->ntiles)
        launch_tile_fill(P<Tile>(h->tiles), h->ntiles, P<int>(h->tstart), P<int>(h->far_off),
                         P<int>(h->far_num), P<FarEnt>(h->far), h->max_bits,
                         P<unsigned>(h->tbm), P<unsigned>(h->twp), P<int>(h->dmap),
                         P<int>(h->ent_u), P<int>(h->ent_src), s);

    TRY(ensure(h->Q, rs * (size_t)ncellp * h->KP));
    TRY(ensure(h->V, sizeof(double) * (size_t)ncellp * h->KP));
    TRY(ensure(h->epart, sizeof(double) * ((N + 255) / 256 + 1)));
    // the near-pair count (statistics only) is taken by fmm_stats on demand
    h->pairs_counted = false;
    KCHECK();
    if (side) CK(cudaStreamWaitEvent(s, h->ev_join, 0));  // D tables (far stream)
    if (h->ev_ok) CK(cudaEventRecord(h->evb[EV_B1], s));
    // The last kernels (tile fill, D tables, pair count) may still run when
    // the build returns: everything later on the handle's stream is ordered
    // after them, their flags are read by the next synchronising call, the
    // host sources of their uploads belong to the handle and change only
    // after the next build's first synchronisation, and stats, accessors and
    // destroy synchronise first.  The next evaluation is enqueued meanwhile.
    h->built = true;
    h->tc_ops_ready = false;
    return CCFMM_OK;
}

// ------------------------------------------------------------ evaluation
// M2L contraction engine for the FP32 path: the tensor-core kernel (orders
// p = 4..7) unless CCFMM_M2L=fma, which selects the FP32 FMA kernel.
static bool m2l_use_tc(ccfmm_t h)
{
    if (h->prec != CCFMM_MIXED || !m2l_tc_supported(h->KP)) return false;
    const char *e = getenv("CCFMM_M2L");
    if (e && !strcmp(e, "fma")) return false;
    if (e && !strcmp(e, "tc")) return true;
    return M2L_TC_DEFAULT;
}

// Row gather of the tensor-core M2L: TMA tile::gather4 copies, or cp.async
// by eight producer warps (CCFMM_TC_GATHER=tma|cp overrides the default).
constexpr bool TC_GATHER_TMA_DEFAULT = false;
static bool tc_gather_tma()
{
    const char *e = getenv("CCFMM_TC_GATHER");
    if (e && !strcmp(e, "cp")) return false;
    if (e && !strcmp(e, "tma")) return true;
    return TC_GATHER_TMA_DEFAULT;
}

// Where the tensor-core M2L keeps its gathered operand: shared memory
// (cp.async or TMA gather; the default) or tensor memory (filled by
// tcgen05.st from registers); CCFMM_TC_A=smem|tmem overrides the default.
constexpr bool TC_A_TMEM_DEFAULT = false;
static bool tc_a_tmem()
{
    const char *e = getenv("CCFMM_TC_A");
    if (e && !strcmp(e, "smem")) return false;
    if (e && !strcmp(e, "tmem")) return true;
    return TC_A_TMEM_DEFAULT;
}

// Buffers and operators of the tensor-core M2L for the current tree, built
// on the handle's stream at the first evaluation after a build (ensemble
// members: before their evaluation is captured).
static ccfmm_status tc_prepare(ccfmm_t h)
{
    const int KT = m2l_tc_kt(h->KP);
    const long long ncellp = 1ll << (h->L + 1);
    TRY(ensure(h->Qs, sizeof(float) * 2 * (size_t)ncellp * KT));
    if (tc_gather_tma() && (h->qmap_for != h->Qs.p || h->qmap_ncell != ncellp)) {
        // host-side encoding; a map the driver cannot make leaves the
        // cp.async gather in use
        h->qmap_ok = m2l_tc_qmap(h->qmap, P<float>(h->Qs), ncellp, h->KP);
        h->qmap_for = h->Qs.p;
        h->qmap_ncell = ncellp;
    }
    if (!h->tc_ops_ready) {
        TRY(ensure(h->Bop, m2l_tc_op_bytes(h->KP) * (size_t)std::max(h->n_d, 1)));
        TRY(ensure(h->gkt, sizeof(float) * (size_t)(LCAP + 1) * KT));
        launch_m2l_tc_ops(h->p, h->KP, h->L, h->n_d, P<Geom>(h->geomd), P<float>(h->D), h->ldD,
                          P<uint16_t>(h->itab), P<float>(h->gkt), P<float>(h->Bop), h->stream);
        h->tc_ops_ready = true;
    }
    return CCFMM_OK;
}

constexpr int OVERLAP_DEFAULT = 1;

// Near/far overlap for standalone handles (ensemble members already run
// eight-way concurrent inside their graph): 0 off (CCFMM_OVERLAP=0); 1 the
// far chain on the high-priority stream; 2 the near field on it.
static int use_overlap(ccfmm_t h)
{
    if (h->quiet) return 0;
    const char *e = getenv("CCFMM_OVERLAP");
    if (e && (!strcmp(e, "0") || !strcmp(e, "1") || !strcmp(e, "2"))) return e[0] - '0';
    return OVERLAP_DEFAULT;
}

static ccfmm_status overlap_prepare(ccfmm_t h)
{
    if (h->s_far) return CCFMM_OK;
    int least = 0, greatest = 0;
    CK(cudaDeviceGetStreamPriorityRange(&least, &greatest));
    CK(cudaStreamCreateWithPriority(&h->s_far, cudaStreamNonBlocking, greatest));
    CK(cudaEventCreateWithFlags(&h->ev_fork, cudaEventDisableTiming));
    CK(cudaEventCreateWithFlags(&h->ev_join, cudaEventDisableTiming));
    return CCFMM_OK;
}

// One evaluation.  The near field (P2P, Appendix updateField) needs only the
// sorted dipoles and the near lists; the far chain (P2M, M2M, M2L, L2L) only
// the tree.  With the overlap they run on two streams, joined before L2P;
// otherwise in sequence on the handle's stream with L2P fused into P2P.
template <typename real>
static ccfmm_status eval_t(ccfmm_t h, double *Hdev)
{
    typedef typename vec4<real>::t R4;
    typedef typename vec2<real>::t R2;
    cudaStream_t s = h->stream;
    const int L = h->L, p = h->p, KP = h->KP;
    const long long ncellp = 1ll << (L + 1);
    const bool tc = sizeof(real) == 4 && m2l_use_tc(h);
    const int mode = use_overlap(h);
    const bool ovl = mode != 0;
    // one-time operator builds go on s before the fork
    if (tc) TRY(tc_prepare(h));
    if (ovl) TRY(overlap_prepare(h));
    // s_far: the extra (high-priority) stream; it carries the far chain
    // (mode 1) or the near field (mode 2)
    cudaStream_t sf = mode == 1 ? h->s_far : s;
    cudaStream_t sn = mode == 2 ? h->s_far : s;
    bool ev = h->ev_ok && !h->quiet;
    cudaEvent_t *evs = h->eve[h->n_eval % EV_RING];
    if (ev) CK(cudaEventRecord(evs[EV_E0], s));
    if (ovl) {
        CK(cudaEventRecord(h->ev_fork, s));
        CK(cudaStreamWaitEvent(h->s_far, h->ev_fork, 0));
        // near field only; L2P after the join
        if (ev) CK(cudaEventRecord(evs[EV_P2P0], sn));
        if (sizeof(real) == 4 && p2p_symmetric())
            launch_p2p_sym(L, P<int>(h->leaf_start), h->near_nl, h->near_leaf, P<Geom>(h->geomd),
                           P<float4>(h->A), P<float2>(h->B), P<float4>(h->H), h->N, sn);
        else
            launch_p2p<real>(p, KP, L, P<int>(h->leaf_start), h->near_nl, h->near_leaf,
                             P<Geom>(h->geomd), P<R4>(h->A), P<R2>(h->B), nullptr, P<R4>(h->H), sn);
        if (ev) CK(cudaEventRecord(evs[EV_P2P1], sn));
    }
    // far chain
    CK(cudaMemsetAsync(h->V.p, 0, sizeof(double) * (size_t)ncellp * KP, sf));
    launch_p2m<real>(p, KP, L, P<int>(h->leaf_start), P<R4>(h->A), P<R2>(h->B), P<real>(h->Q), sf);
    if (ev) CK(cudaEventRecord(evs[EV_P2M], sf));
    launch_m2m_all<real>(p, KP, L, P<Geom>(h->geomd), P<real>(h->Q), sf);
    if (ev) CK(cudaEventRecord(evs[EV_M2M], sf));
    if (tc)
        launch_m2l_tc(p, KP, P<Tile>(h->tiles), h->ntiles, P<M2LItem>(h->items), h->nitems,
                      P<int>(h->titem0), P<int>(h->tnitems), P<int>(h->ent_u), P<int>(h->ent_src),
                      P<float>(h->Q), ncellp, P<float>(h->gkt), P<float>(h->Qs),
                      (tc_gather_tma() && h->qmap_ok && h->qmap_for == h->Qs.p) ? h->qmap : nullptr,
                      tc_a_tmem(), P<float>(h->Bop), P<Geom>(h->geomd), P<float>(h->Ps), P<double>(h->V),
                      &P<Readback>(h->rb)->eflags, sf);
    else if (sizeof(real) == 4 && m2l_f32_supported(KP, h->ldD))
        launch_m2l_f32(p, KP, P<Tile>(h->tiles), h->ntiles, P<M2LItem>(h->items), h->nitems,
                       P<int>(h->titem0), P<int>(h->tnitems), P<int>(h->ent_u), P<int>(h->ent_src),
                       P<float>(h->Q), P<float>(h->D), h->ldD, P<uint16_t>(h->itab), h->maxdeg,
                       P<Geom>(h->geomd), P<float>(h->Ps), P<double>(h->V), sf);
    else
        launch_m2l<real>(p, KP, P<Tile>(h->tiles), h->ntiles, P<int>(h->ent_u), P<int>(h->ent_src),
                         P<real>(h->Q), P<real>(h->D), h->ldD, P<uint16_t>(h->itab), h->maxdeg,
                         P<Geom>(h->geomd), P<double>(h->V), sf);
    if (ev) CK(cudaEventRecord(evs[EV_M2L], sf));
    launch_l2l_all(p, KP, L, P<Geom>(h->geomd), P<int>(h->leaf_start), P<double>(h->V), sf);
    if (ev) CK(cudaEventRecord(evs[EV_L2L], sf));
    if (ovl) {
        CK(cudaEventRecord(h->ev_join, h->s_far));
        CK(cudaStreamWaitEvent(s, h->ev_join, 0));
        if (ev) CK(cudaEventRecord(evs[EV_JOIN], s));
        launch_l2p<real>(p, KP, L, P<int>(h->leaf_start), P<R4>(h->A), P<double>(h->V),
                         P<R4>(h->H), s);
    } else {
        if (ev) CK(cudaEventRecord(evs[EV_P2P0], s));
        const bool sym = sizeof(real) == 4 && p2p_symmetric();
        if (sym)
            launch_p2p_sym(L, P<int>(h->leaf_start), h->near_nl, h->near_leaf, P<Geom>(h->geomd),
                           P<float4>(h->A), P<float2>(h->B), P<float4>(h->H), h->N, s);
        else
            launch_p2p<real>(p, KP, L, P<int>(h->leaf_start), h->near_nl, h->near_leaf,
                             P<Geom>(h->geomd), P<R4>(h->A), P<R2>(h->B), P<double>(h->V),
                             P<R4>(h->H), s);
        if (ev) CK(cudaEventRecord(evs[EV_P2P1], s));
        if (ev) CK(cudaEventRecord(evs[EV_JOIN], s));
        if (sym)
            launch_l2p<real>(p, KP, L, P<int>(h->leaf_start), P<R4>(h->A), P<double>(h->V),
                             P<R4>(h->H), s);
    }
    if (ev) CK(cudaEventRecord(evs[EV_L2P], s));
    Readback *drb = P<Readback>(h->rb);
    launch_finish<real>(P<R4>(h->H), P<int>(h->idx), h->mom_energy ? h->mom_energy : P<double>(h->mom),
                        h->N, Hdev, P<double>(h->epart), h->E_dst ? h->E_dst : &drb->E, s);
    if (ev) CK(cudaEventRecord(evs[EV_FIN], s));
    KCHECK();
    h->evaluated = true;
    if (ev) h->n_eval++;
    return CCFMM_OK;
}

static ccfmm_status evaluate(ccfmm_t h, double *H_out)
{
    if (!h->built) return fail(CCFMM_ERR_STATE, "handle has no tree");
    double *Hdev = nullptr;
    bool host_out = false;
    if (H_out) {
        if (is_device_ptr(H_out)) {
            Hdev = H_out;
        } else {
            TRY(ensure(h->Hout, sizeof(double) * 3 * h->N));
            Hdev = P<double>(h->Hout);
            host_out = true;
        }
    }
    if (h->prec == CCFMM_MIXED)
        TRY(eval_t<float>(h, Hdev));
    else
        TRY(eval_t<double>(h, Hdev));
    if (host_out) {
        CK(cudaMemcpyAsync(H_out, Hdev, sizeof(double) * 3 * h->N, cudaMemcpyDeviceToHost, h->stream));
        CK(cudaMemcpyAsync(&h->hrb->flags, &P<Readback>(h->rb)->flags, sizeof(int),
                           cudaMemcpyDeviceToHost, h->stream));
        CK(cudaMemcpyAsync(&h->hrb->eflags, &P<Readback>(h->rb)->eflags, sizeof(int),
                           cudaMemcpyDeviceToHost, h->stream));
        CK(cudaStreamSynchronize(h->stream));
        if (h->hrb->eflags) {
            CK(cudaMemsetAsync(&P<Readback>(h->rb)->eflags, 0, sizeof(int), h->stream));
            CK(cudaStreamSynchronize(h->stream));
            TRY(check_flags(h, h->hrb->eflags));
        }
        TRY(check_flags(h, h->hrb->flags));
    }
    return CCFMM_OK;
}

// ------------------------------------------------------------ C-ABI
extern "C" {

const char *ccfmm_last_error(void) { return g_err.c_str(); }

int64_t ccfmm_kernel_launches(void) { return (int64_t)g_launches.load(); }

// member: the handle belongs to an ensemble (set before its first build)
static ccfmm_status create_handle(const double *positions, const double *moments, int64_t N,
                                  int p, double theta, double leaf_size, const double *box,
                                  ccfmm_prec prec, void *stream, bool member, ccfmm_t *out,
                                  int item_len = M2L_EC)
{
    g_err.clear();
    if (!out) return fail(CCFMM_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (!positions || !moments) return fail(CCFMM_ERR_ARG, "positions or moments is NULL");
    if (N < 1 || N >= (1ll << 31) - 1) return fail(CCFMM_ERR_ARG, "N = %lld out of range", (long long)N);
    if (p < 1 || p > PMAX) return fail(CCFMM_ERR_ARG, "p = %d out of range 1..%d", p, PMAX);
    if (!(theta > 0.0 && theta < 1.0)) return fail(CCFMM_ERR_ARG, "theta = %g not in (0, 1)", theta);
    if (leaf_size != leaf_size || (leaf_size > 0.0 && leaf_size < 1.0) || isinf(leaf_size))
        return fail(CCFMM_ERR_ARG, "leaf_size = %g invalid", leaf_size);
    if (prec != CCFMM_FP64 && prec != CCFMM_MIXED) return fail(CCFMM_ERR_ARG, "bad precision");
    if (box) {
        for (int a = 0; a < 3; ++a)
            if (!(isfinite(box[a]) && isfinite(box[3 + a]) && box[a] < box[3 + a]))
                return fail(CCFMM_ERR_ARG, "box must have finite lo < hi");
    }
    ccfmm_t h = new (std::nothrow) ccfmm_s();
    if (!h) return fail(CCFMM_ERR_ALLOC, "host allocation failed");
    cudaError_t e = cudaGetDevice(&h->device);
    if (e != cudaSuccess) {
        cudaGetLastError();
        delete h;
        return fail(CCFMM_ERR_CUDA, "no CUDA device: %s", cudaGetErrorString(e));
    }
    h->stream = (cudaStream_t)stream;
    h->quiet = member;
    h->N = N;
    h->p = p;
    h->theta = theta;
    h->leaf_req = leaf_size;
    h->leaf_target = leaf_size > 0.0 ? leaf_size : ccfmm_leaf_size_rule(p);
    h->prec = prec;
    h->rsz = prec == CCFMM_MIXED ? 4 : 8;
    h->K = nterms(p) - 1;
    h->KP = padded_k(p);
    h->maxdeg = 2 * p;
    h->item_len = item_len > 0 ? item_len : M2L_EC;
    if (box) {
        h->has_box = true;
        memcpy(h->box_user, box, sizeof(h->box_user));
    }
    if (cudaMallocHost((void **)&h->hrb, sizeof(Readback)) != cudaSuccess) {
        cudaGetLastError();
        delete h;
        return fail(CCFMM_ERR_ALLOC, "pinned host allocation failed");
    }
    h->ev_ok = true;
    for (int i = 0; i < EV_NB; ++i)
        if (cudaEventCreate(&h->evb[i]) != cudaSuccess) h->ev_ok = false;
    for (int r = 0; r < EV_RING; ++r)
        for (int i = 0; i < EV_NE; ++i)
            if (cudaEventCreate(&h->eve[r][i]) != cudaSuccess) h->ev_ok = false;
    cudaGetLastError();
    ccfmm_status st = build(h, positions, moments);
    if (st != CCFMM_OK) {
        std::string msg = g_err;
        fmm_destroy(h);
        g_err = msg;
        return st;
    }
    *out = h;
    return CCFMM_OK;
}

ccfmm_status fmm_create_ex(const double *positions, const double *moments, int64_t N, int p,
                           double theta, double leaf_size, const double *box, ccfmm_prec prec,
                           void *stream, ccfmm_t *out)
{
    return create_handle(positions, moments, N, p, theta, leaf_size, box, prec, stream, false,
                         out);
}

ccfmm_status fmm_create(const double *positions, const double *moments, int64_t N, int p,
                        double theta, double leaf_size, ccfmm_t *out)
{
    return fmm_create_ex(positions, moments, N, p, theta, leaf_size, nullptr, CCFMM_MIXED, nullptr,
                         out);
}

ccfmm_status fmm_set_positions(ccfmm_t h, const double *positions, const double *moments)
{
    g_err.clear();
    if (!h) return fail(CCFMM_ERR_ARG, "handle is NULL");
    if (!positions || !moments) return fail(CCFMM_ERR_ARG, "positions or moments is NULL");
    CK(cudaSetDevice(h->device));
    return build(h, positions, moments);
}

ccfmm_status fmm_set_moments(ccfmm_t h, const double *moments)
{
    g_err.clear();
    if (!h) return fail(CCFMM_ERR_ARG, "handle is NULL");
    if (!moments) return fail(CCFMM_ERR_ARG, "moments is NULL");
    if (!h->built) return fail(CCFMM_ERR_STATE, "handle has no tree");
    CK(cudaSetDevice(h->device));
    TRY(copy_in(h, h->mom, moments, 3 * h->N));
    Readback *drb = P<Readback>(h->rb);
    CK(cudaMemsetAsync(&drb->flags, 0, sizeof(int), h->stream));
    launch_check_finite(P<double>(h->mom), 3 * h->N, &drb->flags, h->stream);
    if (h->prec == CCFMM_MIXED)
        launch_permute_moments<float>(P<double>(h->mom), P<int>(h->idx), h->N, P<float4>(h->A),
                                      P<float2>(h->B), h->stream);
    else
        launch_permute_moments<double>(P<double>(h->mom), P<int>(h->idx), h->N, P<double4>(h->A),
                                       P<double2>(h->B), h->stream);
    KCHECK();
    int flags = 0;
    CK(cudaMemcpyAsync(&h->hrb->flags, &drb->flags, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    flags = h->hrb->flags;
    h->evaluated = false;
    return check_flags(h, flags);
}

ccfmm_status fmm_set_truncation(ccfmm_t h, int max_degree)
{
    g_err.clear();
    if (!h) return fail(CCFMM_ERR_ARG, "handle is NULL");
    if (h->quiet) return fail(CCFMM_ERR_STATE, "ensemble members keep the square truncation");
    const int bound = max_degree <= 0 ? 2 * h->p : max_degree;
    if (bound < 2 || bound > 2 * h->p)
        return fail(CCFMM_ERR_ARG, "max_degree = %d outside 2..%d", max_degree, 2 * h->p);
    if (bound == h->maxdeg) return CCFMM_OK;
    CK(cudaSetDevice(h->device));
    h->maxdeg = bound;
    if (h->ftable_ready) {
        launch_itable(h->p, h->KP, h->maxdeg, P<uint16_t>(h->itab), h->stream);
        KCHECK();
    }
    h->tc_ops_ready = false;  // the tensor-core operators read the index table
    h->evaluated = false;
    return CCFMM_OK;
}

ccfmm_status fmm_get_truncation(ccfmm_t h, int *max_degree)
{
    g_err.clear();
    if (!h || !max_degree) return fail(CCFMM_ERR_ARG, "handle or output is NULL");
    *max_degree = h->maxdeg;
    return CCFMM_OK;
}

ccfmm_status fmm_field(ccfmm_t h, double *H_out)
{
    g_err.clear();
    if (!h) return fail(CCFMM_ERR_ARG, "handle is NULL");
    CK(cudaSetDevice(h->device));
    return evaluate(h, H_out);
}

ccfmm_status fmm_field_energy(ccfmm_t h, double *H_out, double *E_out)
{
    g_err.clear();
    if (!h) return fail(CCFMM_ERR_ARG, "handle is NULL");
    if (!E_out) return fail(CCFMM_ERR_ARG, "E_out is NULL");
    CK(cudaSetDevice(h->device));
    TRY(evaluate(h, H_out));
    Readback *drb = P<Readback>(h->rb);
    CK(cudaMemcpyAsync(&h->hrb->E, &drb->E, sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    *E_out = h->hrb->E;
    return CCFMM_OK;
}

ccfmm_status fmm_energy(ccfmm_t h, double *E_out) { return fmm_field_energy(h, nullptr, E_out); }

ccfmm_status fmm_stats(ccfmm_t h, ccfmm_stats *out)
{
    g_err.clear();
    if (!h || !out) return fail(CCFMM_ERR_ARG, "NULL argument");
    CK(cudaSetDevice(h->device));
    Readback *drb = P<Readback>(h->rb);
    if (h->built && !h->pairs_counted) {
        CK(cudaMemsetAsync(&drb->pairs, 0, sizeof(unsigned long long), h->stream));
        launch_p2p_pair_count(h->L, P<int>(h->leaf_start), h->near_nl, h->near_leaf,
                              &drb->pairs, h->stream);
        CK(cudaMemcpyAsync(&h->hrb->pairs, &drb->pairs, sizeof(unsigned long long),
                           cudaMemcpyDeviceToHost, h->stream));
        CK(cudaStreamSynchronize(h->stream));
        h->pairs = (long long)h->hrb->pairs;
        h->pairs_counted = true;
    }
    CK(cudaStreamSynchronize(h->stream));
    ccfmm_stats st;
    memset(&st, 0, sizeof(st));
    st.depth = h->L;
    st.depth_capped = h->capped ? 1 : 0;
    st.p = h->p;
    st.precision = (int)h->prec;
    st.theta = h->theta;
    st.leaf_target = h->leaf_target;
    for (int a = 0; a < 3; ++a) {
        st.box[a] = h->geom.lo[a];
        st.box[3 + a] = h->geom.lo[a] + h->geom.ext[a];
        st.leaf_width[a] = h->geom.w[h->L][a];
    }
    st.n = h->N;
    st.nonempty_leaves = h->hrb->ne[h->L];
    st.near_leaf_pairs = h->near_leaf_total;
    st.far_pairs = h->far_total;
    st.p2p_pairs = h->built ? (int64_t)h->pairs : 0;
    st.m2l_tile_entries = h->ent_total;
    st.far_offsets = h->n_d;
    if (h->ev_ok) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, h->evb[EV_B0], h->evb[EV_B1]) == cudaSuccess) st.ms_build = ms;
        const int marks[6] = {EV_B0, EV_BS1, EV_BS2, EV_BS3, EV_BS4, EV_B1};
        for (int i = 0; i < 5; ++i)
            if (cudaEventElapsedTime(&ms, h->evb[marks[i]], h->evb[marks[i + 1]]) == cudaSuccess)
                st.ms_build_stage[i] = ms;
        st.ms_build_stage[5] = h->ms_plan_host;
        // mean over the evaluations since the last fmm_reset_stats (at most
        // the last EV_RING of them)
        long long n = std::min<long long>(h->n_eval - h->n_eval_reset, EV_RING);
        for (long long j = 0; j < n; ++j) {
            cudaEvent_t *e = h->eve[(h->n_eval - 1 - j) % EV_RING];
            if (cudaEventElapsedTime(&ms, e[EV_E0], e[EV_FIN]) == cudaSuccess) st.ms_eval += ms / n;
            // p2m, m2m, m2l, l2l (far chain), l2p, p2p (near field), finish
            const int from[7] = {EV_E0, EV_P2M, EV_M2M, EV_M2L, EV_JOIN, EV_P2P0, EV_L2P};
            const int to[7] = {EV_P2M, EV_M2M, EV_M2L, EV_L2L, EV_L2P, EV_P2P1, EV_FIN};
            for (int i = 0; i < 7; ++i)
                if (cudaEventElapsedTime(&ms, e[from[i]], e[to[i]]) == cudaSuccess)
                    st.ms_stage[i] += ms / n;
        }
        st.ms_stage[7] = (double)n;
        cudaGetLastError();
    }
    *out = st;
    return CCFMM_OK;
}

ccfmm_status fmm_reset_stats(ccfmm_t h)
{
    g_err.clear();
    if (!h) return fail(CCFMM_ERR_ARG, "handle is NULL");
    h->n_eval_reset = h->n_eval;
    return CCFMM_OK;
}

void fmm_destroy(ccfmm_t h)
{
    if (!h) return;
    cudaSetDevice(h->device);
    if (h->stream) cudaStreamSynchronize(h->stream);
    else cudaDeviceSynchronize();
    DevBuf *bufs[] = {&h->pos, &h->mom, &h->keys, &h->keys2, &h->keys3, &h->idx, &h->idx2,
                      &h->idx3, &h->sorttemp, &h->scantemp, &h->geomd, &h->box6, &h->userbox,
                      &h->partial, &h->rb, &h->leaf_start, &h->A, &h->B, &h->H, &h->cube,
                      &h->nl, &h->neA, &h->neB, &h->cflag, &h->crank, &h->oflag, &h->orank,
                      &h->tkeys, &h->tseg,
                      &h->far, &h->far_off, &h->far_num, &h->tiles, &h->tcount, &h->tstart, &h->tbm, &h->twp,
                      &h->ent_u, &h->ent_src, &h->offs, &h->fst, &h->fq, &h->fval, &h->fdense,
                      &h->D, &h->itab, &h->Q, &h->V, &h->Hout, &h->epart, &h->items,
                      &h->titem0, &h->tnitems, &h->Ps, &h->Qs, &h->Bop, &h->gkt, &h->dmap,
                      &h->dsep};
    for (DevBuf *b : bufs)
        if (b->p) cudaFree(b->p);
    if (h->hrb) cudaFreeHost(h->hrb);
    if (h->s_far) {
        cudaStreamSynchronize(h->s_far);
        cudaStreamDestroy(h->s_far);
    }
    if (h->ev_fork) cudaEventDestroy(h->ev_fork);
    if (h->ev_join) cudaEventDestroy(h->ev_join);
    if (h->ev_ok) {
        for (int i = 0; i < EV_NB; ++i) cudaEventDestroy(h->evb[i]);
        for (int r = 0; r < EV_RING; ++r)
            for (int i = 0; i < EV_NE; ++i) cudaEventDestroy(h->eve[r][i]);
    }
    cudaGetLastError();
    delete h;
}

// ------------------------------------------------------------ inspection
ccfmm_status fmm_get_axes(ccfmm_t h, int32_t *axes)
{
    g_err.clear();
    if (!h || !axes) return fail(CCFMM_ERR_ARG, "NULL argument");
    for (int l = 1; l <= h->L; ++l) axes[l - 1] = h->geom.axis[l];
    return CCFMM_OK;
}

ccfmm_status fmm_get_leaf_of(ccfmm_t h, int64_t *leaf_of)
{
    g_err.clear();
    if (!h || !leaf_of) return fail(CCFMM_ERR_ARG, "NULL argument");
    if (!h->leaf_perm_valid) return fail(CCFMM_ERR_STATE, "no tree");
    CK(cudaSetDevice(h->device));
    std::vector<uint32_t> k(h->N);
    std::vector<int> perm(h->N);
    CK(cudaStreamSynchronize(h->stream));
    CK(cudaMemcpy(k.data(), h->keys2.p, sizeof(uint32_t) * h->N, cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(perm.data(), h->idx.p, sizeof(int) * h->N, cudaMemcpyDeviceToHost));
    for (long long s = 0; s < h->N; ++s) leaf_of[perm[s]] = (int64_t)(k[s] >> (LCAP - h->L));
    return CCFMM_OK;
}

ccfmm_status fmm_get_pairs(ccfmm_t h, int kind, int64_t *pairs, int64_t capacity, int64_t *count)
{
    g_err.clear();
    if (!h || !count) return fail(CCFMM_ERR_ARG, "NULL argument");
    if (!h->built) return fail(CCFMM_ERR_STATE, "no tree");
    CK(cudaSetDevice(h->device));
    CK(cudaStreamSynchronize(h->stream));
    const int L = h->L;
    std::vector<int64_t> out;
    if (kind == 0) {
        long long nleaf = 1ll << L;
        std::vector<int2> nl(nleaf);
        CK(cudaMemcpy(nl.data(), h->near_nl, sizeof(int2) * nleaf, cudaMemcpyDeviceToHost));
        std::vector<NearEnt> ent(h->near_leaf_bytes / sizeof(NearEnt));
        CK(cudaMemcpy(ent.data(), h->near_leaf, h->near_leaf_bytes, cudaMemcpyDeviceToHost));
        for (long long k = 0; k < nleaf; ++k)
            for (int e = nl[k].x; e < nl[k].x + nl[k].y; ++e) {
                out.push_back(nleaf + k);
                out.push_back(nleaf + ent[e].src);
            }
    } else if (kind == 1) {
        long long ncellp = 1ll << (L + 1);
        std::vector<int> off(ncellp), num(ncellp);
        CK(cudaMemcpy(off.data(), h->far_off.p, sizeof(int) * ncellp, cudaMemcpyDeviceToHost));
        CK(cudaMemcpy(num.data(), h->far_num.p, sizeof(int) * ncellp, cudaMemcpyDeviceToHost));
        size_t nfar = h->far.bytes / sizeof(FarEnt);
        std::vector<FarEnt> far(nfar);
        CK(cudaMemcpy(far.data(), h->far.p, sizeof(FarEnt) * nfar, cudaMemcpyDeviceToHost));
        for (long long hid = 1; hid < ncellp; ++hid) {
            int l = 63 - __builtin_clzll((unsigned long long)hid);
            for (int e = 0; e < num[hid]; ++e) {
                out.push_back(hid);
                out.push_back((1ll << l) + far[off[hid] + e].src);
            }
        }
    } else {
        return fail(CCFMM_ERR_ARG, "kind must be 0 (near) or 1 (far)");
    }
    *count = (int64_t)(out.size() / 2);
    if (pairs && capacity >= *count) memcpy(pairs, out.data(), sizeof(int64_t) * out.size());
    return CCFMM_OK;
}

ccfmm_status fmm_get_m2l_data(ccfmm_t h, int64_t *sizes, double *D_out, int32_t *ent_u_out,
                              int32_t *ent_src_out, int32_t *tiles_out)
{
    g_err.clear();
    if (!h || !sizes) return fail(CCFMM_ERR_ARG, "NULL argument");
    if (!h->built) return fail(CCFMM_ERR_STATE, "no tree");
    CK(cudaSetDevice(h->device));
    CK(cudaStreamSynchronize(h->stream));
    sizes[0] = h->n_d;
    sizes[1] = h->TD;
    sizes[2] = h->ent_total;
    sizes[3] = h->ntiles;
    if (D_out && h->n_d > 0) {
        size_t n = (size_t)h->n_d * h->ldD;
        std::vector<double> d(n);
        if (h->prec == CCFMM_MIXED) {
            std::vector<float> f(n);
            CK(cudaMemcpy(f.data(), h->D.p, sizeof(float) * n, cudaMemcpyDeviceToHost));
            for (size_t i = 0; i < n; ++i) d[i] = f[i];
        } else {
            CK(cudaMemcpy(d.data(), h->D.p, sizeof(double) * n, cudaMemcpyDeviceToHost));
        }
        for (int r = 0; r < h->n_d; ++r)
            for (int t = 0; t < h->TD; ++t) D_out[(size_t)r * h->TD + t] = d[(size_t)r * h->ldD + t];
    }
    if (ent_u_out && h->ent_total > 0)
        CK(cudaMemcpy(ent_u_out, h->ent_u.p, sizeof(int) * h->ent_total, cudaMemcpyDeviceToHost));
    if (ent_src_out && h->ent_total > 0)
        CK(cudaMemcpy(ent_src_out, h->ent_src.p, sizeof(int) * TT * h->ent_total,
                      cudaMemcpyDeviceToHost));
    if (tiles_out && h->ntiles > 0) {
        std::vector<Tile> t(h->ntiles);
        CK(cudaMemcpy(t.data(), h->tiles.p, sizeof(Tile) * h->ntiles, cudaMemcpyDeviceToHost));
        for (int i = 0; i < h->ntiles; ++i) {
            const int v[8] = {t[i].level, t[i].first, t[i].parity, t[i].nt,
                              t[i].ent_start, t[i].ent_count, t[i].nbits, t[i].gid_base};
            memcpy(tiles_out + 8 * (size_t)i, v, sizeof(v));
        }
    }
    return CCFMM_OK;
}

ccfmm_status ccfmm_multi_indices(int order, int32_t *out)
{
    g_err.clear();
    if (!out || order < 0 || order > 2 * PMAX) return fail(CCFMM_ERR_ARG, "bad argument");
    for (int t = 0; t < nterms(order); ++t) {
        int x, y, z;
        midx_inv(t, x, y, z);
        out[3 * t] = x;
        out[3 * t + 1] = y;
        out[3 * t + 2] = z;
    }
    return CCFMM_OK;
}

ccfmm_status fmm_get_expansions(ccfmm_t h, int kind, double *out)
{
    g_err.clear();
    if (!h || !out) return fail(CCFMM_ERR_ARG, "NULL argument");
    if (!h->evaluated) return fail(CCFMM_ERR_STATE, "no evaluation yet");
    CK(cudaSetDevice(h->device));
    CK(cudaStreamSynchronize(h->stream));
    long long ncellp = 1ll << (h->L + 1);
    int T = nterms(h->p), KP = h->KP, K = h->K;
    std::vector<double> rows((size_t)ncellp * KP);
    if (kind == 0) {
        if (h->prec == CCFMM_MIXED) {
            std::vector<float> f((size_t)ncellp * KP);
            CK(cudaMemcpy(f.data(), h->Q.p, sizeof(float) * f.size(), cudaMemcpyDeviceToHost));
            for (size_t i = 0; i < f.size(); ++i) rows[i] = f[i];
        } else {
            CK(cudaMemcpy(rows.data(), h->Q.p, sizeof(double) * rows.size(), cudaMemcpyDeviceToHost));
        }
    } else if (kind == 1) {
        CK(cudaMemcpy(rows.data(), h->V.p, sizeof(double) * rows.size(), cudaMemcpyDeviceToHost));
    } else {
        return fail(CCFMM_ERR_ARG, "kind must be 0 (Q) or 1 (V)");
    }
    for (long long r = 0; r < ncellp; ++r) {
        out[r * T] = 0.0;
        for (int c = 0; c < K; ++c) out[r * T + c + 1] = r ? rows[r * KP + c] : 0.0;
    }
    return CCFMM_OK;
}

ccfmm_status ccfmm_direct_field(const double *positions, const double *moments, int64_t N,
                                const int64_t *tgt, int64_t nt, double *H_out, void *stream)
{
    g_err.clear();
    if (!positions || !moments || !H_out) return fail(CCFMM_ERR_ARG, "NULL argument");
    if (N < 1) return fail(CCFMM_ERR_ARG, "N < 1");
    if (!tgt) nt = N;
    if (nt < 1) return fail(CCFMM_ERR_ARG, "nt < 1");
    cudaStream_t s = (cudaStream_t)stream;
    DevBuf pos, mom, tg, out;
    const double *dp = positions, *dm = moments;
    const long long *dt = nullptr;
    double *dout = H_out;
    ccfmm_status st = CCFMM_OK;
    auto cleanup = [&]() {
        cudaFree(pos.p);
        cudaFree(mom.p);
        cudaFree(tg.p);
        cudaFree(out.p);
    };
#define DTRY(x)                                                                                  \
    do {                                                                                         \
        st = (x);                                                                                \
        if (st != CCFMM_OK) {                                                                    \
            cleanup();                                                                           \
            return st;                                                                           \
        }                                                                                        \
    } while (0)
#define DCK(call)                                                                                \
    do {                                                                                         \
        cudaError_t e_ = (call);                                                                 \
        if (e_ != cudaSuccess) {                                                                 \
            cudaGetLastError();                                                                  \
            cleanup();                                                                           \
            return fail(CCFMM_ERR_CUDA, "%s: %s", #call, cudaGetErrorString(e_));               \
        }                                                                                        \
    } while (0)
    if (!is_device_ptr(positions)) {
        DTRY(ensure(pos, sizeof(double) * 3 * N));
        DCK(cudaMemcpyAsync(pos.p, positions, sizeof(double) * 3 * N, cudaMemcpyHostToDevice, s));
        dp = P<double>(pos);
    }
    if (!is_device_ptr(moments)) {
        DTRY(ensure(mom, sizeof(double) * 3 * N));
        DCK(cudaMemcpyAsync(mom.p, moments, sizeof(double) * 3 * N, cudaMemcpyHostToDevice, s));
        dm = P<double>(mom);
    }
    if (tgt) {
        if (!is_device_ptr(tgt)) {
            DTRY(ensure(tg, sizeof(long long) * nt));
            DCK(cudaMemcpyAsync(tg.p, tgt, sizeof(long long) * nt, cudaMemcpyHostToDevice, s));
            dt = P<long long>(tg);
        } else {
            dt = reinterpret_cast<const long long *>(tgt);
        }
    }
    bool host_out = !is_device_ptr(H_out);
    if (host_out) {
        DTRY(ensure(out, sizeof(double) * 3 * nt));
        dout = P<double>(out);
    }
    launch_direct(dp, dm, N, dt, nt, dout, s);
    DCK(cudaGetLastError());
    if (host_out)
        DCK(cudaMemcpyAsync(H_out, dout, sizeof(double) * 3 * nt, cudaMemcpyDeviceToHost, s));
    DCK(cudaStreamSynchronize(s));
    cleanup();
#undef DTRY
#undef DCK
    return CCFMM_OK;
}

}  // extern "C"

// ------------------------------------------------------------ ensemble
// A batch of independent samples: one handle (tree, lists, buffers) per
// sample, built once; a step turns every moment (k_rotate) and evaluates
// every sample.  The whole step is one CUDA graph launch: the rotation, then
// the samples' evaluations on BR parallel branches (samples s, s+BR, ... on
// branch s % BR).
struct ccfmm_batch_s {
    int device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    int ns = 0, nbr = 0;
    std::vector<long long> off;
    long long total = 0;
    ccfmm_prec prec = CCFMM_MIXED;
    std::vector<ccfmm_t> h;
    std::vector<cudaStream_t> br;
    std::vector<cudaEvent_t> evj;
    cudaEvent_t evf = nullptr;
    DevBuf mom, H, E, prm;
    RotateParams *hprm = nullptr;  // pinned
    cudaGraphExec_t exec[2] = {nullptr, nullptr};  // [0] evaluate, [1] rotate + evaluate
    long long graph_kernels[2] = {0, 0};
    // batched stages: one launch per stage for every member (FP32 path with
    // the tensor-core M2L); the per-member graph otherwise
    struct Stage {
        DevBuf args, bstart;
        int nblocks = 0;
    };
    bool batched = false, planned = false;
    Stage st_perm, st_p2m, st_qs, st_m2l, st_red, st_p2p, st_l2p, st_fin;
    cudaEvent_t ev_near0 = nullptr, ev_near1 = nullptr;  // near field on a second branch
    cudaStream_t s_hi = nullptr;  // the far chain, at the highest stream priority
    cudaEvent_t ev_far1 = nullptr;
    std::vector<Stage> st_m2m, st_l2l;
    DevBuf eflag;  // raised by the batched tensor-core M2L's bounded waits
    int *heflag = nullptr;
    bool tuned = false;
    std::vector<struct TuneClass> tune;
    std::vector<int> tune_of;
};

// batched stages are used when every member runs the FP32 path with the
// tensor-core M2L (CCFMM_BATCH_MODE=graph keeps the per-member graph)
static bool batch_can_batch(ccfmm_batch_t b)
{
    const char *e = getenv("CCFMM_BATCH_MODE");
    if (e && !strcmp(e, "graph")) return false;
    for (ccfmm_t hs : b->h)
        if (hs->prec != CCFMM_MIXED || !m2l_use_tc(hs)) return false;
    return true;
}

template <typename A>
static ccfmm_status stage_upload(ccfmm_batch_s::Stage &st, const std::vector<A> &args,
                                 const std::vector<int> &blocks)
{
    std::vector<int> bs(blocks.size() + 1, 0);
    for (size_t m = 0; m < blocks.size(); ++m) bs[m + 1] = bs[m] + blocks[m];
    st.nblocks = bs.back();
    TRY(ensure(st.args, sizeof(A) * std::max<size_t>(args.size(), 1)));
    TRY(ensure(st.bstart, sizeof(int) * bs.size()));
    CK(cudaMemcpy(st.args.p, args.data(), sizeof(A) * args.size(), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(st.bstart.p, bs.data(), sizeof(int) * bs.size(), cudaMemcpyHostToDevice));
    return CCFMM_OK;
}

// Arguments of every batched stage, from the members' buffers (built once;
// the members' trees and operators are fixed for the batch's life).
static ccfmm_status batch_plan(ccfmm_batch_t b)
{
    const int nm = b->ns;
    TRY(ensure(b->eflag, sizeof(int)));
    CK(cudaMemset(b->eflag.p, 0, sizeof(int)));
    std::vector<PermuteArgs> a_perm(nm);
    std::vector<P2MArgs> a_p2m(nm);
    std::vector<QSplitArgs> a_qs(nm);
    std::vector<M2LTCArgs> a_m2l(nm);
    std::vector<ReduceArgs> a_red(nm);
    std::vector<P2PArgs> a_p2p(nm), a_l2p(nm);
    std::vector<int> b_l2p(nm);
    std::vector<FinishArgs> a_fin(nm);
    std::vector<int> b_perm(nm), b_p2m(nm), b_qs(nm), b_m2l(nm), b_red(nm), b_p2p(nm), b_fin(nm);
    int maxr_m2m = 0, maxr_l2l = 0;
    for (int m = 0; m < nm; ++m) {
        int l0[LCAP + 1], D[LCAP + 1];
        maxr_m2m = std::max(maxr_m2m, m2m_rounds(b->h[m]->L, l0, D));
        maxr_l2l = std::max(maxr_l2l, l2l_rounds(b->h[m]->L, l0, D));
    }
    std::vector<std::vector<M2MArgs>> a_m2m(maxr_m2m, std::vector<M2MArgs>(nm));
    std::vector<std::vector<L2LArgs>> a_l2l(maxr_l2l, std::vector<L2LArgs>(nm));
    std::vector<std::vector<int>> b_m2m(maxr_m2m, std::vector<int>(nm, 0)),
        b_l2l(maxr_l2l, std::vector<int>(nm, 0));
    for (int m = 0; m < nm; ++m) {
        ccfmm_t h = b->h[m];
        const int L = h->L, p = h->p, KP = h->KP;
        const long long ncellp = 1ll << (L + 1);
        const Geom *g = P<Geom>(h->geomd);
        a_perm[m] = PermuteArgs{P<double>(b->mom) + 3 * b->off[m], P<int>(h->idx), h->N,
                                P<float4>(h->A), P<float2>(h->B), P<double>(h->V), ncellp * KP};
        b_perm[m] = permute_blocks(h->N);
        a_p2m[m] = P2MArgs{p, KP, L, P<int>(h->leaf_start), P<float4>(h->A), P<float2>(h->B),
                           P<float>(h->Q)};
        b_p2m[m] = p2m_blocks(L);
        int l0[LCAP + 1], D[LCAP + 1];
        const int nr = m2m_rounds(L, l0, D);
        for (int r = 0; r < nr; ++r) {
            a_m2m[r][m] = M2MArgs{p, KP, l0[r], D[r], g, P<float>(h->Q)};
            b_m2m[r][m] = (int)(1ll << l0[r]);
        }
        a_qs[m] = QSplitArgs{p, ncellp, P<float>(h->Q), P<float>(h->gkt), P<float>(h->Qs)};
        b_qs[m] = h->nitems > 0 ? q_split_blocks(KP, ncellp) : 0;
        a_m2l[m] = M2LTCArgs{P<M2LItem>(h->items), P<int>(h->ent_u), P<int>(h->ent_src),
                             P<float>(h->Qs), ncellp * m2l_tc_kt(KP),
                             reinterpret_cast<const unsigned char *>(h->Bop.p), P<float>(h->Ps),
                             P<int>(b->eflag)};
        b_m2l[m] = h->nitems;
        a_red[m] = ReduceArgs{p, KP, P<Tile>(h->tiles), P<int>(h->titem0), P<int>(h->tnitems),
                              P<float>(h->Ps), g, P<double>(h->V)};
        b_red[m] = h->nitems > 0 ? h->ntiles : 0;
        const int nl2 = l2l_rounds(L, l0, D);
        for (int r = 0; r < nl2; ++r) {
            a_l2l[r][m] = L2LArgs{p, KP, l0[r], D[r], L, g, P<int>(h->leaf_start), P<double>(h->V)};
            b_l2l[r][m] = (int)(1ll << l0[r]);
        }
        // near field alone (it runs beside the far chain), then the smooth field
        a_p2p[m] = P2PArgs{p, KP, L, P<int>(h->leaf_start), h->near_nl, h->near_leaf, g,
                           P<float4>(h->A), P<float2>(h->B), nullptr, P<float4>(h->H)};
        b_p2p[m] = (int)(1ll << L);
        a_l2p[m] = a_p2p[m];
        a_l2p[m].V = P<double>(h->V);
        b_l2p[m] = l2p_blocks(L);
        a_fin[m] = FinishArgs{P<float4>(h->H), P<int>(h->idx), h->mom_energy, h->N,
                              P<double>(b->H) + 3 * b->off[m], P<double>(h->epart), h->E_dst};
        b_fin[m] = finish_blocks(h->N);
    }
    TRY(stage_upload(b->st_perm, a_perm, b_perm));
    TRY(stage_upload(b->st_p2m, a_p2m, b_p2m));
    b->st_m2m.assign(maxr_m2m, ccfmm_batch_s::Stage());
    for (int r = 0; r < maxr_m2m; ++r) TRY(stage_upload(b->st_m2m[r], a_m2m[r], b_m2m[r]));
    TRY(stage_upload(b->st_qs, a_qs, b_qs));
    TRY(stage_upload(b->st_m2l, a_m2l, b_m2l));
    TRY(stage_upload(b->st_red, a_red, b_red));
    b->st_l2l.assign(maxr_l2l, ccfmm_batch_s::Stage());
    for (int r = 0; r < maxr_l2l; ++r) TRY(stage_upload(b->st_l2l[r], a_l2l[r], b_l2l[r]));
    {
        // the near field takes the largest samples first (their leaves stay
        // together, in key order), so that the launch ends on small ones
        std::vector<int> ord(nm);
        for (int m = 0; m < nm; ++m) ord[m] = m;
        std::stable_sort(ord.begin(), ord.end(),
                         [&](int x, int y) { return b->h[x]->N > b->h[y]->N; });
        std::vector<P2PArgs> a2(nm);
        std::vector<int> b2(nm);
        for (int m = 0; m < nm; ++m) {
            a2[m] = a_p2p[ord[m]];
            b2[m] = b_p2p[ord[m]];
        }
        TRY(stage_upload(b->st_p2p, a2, b2));
    }
    TRY(stage_upload(b->st_l2p, a_l2p, b_l2p));
    if (!b->ev_near0) CK(cudaEventCreateWithFlags(&b->ev_near0, cudaEventDisableTiming));
    if (!b->ev_near1) CK(cudaEventCreateWithFlags(&b->ev_near1, cudaEventDisableTiming));
    if (!b->ev_far1) CK(cudaEventCreateWithFlags(&b->ev_far1, cudaEventDisableTiming));
    if (!b->s_hi) {
        int least = 0, greatest = 0;
        CK(cudaDeviceGetStreamPriorityRange(&least, &greatest));
        CK(cudaStreamCreateWithPriority(&b->s_hi, cudaStreamNonBlocking, greatest));
    }
    TRY(stage_upload(b->st_fin, a_fin, b_fin));
    b->planned = true;
    return CCFMM_OK;
}

// the batched stages of one step, in order, on the batch's stream
static void batch_enqueue(ccfmm_batch_t b, cudaStream_t s)
{
    const int nm = b->ns;
    const int KP = b->h[0]->KP, p = b->h[0]->p;
    const char *sv = getenv("CCFMM_TC_STALL");
    const int stall = (sv && atoi(sv)) ? 1 : 0;
    const long long spin = stall ? (1ll << 12) : (1ll << 22);
    auto A = [](ccfmm_batch_s::Stage &st) { return st.args.p; };
    auto B = [](ccfmm_batch_s::Stage &st) { return P<int>(st.bstart); };
    launch_permute_batch((const PermuteArgs *)A(b->st_perm), B(b->st_perm), nm, b->st_perm.nblocks, s);
    // the near field of every member on a second branch, beside the far chain
    cudaStream_t sn = b->br[0];
    cudaEventRecord(b->ev_near0, s);
    cudaStreamWaitEvent(sn, b->ev_near0, 0);
    launch_p2p_batch((const P2PArgs *)A(b->st_p2p), B(b->st_p2p), nm, b->st_p2p.nblocks, KP, sn);
    cudaEventRecord(b->ev_near1, sn);
    // the far chain on a high-priority stream: its blocks are dispatched
    // first whenever near-field blocks retire
    cudaStream_t sf = b->s_hi;
    cudaStreamWaitEvent(sf, b->ev_near0, 0);
    launch_p2m_batch((const P2MArgs *)A(b->st_p2m), B(b->st_p2m), nm, b->st_p2m.nblocks, sf);
    for (auto &st : b->st_m2m) launch_m2m_batch((const M2MArgs *)A(st), B(st), nm, st.nblocks, sf);
    launch_q_split_batch(KP, (const QSplitArgs *)A(b->st_qs), B(b->st_qs), nm, b->st_qs.nblocks, sf);
    launch_m2l_tc_batch(KP, (const M2LTCArgs *)A(b->st_m2l), B(b->st_m2l), nm, b->st_m2l.nblocks,
                        spin, stall, sf);
    launch_reduce_h_batch(p, KP, (const ReduceArgs *)A(b->st_red), B(b->st_red), nm,
                          b->st_red.nblocks, sf);
    for (auto &st : b->st_l2l) launch_l2l_batch((const L2LArgs *)A(st), B(st), nm, st.nblocks, sf);
    cudaEventRecord(b->ev_far1, sf);
    cudaStreamWaitEvent(s, b->ev_far1, 0);
    cudaStreamWaitEvent(s, b->ev_near1, 0);
    launch_l2p_batch(p, (const P2PArgs *)A(b->st_l2p), B(b->st_l2p), nm, b->st_l2p.nblocks, s);
    launch_finish_batch((const FinishArgs *)A(b->st_fin), B(b->st_fin), nm, b->st_fin.nblocks, s);
}

static ccfmm_status batch_capture(ccfmm_batch_t b, int rotate)
{
    cudaStream_t s = b->stream;
    cudaGraph_t g = nullptr;
    // allocations and one-time operator builds happen before the capture
    bool prepared = false;
    for (ccfmm_t hs : b->h)
        if (m2l_use_tc(hs)) {
            TRY(tc_prepare(hs));
            prepared = true;
        }
    if (prepared)
        for (int r = 0; r < b->nbr; ++r) CK(cudaStreamSynchronize(b->br[r]));
    if (b->batched && !b->planned) TRY(batch_plan(b));
    CK(cudaStreamBeginCapture(s, cudaStreamCaptureModeRelaxed));
    ccfmm_status st = CCFMM_OK;
    do {
        if (rotate) launch_rotate(P<double>(b->mom), b->total, P<RotateParams>(b->prm), s);
        if (b->batched) {
            batch_enqueue(b, s);
            break;
        }
        if (cudaEventRecord(b->evf, s) != cudaSuccess) { st = fail(CCFMM_ERR_CUDA, "capture fork"); break; }
        for (int r = 0; r < b->nbr; ++r)
            if (cudaStreamWaitEvent(b->br[r], b->evf, 0) != cudaSuccess) st = fail(CCFMM_ERR_CUDA, "capture wait");
        if (st != CCFMM_OK) break;
        for (int i = 0; i < b->ns && st == CCFMM_OK; ++i) {
            ccfmm_t hs = b->h[i];
            const double *ms = P<double>(b->mom) + 3 * b->off[i];
            if (hs->prec == CCFMM_MIXED) {
                launch_permute_moments<float>(ms, P<int>(hs->idx), hs->N, P<float4>(hs->A),
                                              P<float2>(hs->B), hs->stream);
                st = eval_t<float>(hs, P<double>(b->H) + 3 * b->off[i]);
            } else {
                launch_permute_moments<double>(ms, P<int>(hs->idx), hs->N, P<double4>(hs->A),
                                               P<double2>(hs->B), hs->stream);
                st = eval_t<double>(hs, P<double>(b->H) + 3 * b->off[i]);
            }
        }
        if (st != CCFMM_OK) break;
        for (int r = 0; r < b->nbr; ++r) {
            if (cudaEventRecord(b->evj[r], b->br[r]) != cudaSuccess ||
                cudaStreamWaitEvent(s, b->evj[r], 0) != cudaSuccess)
                st = fail(CCFMM_ERR_CUDA, "capture join");
        }
    } while (0);
    cudaError_t e = cudaStreamEndCapture(s, &g);
    if (st != CCFMM_OK) {
        if (g) cudaGraphDestroy(g);
        cudaGetLastError();
        return st;
    }
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(CCFMM_ERR_CUDA, "stream capture failed: %s", cudaGetErrorString(e));
    }
    size_t nn = 0;
    CK(cudaGraphGetNodes(g, nullptr, &nn));
    std::vector<cudaGraphNode_t> nodes(nn);
    CK(cudaGraphGetNodes(g, nodes.data(), &nn));
    long long nk = 0;
    for (size_t i = 0; i < nn; ++i) {
        cudaGraphNodeType ty;
        if (cudaGraphNodeGetType(nodes[i], &ty) == cudaSuccess && ty == cudaGraphNodeTypeKernel) ++nk;
    }
    b->graph_kernels[rotate] = nk;
    // node priorities from the capturing streams (the far chain's is higher)
    e = cudaGraphInstantiateWithFlags(&b->exec[rotate], g, cudaGraphInstantiateFlagUseNodePriority);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
        cudaGetLastError();
        b->exec[rotate] = nullptr;
        return fail(CCFMM_ERR_CUDA, "graph instantiation failed: %s", cudaGetErrorString(e));
    }
    return CCFMM_OK;
}

// the step without a graph: the same launches issued directly on the branch
// streams (CCFMM_BATCH_NOGRAPH=1)
static ccfmm_status batch_direct(ccfmm_batch_t b, int rotate)
{
    cudaStream_t s = b->stream;
    if (rotate) launch_rotate(P<double>(b->mom), b->total, P<RotateParams>(b->prm), s);
    if (b->batched) {
        if (!b->planned) {
            for (ccfmm_t hs : b->h) TRY(tc_prepare(hs));
            for (int r = 0; r < b->nbr; ++r) CK(cudaStreamSynchronize(b->br[r]));
            TRY(batch_plan(b));
        }
        batch_enqueue(b, s);
        KCHECK();
        return CCFMM_OK;
    }
    CK(cudaEventRecord(b->evf, s));
    for (int r = 0; r < b->nbr; ++r) CK(cudaStreamWaitEvent(b->br[r], b->evf, 0));
    for (int i = 0; i < b->ns; ++i) {
        ccfmm_t hs = b->h[i];
        const double *ms = P<double>(b->mom) + 3 * b->off[i];
        if (hs->prec == CCFMM_MIXED) {
            launch_permute_moments<float>(ms, P<int>(hs->idx), hs->N, P<float4>(hs->A),
                                          P<float2>(hs->B), hs->stream);
            TRY(eval_t<float>(hs, P<double>(b->H) + 3 * b->off[i]));
        } else {
            launch_permute_moments<double>(ms, P<int>(hs->idx), hs->N, P<double4>(hs->A),
                                           P<double2>(hs->B), hs->stream);
            TRY(eval_t<double>(hs, P<double>(b->H) + 3 * b->off[i]));
        }
    }
    for (int r = 0; r < b->nbr; ++r) {
        CK(cudaEventRecord(b->evj[r], b->br[r]));
        CK(cudaStreamWaitEvent(s, b->evj[r], 0));
    }
    return CCFMM_OK;
}

static ccfmm_status batch_run(ccfmm_batch_t b, int rotate, double *H_out, double *E_out)
{
    const char *ng = getenv("CCFMM_BATCH_NOGRAPH");
    if (ng && atoi(ng)) {
        TRY(batch_direct(b, rotate));
    } else {
        if (!b->exec[rotate]) TRY(batch_capture(b, rotate));
        CK(cudaGraphLaunch(b->exec[rotate], b->stream));
        note_launch((int)b->graph_kernels[rotate]);
    }
    // the batched stages evaluate every member without its own eval_t
    for (ccfmm_t hs : b->h) hs->evaluated = true;
    if (H_out) {
        cudaMemcpyKind k = is_device_ptr(H_out) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
        CK(cudaMemcpyAsync(H_out, b->H.p, sizeof(double) * 3 * b->total, k, b->stream));
    }
    if (E_out) {
        cudaMemcpyKind k = is_device_ptr(E_out) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
        CK(cudaMemcpyAsync(E_out, b->E.p, sizeof(double) * b->ns, k, b->stream));
    }
    const bool sync = (H_out && !is_device_ptr(H_out)) || (E_out && !is_device_ptr(E_out));
    if (b->batched && b->eflag.p) {
        // a bounded wait that gave up in a batched launch is reported by the
        // next call that synchronises
        CK(cudaMemcpyAsync(b->heflag, b->eflag.p, sizeof(int), cudaMemcpyDeviceToHost, b->stream));
    }
    if (sync) {
        CK(cudaStreamSynchronize(b->stream));
        if (b->batched && b->eflag.p && *b->heflag) {
            CK(cudaMemset(b->eflag.p, 0, sizeof(int)));
            *b->heflag = 0;
            return fail(CCFMM_ERR_TIMEOUT, "a bounded wait in the tensor-core M2L gave up");
        }
    }
    return CCFMM_OK;
}

static ccfmm_status batch_create(const double *positions, const double *moments,
                                 const int64_t *offsets, int nsamples, int p, double theta,
                                 double leaf_size, ccfmm_prec prec, const ccfmm_batch_opts *opts,
                                 void *stream, ccfmm_batch_t *out, double leaf_all, int il_all);

extern "C" {

void fmm_batch_destroy(ccfmm_batch_t b)
{
    if (!b) return;
    cudaSetDevice(b->device);
    if (b->stream) cudaStreamSynchronize(b->stream);
    for (int r = 0; r < 2; ++r)
        if (b->exec[r]) cudaGraphExecDestroy(b->exec[r]);
    for (ccfmm_t h : b->h) fmm_destroy(h);
    for (cudaStream_t s : b->br) cudaStreamDestroy(s);
    for (cudaEvent_t e : b->evj) cudaEventDestroy(e);
    if (b->evf) cudaEventDestroy(b->evf);
    DevBuf *bufs[] = {&b->mom, &b->H, &b->E, &b->prm, &b->eflag};
    for (DevBuf *d : bufs)
        if (d->p) cudaFree(d->p);
    ccfmm_batch_s::Stage *sts[] = {&b->st_perm, &b->st_p2m, &b->st_qs, &b->st_m2l, &b->st_red,
                                   &b->st_p2p, &b->st_l2p, &b->st_fin};
    if (b->ev_near0) cudaEventDestroy(b->ev_near0);
    if (b->ev_near1) cudaEventDestroy(b->ev_near1);
    if (b->ev_far1) cudaEventDestroy(b->ev_far1);
    if (b->s_hi) cudaStreamDestroy(b->s_hi);
    for (auto *st : sts) {
        if (st->args.p) cudaFree(st->args.p);
        if (st->bstart.p) cudaFree(st->bstart.p);
    }
    for (auto *v : {&b->st_m2m, &b->st_l2l})
        for (auto &st : *v) {
            if (st.args.p) cudaFree(st.args.p);
            if (st.bstart.p) cudaFree(st.bstart.p);
        }
    if (b->heflag) cudaFreeHost(b->heflag);
    if (b->hprm) cudaFreeHost(b->hprm);
    if (b->own_stream) cudaStreamDestroy(b->stream);
    cudaGetLastError();
    delete b;
}

// ------------------------------------------------------------ autotuner
// Leaf occupancy and M2L item length per sample-size class of an ensemble,
// chosen by timed trial steps.  Classes are the octaves of N
// (floor(log2 N)).  Each class is tuned on a sub-ensemble of up to TUNE_SUB
// of its samples spread over its sizes, run the way the ensemble runs (the
// batched stages), so that what is timed is throughput, not the latency of
// one small system: for every candidate (leaf = s x {1/2, 1/sqrt2, 1,
// sqrt2, 2}, s = the requested occupancy or Eq. so; item length 32 or 64
// entries on the tensor-core path) the sub-ensemble is built, evaluated
// once untimed and `trials` times timed with CUDA events; the fastest mean
// wins.
struct TuneClass {
    int octave;
    long long nmin;
    double leaf;
    int item_len;
};
constexpr int TUNE_SUB = 16;

static ccfmm_status batch_autotune(const double *positions, const double *moments,
                                   const std::vector<long long> &off, int p, double theta,
                                   double leaf_size, ccfmm_prec prec, int trials,
                                   cudaStream_t s, std::vector<TuneClass> &classes,
                                   std::vector<int> &class_of)
{
    const int ns = (int)off.size() - 1;
    const double base = leaf_size > 0.0 ? leaf_size : ccfmm_leaf_size_rule(p);
    const double fac[5] = {0.5, 0.70710678118654752, 1.0, 1.41421356237309505, 2.0};
    std::map<int, std::vector<int>> by_oct;
    for (int i = 0; i < ns; ++i) {
        const long long n = off[i + 1] - off[i];
        int o = 0;
        while ((2ll << o) <= n) ++o;
        by_oct[o].push_back(i);
    }
    class_of.assign(ns, 0);
    classes.clear();
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    double *dpos = nullptr, *dmom = nullptr;
    ccfmm_status st = CCFMM_OK;
    for (auto &kv : by_oct) {
        std::vector<int> mem = kv.second;
        std::sort(mem.begin(), mem.end(),
                  [&](int x, int y) { return off[x + 1] - off[x] < off[y + 1] - off[y]; });
        // the sub-ensemble: samples spread evenly over the class's sizes
        std::vector<int> sub;
        const int k = std::min((int)mem.size(), TUNE_SUB);
        for (int j = 0; j < k; ++j) sub.push_back(mem[(size_t)j * mem.size() / k]);
        std::vector<int64_t> so(1, 0);
        for (int i : sub) so.push_back(so.back() + (off[i + 1] - off[i]));
        if (cudaMalloc(&dpos, sizeof(double) * 3 * so.back()) != cudaSuccess ||
            cudaMalloc(&dmom, sizeof(double) * 3 * so.back()) != cudaSuccess) {
            cudaGetLastError();
            st = fail(CCFMM_ERR_ALLOC, "autotuner: device allocation failed");
            break;
        }
        for (size_t j = 0; j < sub.size() && st == CCFMM_OK; ++j) {
            const size_t nb = sizeof(double) * 3 * (size_t)(so[j + 1] - so[j]);
            if (cudaMemcpyAsync(dpos + 3 * so[j], positions + 3 * off[sub[j]], nb, cudaMemcpyDefault, s) != cudaSuccess ||
                cudaMemcpyAsync(dmom + 3 * so[j], moments + 3 * off[sub[j]], nb, cudaMemcpyDefault, s) != cudaSuccess)
                st = fail(CCFMM_ERR_CUDA, "autotuner: copy failed");
        }
        if (st == CCFMM_OK && cudaStreamSynchronize(s) != cudaSuccess)
            st = fail(CCFMM_ERR_CUDA, "autotuner: copy failed");
        TuneClass best{kv.first, off[mem[0] + 1] - off[mem[0]], base, M2L_EC};
        double best_ms = INFINITY;
        for (int fi = 0; fi < 5 && st == CCFMM_OK; ++fi)
            for (int il : {64, 32}) {
                const double lf = std::max(1.0, base * fac[fi]);
                ccfmm_batch_t sb = nullptr;
                st = batch_create(dpos, dmom, so.data(), (int)sub.size(), p, theta, lf, prec,
                                  nullptr, s, &sb, lf, il);
                if (st != CCFMM_OK) break;
                if (!sb->batched && il != 64) {  // the item length matters to the batched M2L only
                    fmm_batch_destroy(sb);
                    continue;
                }
                st = batch_run(sb, 0, nullptr, nullptr);
                float t_ms = 0.f;
                if (st == CCFMM_OK) {
                    if (cudaStreamSynchronize(s) != cudaSuccess || cudaEventRecord(e0, s) != cudaSuccess)
                        st = fail(CCFMM_ERR_CUDA, "autotuner: timing failed");
                    for (int t = 0; t < trials && st == CCFMM_OK; ++t) st = batch_run(sb, 0, nullptr, nullptr);
                    if (st == CCFMM_OK && (cudaEventRecord(e1, s) != cudaSuccess ||
                                           cudaEventSynchronize(e1) != cudaSuccess ||
                                           cudaEventElapsedTime(&t_ms, e0, e1) != cudaSuccess))
                        st = fail(CCFMM_ERR_CUDA, "autotuner: timing failed");
                }
                fmm_batch_destroy(sb);
                if (st != CCFMM_OK) break;
                const double ms = t_ms / std::max(trials, 1);
                if (ms < best_ms) {
                    best_ms = ms;
                    best.leaf = lf;
                    best.item_len = il;
                }
            }
        cudaFree(dpos);
        cudaFree(dmom);
        dpos = dmom = nullptr;
        if (st != CCFMM_OK) break;
        for (int i : mem) class_of[i] = (int)classes.size();
        classes.push_back(best);
    }
    if (dpos) cudaFree(dpos);
    if (dmom) cudaFree(dmom);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaGetLastError();
    return st;
}

ccfmm_status fmm_batch_create(const double *positions, const double *moments,
                              const int64_t *offsets, int nsamples, int p, double theta,
                              double leaf_size, ccfmm_prec prec, void *stream, ccfmm_batch_t *out)
{
    return fmm_batch_create_ex(positions, moments, offsets, nsamples, p, theta, leaf_size, prec,
                               nullptr, stream, out);
}

ccfmm_status fmm_batch_create_ex(const double *positions, const double *moments,
                                 const int64_t *offsets, int nsamples, int p, double theta,
                                 double leaf_size, ccfmm_prec prec, const ccfmm_batch_opts *opts,
                                 void *stream, ccfmm_batch_t *out)
{
    return batch_create(positions, moments, offsets, nsamples, p, theta, leaf_size, prec, opts,
                        stream, out, 0.0, 0);
}

}  // extern "C"

// leaf_all > 0 / il_all > 0: every sample's leaf occupancy and M2L item
// length (the autotuner's trial sub-ensembles)
static ccfmm_status batch_create(const double *positions, const double *moments,
                                 const int64_t *offsets, int nsamples, int p, double theta,
                                 double leaf_size, ccfmm_prec prec, const ccfmm_batch_opts *opts,
                                 void *stream, ccfmm_batch_t *out, double leaf_all, int il_all)
{
    g_err.clear();
    if (!out || !positions || !moments || !offsets) return fail(CCFMM_ERR_ARG, "NULL argument");
    *out = nullptr;
    if (nsamples < 1) return fail(CCFMM_ERR_ARG, "nsamples < 1");
    if (offsets[0] != 0) return fail(CCFMM_ERR_ARG, "offsets[0] must be 0");
    for (int i = 0; i < nsamples; ++i)
        if (offsets[i + 1] <= offsets[i]) return fail(CCFMM_ERR_ARG, "sample %d is empty", i);
    ccfmm_batch_t b = new (std::nothrow) ccfmm_batch_s();
    if (!b) return fail(CCFMM_ERR_ALLOC, "host allocation failed");
    ccfmm_status st = CCFMM_OK;
#define BTRY(x)                                                                                  \
    do {                                                                                         \
        st = (x);                                                                                \
        if (st != CCFMM_OK) {                                                                    \
            std::string m_ = g_err;                                                              \
            fmm_batch_destroy(b);                                                                \
            g_err = m_;                                                                          \
            return st;                                                                           \
        }                                                                                        \
    } while (0)
#define BCK(call)                                                                                \
    do {                                                                                         \
        cudaError_t e_ = (call);                                                                 \
        if (e_ != cudaSuccess) {                                                                 \
            cudaGetLastError();                                                                  \
            fmm_batch_destroy(b);                                                                \
            return fail(CCFMM_ERR_CUDA, "%s failed: %s", #call, cudaGetErrorString(e_));        \
        }                                                                                        \
    } while (0)
    BCK(cudaGetDevice(&b->device));
    b->ns = nsamples;
    b->prec = prec;
    b->off.assign(offsets, offsets + nsamples + 1);
    b->total = b->off[nsamples];
    if (stream) {
        b->stream = (cudaStream_t)stream;
    } else {
        BCK(cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking));
        b->own_stream = true;
    }
    // parallel branches of the step graph (CCFMM_BATCH_BRANCHES overrides)
    int maxbr = 32;
    if (const char *e = getenv("CCFMM_BATCH_BRANCHES")) maxbr = std::max(1, atoi(e));
    b->nbr = std::min(nsamples, maxbr);
    for (int r = 0; r < b->nbr; ++r) {
        cudaStream_t s;
        cudaEvent_t e;
        BCK(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
        b->br.push_back(s);
        BCK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
        b->evj.push_back(e);
    }
    BCK(cudaEventCreateWithFlags(&b->evf, cudaEventDisableTiming));
    BTRY(ensure(b->mom, sizeof(double) * 3 * b->total));
    BTRY(ensure(b->H, sizeof(double) * 3 * b->total));
    BTRY(ensure(b->E, sizeof(double) * nsamples));
    BTRY(ensure(b->prm, sizeof(RotateParams)));
    BCK(cudaMallocHost((void **)&b->hprm, sizeof(RotateParams)));
    {
        cudaMemcpyKind k = is_device_ptr(moments) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
        BCK(cudaMemcpyAsync(b->mom.p, moments, sizeof(double) * 3 * b->total, k, b->stream));
        BCK(cudaStreamSynchronize(b->stream));
    }
    if (opts && opts->autotune) {
        // the positions may be host memory: the trial handles copy them in
        BTRY(batch_autotune(positions, P<double>(b->mom), b->off, p, theta, leaf_size, prec,
                            opts->trials > 0 ? opts->trials : 3, b->br[0], b->tune, b->tune_of));
        b->tuned = true;
    }
    for (int i = 0; i < nsamples; ++i) {
        ccfmm_t hs = nullptr;
        long long o = b->off[i], n = b->off[i + 1] - o;
        const double lf = b->tuned ? b->tune[b->tune_of[i]].leaf
                                   : (leaf_all > 0.0 ? leaf_all : leaf_size);
        const int il = b->tuned ? b->tune[b->tune_of[i]].item_len : (il_all > 0 ? il_all : M2L_EC);
        BTRY(create_handle(positions + 3 * o, P<double>(b->mom) + 3 * o, n, p, theta, lf,
                           nullptr, prec, b->br[i % b->nbr], true, &hs, il));
        hs->mom_energy = P<double>(b->mom) + 3 * o;
        hs->E_dst = P<double>(b->E) + i;
        b->h.push_back(hs);
    }
    // the handles' builds end with kernels still queued on the branch
    // streams; a captured graph would not depend on them
    for (cudaStream_t s : b->br) BCK(cudaStreamSynchronize(s));
    b->batched = batch_can_batch(b);
    BCK(cudaMallocHost((void **)&b->heflag, sizeof(int)));
    *b->heflag = 0;
#undef BTRY
#undef BCK
    *out = b;
    return CCFMM_OK;
}

extern "C" {

ccfmm_status fmm_batch_step(ccfmm_batch_t b, uint64_t seed, uint64_t step, double max_angle,
                            double *H_out, double *E_out)
{
    g_err.clear();
    if (!b) return fail(CCFMM_ERR_ARG, "batch is NULL");
    if (!(max_angle >= 0.0) || isinf(max_angle)) return fail(CCFMM_ERR_ARG, "bad max_angle");
    CK(cudaSetDevice(b->device));
    // the previous step's graph may still read the parameter block
    CK(cudaStreamSynchronize(b->stream));
    b->hprm->seed = seed;
    b->hprm->step = step;
    b->hprm->max_angle = max_angle;
    CK(cudaMemcpyAsync(b->prm.p, b->hprm, sizeof(RotateParams), cudaMemcpyHostToDevice, b->stream));
    return batch_run(b, 1, H_out, E_out);
}

ccfmm_status fmm_batch_evaluate(ccfmm_batch_t b, double *H_out, double *E_out)
{
    g_err.clear();
    if (!b) return fail(CCFMM_ERR_ARG, "batch is NULL");
    CK(cudaSetDevice(b->device));
    return batch_run(b, 0, H_out, E_out);
}

ccfmm_status fmm_batch_get_moments(ccfmm_batch_t b, double *out)
{
    g_err.clear();
    if (!b || !out) return fail(CCFMM_ERR_ARG, "NULL argument");
    CK(cudaSetDevice(b->device));
    cudaMemcpyKind k = is_device_ptr(out) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    CK(cudaMemcpyAsync(out, b->mom.p, sizeof(double) * 3 * b->total, k, b->stream));
    CK(cudaStreamSynchronize(b->stream));
    return CCFMM_OK;
}

ccfmm_status fmm_batch_set_moments(ccfmm_batch_t b, const double *moments)
{
    g_err.clear();
    if (!b || !moments) return fail(CCFMM_ERR_ARG, "NULL argument");
    CK(cudaSetDevice(b->device));
    CK(cudaStreamSynchronize(b->stream));
    cudaMemcpyKind k = is_device_ptr(moments) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    CK(cudaMemcpyAsync(b->mom.p, moments, sizeof(double) * 3 * b->total, k, b->stream));
    CK(cudaStreamSynchronize(b->stream));
    return CCFMM_OK;
}

ccfmm_status fmm_batch_sample(ccfmm_batch_t b, int i, ccfmm_t *out)
{
    g_err.clear();
    if (!b || !out || i < 0 || i >= b->ns) return fail(CCFMM_ERR_ARG, "bad argument");
    CK(cudaStreamSynchronize(b->stream));
    *out = b->h[i];
    return CCFMM_OK;
}

ccfmm_status fmm_batch_tuning(ccfmm_batch_t b, int32_t *nclasses, int64_t *class_nmin,
                              double *class_leaf, int32_t *class_item_len, int32_t capacity)
{
    g_err.clear();
    if (!b || !nclasses) return fail(CCFMM_ERR_ARG, "NULL argument");
    *nclasses = b->tuned ? (int32_t)b->tune.size() : 0;
    for (int i = 0; i < *nclasses && i < capacity; ++i) {
        if (class_nmin) class_nmin[i] = b->tune[i].nmin;
        if (class_leaf) class_leaf[i] = b->tune[i].leaf;
        if (class_item_len) class_item_len[i] = b->tune[i].item_len;
    }
    return CCFMM_OK;
}

ccfmm_status fmm_batch_info(ccfmm_batch_t b, int64_t *total_n, int64_t *kernels_per_step)
{
    g_err.clear();
    if (!b) return fail(CCFMM_ERR_ARG, "batch is NULL");
    if (total_n) *total_n = b->total;
    if (kernels_per_step) *kernels_per_step = b->graph_kernels[1];
    return CCFMM_OK;
}

}  // extern "C"
