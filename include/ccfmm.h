/*
 * ccfmm.h -- C-ABI of libccfmm, a GB300 (sm_103a) implementation of the
 * Cartesian-coordinates fast multipole method for point dipoles of
 * W. Zhang and S. Haas, "Adaptation and Performance of the Cartesian
 * Coordinates Fast Multipole Method for Nanomagnetic Simulations".
 *
 * Problem (Sec. III, Eqs. H and H2): N point dipoles m_i at positions r_i,
 * open boundaries.  The library returns the dipolar field at every dipole,
 *     H_i = sum_{j != i} [3 (m_j . u_ij) u_ij - m_j] / |r_i - r_j|^3,
 *     u_ij = (r_i - r_j) / |r_i - r_j|,
 * and the energy E = -1/2 sum_i m_i . H_i (Appendix, updateField), both in
 * units where mu0/4pi = 1.  A source located exactly at the field point
 * contributes nothing (Appendix, updateField).  The fast method replaces the
 * far part of the sum by the multipole / Taylor expansions of Sec. III.
 *
 * Conventions for every entry point:
 *   - Arrays of 3-vectors are N x 3, row-major, float64 (x0 y0 z0 x1 ...).
 *   - A pointer may be host memory (pageable or pinned) or device memory of
 *     the current CUDA device; the kind is detected per call.  Inputs are
 *     copied into library-owned device memory before the call returns or, for
 *     device pointers, in stream order on the handle's stream.  Outputs are
 *     caller-owned.  Host outputs are complete when the call returns; device
 *     outputs are complete in stream order on the handle's stream.
 *   - No entry point throws, aborts or exits.  Each returns a ccfmm_status;
 *     on failure ccfmm_last_error() gives a message for the calling thread.
 *   - A handle is used by one host thread at a time.
 *   - All GPU work runs on the handle's stream (fmm_create_ex) or on the
 *     legacy default stream (fmm_create).
 */
#ifndef CCFMM_H
#define CCFMM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ccfmm_s *ccfmm_t; /* opaque; owned by the library */

typedef enum {
    CCFMM_OK = 0,
    CCFMM_ERR_ARG = -1,     /* invalid argument (sizes, ranges, NaN, null) */
    CCFMM_ERR_ALLOC = -2,   /* device or host allocation failed */
    CCFMM_ERR_CUDA = -3,    /* a CUDA call failed; message has the reason */
    CCFMM_ERR_TIMEOUT = -4, /* a bounded device wait gave up */
    CCFMM_ERR_STATE = -5    /* call not valid in the handle's state */
} ccfmm_status;

typedef enum {
    CCFMM_FP64 = 0,  /* every stage in FP64 */
    CCFMM_MIXED = 1  /* FP32 bulk; FP64 derivative tensors (Eqs. Dn, Dnr) and
                        FP64 per-cell local-expansion accumulation */
} ccfmm_prec;

/* Counters and per-stage times of the last build / evaluation. */
typedef struct {
    int32_t depth;            /* L: leaves are at level L (Sec. II) */
    int32_t depth_capped;     /* 1 if the depth rule wanted L > 24 */
    int32_t p;                /* expansion order p_m */
    int32_t precision;        /* ccfmm_prec */
    double theta;             /* opening-angle threshold alpha_m */
    double leaf_target;       /* s used by the depth rule */
    double box[6];            /* lo xyz, hi xyz */
    double leaf_width[3];     /* widths of a leaf cell */
    int64_t n;                /* number of dipoles */
    int64_t nonempty_leaves;
    int64_t near_leaf_pairs;  /* (leaf, nearPartner) entries, self included */
    int64_t far_pairs;        /* (cell, Partner) entries over all levels */
    int64_t p2p_pairs;        /* dipole pairs evaluated by the near field (j != i) */
    int64_t m2l_tile_entries; /* (target tile, offset) work items of M2L */
    int64_t far_offsets;      /* distinct D tables (scaled separations) of the far offsets */
    double ms_build;          /* tree + lists + D tables of the last build */
    double ms_eval;           /* mean evaluation time (P2M ... unpermute) */
    double ms_stage[8];       /* mean stage times: P2M, M2M, M2L, L2L, L2P, P2P,
                                 finish; [7] = number of evaluations averaged.
                                 With the near/far overlap (default) P2P runs
                                 concurrently with P2M..L2L, so the stages do
                                 not add up to ms_eval */
    double ms_build_stage[6]; /* the last build by phase (device time between
                                 stream events, so waits for the host count):
                                 [0] input upload, box, keys, sort;
                                 [1] depth choice (host), leaf ranges, sorted
                                 points, cells per level; [2] lists of every
                                 level and tile counts (after the plan, which
                                 the host builds while [1] runs); [3] M2L
                                 work items (host) and their upload; [4] tile
                                 fill, F table (first build), D tables;
                                 [5] host time of the plan alone */
} ccfmm_stats;

/* ------------------------------------------------------------------------
 * fmm_create: build the tree, the interaction lists and the derivative
 * tensors for N dipoles (Sec. II steps 0-1, Appendix createPartners) and
 * upload the moments.
 *   positions, moments  N x 3 float64, host or device.
 *   N                   >= 1 and < 2^31.
 *   p                   expansion order p_m, 1..8 (Sec. III truncation).
 *   theta               opening-angle threshold alpha_m, 0 < theta < 1
 *                       (Sec. II: a pair is near iff 2r/d > alpha_m).
 *   leaf_size           target mean number of dipoles in a leaf, s (Sec. IV);
 *                       <= 0 selects Eq. so (0.74 p^2 for p > 3, else 8);
 *                       0 < leaf_size < 1 is rejected.
 *   out                 receives the handle.
 * The box is the bounding box widened by 2^-20 of its largest extent on
 * every side; the precision is CCFMM_MIXED; the stream is the legacy default
 * stream.  Errors: CCFMM_ERR_ARG for bad sizes, ranges, null or non-finite
 * input; CCFMM_ERR_ALLOC; CCFMM_ERR_CUDA.
 * ---------------------------------------------------------------------- */
ccfmm_status fmm_create(const double *positions, const double *moments, int64_t N, int p,
                        double theta, double leaf_size, ccfmm_t *out);

/* As fmm_create, with
 *   box     NULL, or {lo_x, lo_y, lo_z, hi_x, hi_y, hi_z} with lo < hi; every
 *           position must lie in [lo, hi] (else CCFMM_ERR_ARG).  The paper's
 *           lattice examples use the lattice-cell box (Sec. IV).
 *   prec    CCFMM_FP64 or CCFMM_MIXED.
 *   stream  a cudaStream_t of the current device, or NULL for the legacy
 *           default stream.  The library never synchronises other streams. */
ccfmm_status fmm_create_ex(const double *positions, const double *moments, int64_t N, int p,
                           double theta, double leaf_size, const double *box, ccfmm_prec prec,
                           void *stream, ccfmm_t *out);

/* Rebuild tree, lists and derivative tensors for new positions (and
 * moments) with the same N, p, theta, leaf_size, box rule and precision,
 * reusing the handle's device memory where it suffices.  Returns once the
 * inputs have been read (the caller may then change or free them); the last
 * build kernels may still be running on the handle's stream, and every later
 * call on the handle is ordered after them.  (fmm_create builds the same
 * way.) */
ccfmm_status fmm_set_positions(ccfmm_t h, const double *positions, const double *moments);

/* Replace the moments; the tree and lists are kept (positions unchanged). */
ccfmm_status fmm_set_moments(ccfmm_t h, const double *moments);

/* Truncation of the far-field series of Eq. taylorcalc (Sec. II, the error
 * estimate "after the p-th order").  max_degree <= 0 selects the default
 * square truncation: every stored Q_k (1 <= |k| <= p) feeds every stored V_n
 * (1 <= |n| <= p).  Otherwise only the terms with |n| + |k| <= max_degree
 * are kept, 2 <= max_degree <= 2p.  2p is the square truncation again.
 * max_degree = p + 1 makes every far interaction the Taylor polynomial of
 * degree p - 1 of the dipole field in the target-source offset.  It applies
 * to every later evaluation, on all M2L engines.  The FMA engines (FP64,
 * and FP32 under CCFMM_M2L=fma) skip the dropped terms.  The tensor-core
 * engine multiplies zero operands in their place, so its cost is unchanged.
 * Errors: CCFMM_ERR_ARG for a bound outside that range; CCFMM_ERR_STATE for
 * a handle owned by an ensemble (fmm_batch_sample), which keeps the square
 * truncation.  Asynchronous on the handle's stream, like fmm_set_positions. */
ccfmm_status fmm_set_truncation(ccfmm_t h, int max_degree);

/* The handle's current bound on |n| + |k| (2p for the square truncation). */
ccfmm_status fmm_get_truncation(ccfmm_t h, int *max_degree);

/* Evaluate the field at every dipole: upward pass (Eqs. multipolemoments,
 * momentshift), downward pass (Eqs. taylorcalc, taylorshift), smooth field
 * (Eq. H) and near field (Eq. H2).  H_out: N x 3 float64 in input order,
 * host or device, caller-owned; NULL evaluates without copying out (the
 * result stays in the handle for fmm_energy / fmm_get_field). */
ccfmm_status fmm_field(ccfmm_t h, double *H_out);

/* Evaluate (as fmm_field) and return E = -1/2 sum_i m_i . H_i in *E_out
 * (host pointer).  H_out may be NULL. */
ccfmm_status fmm_field_energy(ccfmm_t h, double *H_out, double *E_out);

/* E of the current moments (evaluates the field first). */
ccfmm_status fmm_energy(ccfmm_t h, double *E_out);

/* Counters and stage times (host struct).  Stage times are CUDA-event
 * durations on the handle's stream, averaged over the evaluations since the
 * last fmm_reset_stats (at most the last 32).  Synchronises the stream. */
ccfmm_status fmm_stats(ccfmm_t h, ccfmm_stats *out);

/* Start a new averaging window for the stage times of fmm_stats. */
ccfmm_status fmm_reset_stats(ccfmm_t h);

/* Release the handle and its device memory.  NULL is ignored. */
void fmm_destroy(ccfmm_t h);

/* Message of the last failed call on this thread ("" if none). */
const char *ccfmm_last_error(void);

/* ------------------------------------------------------------------------
 * Inspection of the build, for verification (tests compare each stage with
 * an independent implementation).  All outputs are host arrays.
 * Cell numbering: level l holds 2^l cells keyed 0..2^l-1 by the bits of the
 * recursive bisection (bit 0 = lower half along the axis split at that
 * level, most significant bit = level 1); the cell's heap id is 2^l + key.
 * ---------------------------------------------------------------------- */

/* Split axis (0=x,1=y,2=z) of levels 1..L into axes[0..L). */
ccfmm_status fmm_get_axes(ccfmm_t h, int32_t *axes);

/* Leaf key of every dipole, input order (N int64). */
ccfmm_status fmm_get_leaf_of(ccfmm_t h, int64_t *leaf_of);

/* Interaction lists as (cell heap id, partner heap id) pairs.
 * kind 0: nearPartners of the leaves (self included);
 * kind 1: Partners (far pairs, M2L) of every cell.
 * Only non-empty cells appear.  *count receives the number of pairs; pairs
 * (2 x count int64) is filled when not NULL and capacity >= count. */
ccfmm_status fmm_get_pairs(ccfmm_t h, int kind, int64_t *pairs, int64_t capacity,
                           int64_t *count);

/* M2L operands: sizes[0..3] = (D tables, T(2p), M2L entries, tiles); D_out
 * (tables x T(2p) float64, the D tensors at scaled separations c/h, Eqs.
 * Dn/Dnr; one per distinct scaled separation, shared by levels of the same
 * cell shape), ent_u_out (entries: D table id), ent_src_out
 * (entries x 128: partner heap id or -1), tiles_out (tiles x 8 int32:
 * level, first, parity, cells, entry start, entry count, offsets, first
 * offset id; a tile's cells are the non-empty cells of its level with that
 * parity of the key, numbers first .. first + cells - 1 of them in key
 * order).  Any output may be NULL; call with all NULL to get sizes. */
ccfmm_status fmm_get_m2l_data(ccfmm_t h, int64_t *sizes, double *D_out, int32_t *ent_u_out,
                              int32_t *ent_src_out, int32_t *tiles_out);

/* Multi-index ordering of the library: orders 0..order, T(order) x 3 int32. */
ccfmm_status ccfmm_multi_indices(int order, int32_t *out);

/* Multipole moments Q (kind 0) or Taylor coefficients V (kind 1) of every
 * cell after the last evaluation, float64, (2^(L+1)) x T(p) in heap-id rows
 * (row 0 unused) and library multi-index order.  Q_0 = V_0 = 0. */
ccfmm_status fmm_get_expansions(ccfmm_t h, int kind, double *out);

/* ------------------------------------------------------------------------
 * Direct sum (the O(N^2) definition, Eq. H2 as above) on the GPU in FP64,
 * at the targets tgt[0..nt) (NULL: every dipole, nt = N).  Used to measure
 * the error of the fast method; not part of the fast path.
 *   positions, moments  N x 3 float64, host or device.
 *   H_out               nt x 3 float64, host or device.
 *   stream              cudaStream_t or NULL.
 * ---------------------------------------------------------------------- */
ccfmm_status ccfmm_direct_field(const double *positions, const double *moments, int64_t N,
                                const int64_t *tgt, int64_t nt, double *H_out, void *stream);

/* ------------------------------------------------------------------------
 * Ensemble of independent samples (a project addition; the paper evaluates
 * one system).  The samples' trees, lists and derivative tensors are built
 * once (positions stay fixed); each step turns every moment by a random
 * rotation and evaluates every sample's field, as one CUDA graph launch.
 *   positions, moments  concatenated samples, total x 3 float64, host or
 *                       device; sample i is rows offsets[i] .. offsets[i+1].
 *   offsets             nsamples + 1 host int64, offsets[0] = 0, increasing.
 *   p, theta, leaf_size, prec   as in fmm_create_ex, shared by the samples.
 *   stream              cudaStream_t (not the legacy default stream) or NULL
 *                       for a stream owned by the batch.
 * ---------------------------------------------------------------------- */
typedef struct ccfmm_batch_s *ccfmm_batch_t;

ccfmm_status fmm_batch_create(const double *positions, const double *moments,
                              const int64_t *offsets, int nsamples, int p, double theta,
                              double leaf_size, ccfmm_prec prec, void *stream, ccfmm_batch_t *out);

/* Options of fmm_batch_create_ex (fmm_batch_create = all zero).
 *   autotune  nonzero: the library picks, per sample-size class (the
 *             octaves of N, floor(log2 N)), the leaf occupancy and the
 *             M2L work-item length (entries of a tile per tensor-core work
 *             item) by timed trial evaluations of the class's median-size
 *             sample: leaf = s x {1/2, 1/sqrt2, 1, sqrt2, 2} with s =
 *             leaf_size (or Eq. so when leaf_size <= 0), item length 32 or
 *             64; the fastest mean evaluation time wins.  Trials run on the
 *             batch's first branch stream at creation.
 *   trials    timed evaluations per candidate (<= 0: 3). */
typedef struct {
    int32_t autotune;
    int32_t trials;
} ccfmm_batch_opts;

ccfmm_status fmm_batch_create_ex(const double *positions, const double *moments,
                                 const int64_t *offsets, int nsamples, int p, double theta,
                                 double leaf_size, ccfmm_prec prec, const ccfmm_batch_opts *opts,
                                 void *stream, ccfmm_batch_t *out);

/* The autotuner's choice: nclasses size classes (0 without autotune); for
 * class i < capacity, the smallest N of the class, its leaf occupancy and
 * its M2L item length (any output array may be NULL). */
ccfmm_status fmm_batch_tuning(ccfmm_batch_t b, int32_t *nclasses, int64_t *class_nmin,
                              double *class_leaf, int32_t *class_item_len, int32_t capacity);

/* One time step: every moment m_i (global row i) is turned about a random
 * axis by a random angle, drawn from Philox4x64-10 (Salmon et al., SC 2011)
 * with key (seed, step) and counter (i, 0, 0, 0): from its outputs x0..x3,
 * u_j = (x_j >> 11) 2^-53, axis = (sqrt(1-z^2) cos phi, sqrt(1-z^2) sin phi,
 * z) with z = 1 - 2 u0, phi = 2 pi u1, angle = max_angle u2 (Rodrigues'
 * formula, FP64).  Then every sample's field is evaluated.
 *   H_out  total x 3 float64 (host, device or NULL).
 *   E_out  nsamples float64 energies, E = -1/2 sum m.H per sample (host,
 *          device or NULL). */
ccfmm_status fmm_batch_step(ccfmm_batch_t b, uint64_t seed, uint64_t step, double max_angle,
                            double *H_out, double *E_out);

/* Evaluate every sample for the current moments (no rotation). */
ccfmm_status fmm_batch_evaluate(ccfmm_batch_t b, double *H_out, double *E_out);

/* Current moments (total x 3), and replacing them. */
ccfmm_status fmm_batch_get_moments(ccfmm_batch_t b, double *out);
ccfmm_status fmm_batch_set_moments(ccfmm_batch_t b, const double *moments);

/* Handle of sample i, owned by the batch (valid until fmm_batch_destroy),
 * for inspection with fmm_stats / fmm_get_* only. */
ccfmm_status fmm_batch_sample(ccfmm_batch_t b, int i, ccfmm_t *out);

/* Total dipoles and kernels launched by one step's graph.  With the FP32
 * path and the tensor-core M2L every stage of a step is one launch over all
 * samples (tens of kernels per step, independent of nsamples); otherwise the
 * graph holds each sample's own launches on parallel branches. */
ccfmm_status fmm_batch_info(ccfmm_batch_t b, int64_t *total_n, int64_t *kernels_per_step);

void fmm_batch_destroy(ccfmm_batch_t b);

/* ------------------------------------------------------------------------
 * Parameter selector (a project addition).  The paper chooses the leaf
 * occupancy by Eq. so and (p_m, alpha_m) by hand from Table II / Fig. 3
 * (Sec. IV).  Here a small network predicts, for a dipole set's features and
 * a configuration (p, theta, leaf), y0 = log10(time per dipole in ns) and
 * y1 = log10(relative RMS field error) of the FMM; fmm_select picks the
 * fastest grid configuration predicted to meet a target error.
 *
 * Features (ccfmm_features, 9 floats): log10 N; occupancy of the depth-Lr
 * cells of the bisection tree (Lr = max(0, floor(log2(N/16)))):
 * slog(CV^2), slog(skewness), slog(excess kurtosis), slog(x) = sign(x)
 * log10(1+|x|); the nearest-neighbour distances of min(N, 2048) sample
 * points: coefficient of variation, min/mean, Clark-Evans ratio
 * mean / (0.55396 (V/N)^(1/3)); the box extents sorted: middle/largest,
 * smallest/largest.  The network input is the 9 features followed by
 * p, theta and log2(leaf).
 *
 * Network: 12-64-64-64-2, ReLU, parameters in the order W1 (12x64,
 * row-major), b1, W2, b2, W3, b3, W4 (64x2), b4 (ccfmm_mlp_num_params()
 * floats); normalisation block mu_x[12], sd_x[12], mu_y[2], sd_y[2]
 * (inputs and targets standardised).  FP32 master weights; the forward and
 * backward passes use their BF16 roundings with FP32 accumulation.  Loss:
 * masked mean squared error in standardised units.  Training: Adam
 * (beta 0.9/0.999, eps 1e-8) over contiguous mini-batches.
 * All arrays may be host or device memory; calls synchronise the device.
 * ---------------------------------------------------------------------- */
typedef struct ccfmm_mlp_s *ccfmm_mlp_t;

ccfmm_status ccfmm_mlp_create(ccfmm_mlp_t *out);
void ccfmm_mlp_destroy(ccfmm_mlp_t m);
int32_t ccfmm_mlp_num_params(void);
/* params: ccfmm_mlp_num_params() floats or NULL; norm: 28 floats or NULL.
 * Setting resets the Adam state. */
ccfmm_status ccfmm_mlp_set_params(ccfmm_mlp_t m, const float *params, const float *norm);
ccfmm_status ccfmm_mlp_get_params(ccfmm_mlp_t m, float *params, float *norm);
/* Normalisation from data: X (B x 12), T (B x 2) targets, mask (B x 2, 0/1). */
ccfmm_status ccfmm_mlp_fit_norm(ccfmm_mlp_t m, const float *X, const float *T, const float *mask,
                                int64_t B);
/* Loss and its gradient with respect to the (BF16-rounded) parameters. */
ccfmm_status ccfmm_mlp_gradient(ccfmm_mlp_t m, const float *X, const float *T, const float *mask,
                                int64_t B, float *grad_out, float *loss_out);
/* `epochs` passes of Adam over mini-batches of `batch` rows; *loss_out gets
 * the mean mini-batch loss of the last epoch. */
ccfmm_status ccfmm_mlp_train(ccfmm_mlp_t m, const float *X, const float *T, const float *mask,
                             int64_t B, int64_t batch, int32_t epochs, float lr, uint64_t seed,
                             float *loss_out);
/* Predictions in physical units: Y (B x 2) = (log10 ns per dipole, log10 error). */
ccfmm_status ccfmm_mlp_predict(ccfmm_mlp_t m, const float *X, int64_t B, float *Y);
/* The nine features of a dipole set (positions N x 3 float64). */
ccfmm_status ccfmm_features(const double *positions, int64_t N, float *out9);
/* Choose (p, theta, leaf) for a target relative RMS field error: the fastest
 * configuration on the grid p in 2..8, theta in {0.3..0.7}, leaf in
 * {4, 8, 16, 32, 64} whose predicted error is below target/2.  Falls back to
 * the rule of thumb (Eq. so; (5, 0.71) for targets >= 1e-2, else (6, 0.48),
 * Sec. IV) when m is NULL, the features lie outside the training range (more
 * than 5 standard deviations) or no configuration qualifies;
 * *fallback_out (may be NULL) tells which. */
ccfmm_status fmm_select(ccfmm_mlp_t m, const double *positions, int64_t N, double target_error,
                        int32_t *p_out, double *theta_out, double *leaf_out, int32_t *fallback_out);

/* ------------------------------------------------------------------------
 * Lattice FFT comparator (Sec. V: the FFT method the paper compares the
 * Cartesian FMM with, on the simple-cubic lattice benchmark of Sec. IV).
 * For dipoles on the lattice r = a (ix, iy, iz), 0 <= ix < nx, ... , the
 * field of every site, H_i = sum_{j != i} G(r_i - r_j) m_j with
 * G(r) = (3 r r^T - |r|^2 I) / |r|^5 (Eq. H2 as read), is a discrete
 * convolution; the library evaluates it exactly (up to rounding) by
 * zero-padded 3-D FFTs: each axis padded to 2n, so that no wrapped image
 * overlaps (open boundaries).  The tensor spectra are computed once per
 * handle.  The FFTs are cuFFT calls (opened at run time); the scatter, the
 * 3 x 3 spectral product, the gather and the energy are the library's
 * kernels.
 *   nx, ny, nz   sites per axis, 1 .. 4096 each.
 *   spacing      a > 0.
 *   precision    CCFMM_FP64 (FP64 transforms) or CCFMM_MIXED (FP32
 *                transforms; tensor built in FP64, energy summed in FP64).
 *   moments      N x 3 float64 (N = nx ny nz), site (ix, iy, iz) at row
 *                (ix ny + iy) nz + iz; host or device memory.
 *   H_out        N x 3 float64, same order, or NULL; host or device.
 *   E_out        E = -1/2 sum m.H, or NULL; host or device.
 * fmm_lattice_field synchronises the handle's stream before it returns
 * (outputs complete).  Errors: CCFMM_ERR_ARG for sizes, spacing or
 * precision out of range and for non-finite moments (reported after the
 * evaluation; outputs then undefined); CCFMM_ERR_ALLOC; CCFMM_ERR_CUDA when
 * cuFFT cannot be opened or a CUDA/cuFFT call fails.
 * ---------------------------------------------------------------------- */
typedef struct ccfmm_lattice_s *ccfmm_lattice_t;

ccfmm_status fmm_lattice_create(int32_t nx, int32_t ny, int32_t nz, double spacing,
                                int32_t precision, void *cuda_stream, ccfmm_lattice_t *out);
ccfmm_status fmm_lattice_field(ccfmm_lattice_t h, const double *moments, double *H_out,
                               double *E_out);
void fmm_lattice_destroy(ccfmm_lattice_t h);

/* ------------------------------------------------------------------------
 * Allocation-free direct field and energy.  The paper has no counterpart:
 * this entry point exists for callers that cannot call cudaMalloc, such as
 * code running inside a host application that owns all GPU memory through
 * its own pool, or a plugin that must not change the device's allocation
 * state.  It computes what ccfmm_direct_field computes (FP64 O(N^2) field,
 * j != i and coincident points skipped) and E = -1/2 sum_i m_i . H_i, and
 * allocates nothing: no cudaMalloc, cudaFree or allocating library call.
 *   positions, moments  N x 3 float64, DEVICE memory of the current device
 *                       (or managed memory); memory of another GPU is
 *                       rejected with CCFMM_ERR_ARG.
 *   N                   1 <= N <= 4,194,304; larger N returns CCFMM_ERR_ARG.
 *   H_out               N x 3 float64, DEVICE memory of the current device,
 *                       caller-owned.
 *   E_out               one float64, host memory or device memory of the
 *                       current device (another GPU's: CCFMM_ERR_ARG).
 *   stream              cudaStream_t or NULL; the call synchronises it.
 * Scratch: a fixed array of 32,769 doubles (about 256 KB) in the library's
 * device memory, held on every GPU that loads the library until the process
 * exits.  Its device address is looked up on the first call on each device
 * (with that device current).  The call synchronises its stream, so it
 * cannot be made while that stream is being captured (CCFMM_ERR_ARG).  All
 * calls share the array and it keeps the last call's values;
 * every value a call reads is written earlier in the same call.  Calls whose
 * GPU work overlaps (other streams, other host threads) race on the array:
 * serialise them.  Errors: CCFMM_ERR_ARG for NULL, N out of range, or
 * arrays that are not on the current device (the message names it);
 * CCFMM_ERR_CUDA.
 * ---------------------------------------------------------------------- */
ccfmm_status ccfmm_direct_field_energy_noalloc(const double *positions, const double *moments,
                                               int64_t N, double *H_out, double *E_out,
                                               void *stream);

/* Number of kernels the library has launched in this process (all handles,
 * all threads); a diagnostic for counting GPU work per call. */
int64_t ccfmm_kernel_launches(void);

/* Eq. so: rule-of-thumb leaf occupancy for order p (8 for p <= 3, else 0.74 p^2). */
double ccfmm_leaf_size_rule(int p);

/* ------------------------------------------------------------------------
 * Adaptive-depth tree (a project addition: the paper's tree is complete,
 * every leaf at one depth, Sec. II).  The complete tree's box, split
 * sequence (halve the widest axis, ties x < y < z) and point membership, but
 * a cell splits only while it holds more than s dipoles (to level 40 at
 * most) and empty children are not created.  Cells A and B of different
 * levels are near when (r_A + r_B) / d > theta, r = half the cell diagonal,
 * d = distance of the centres; for equal levels this is the paper's
 * 2r/d > alpha_m (Sec. II).  The interaction lists extend the Appendix's
 * createPartners to unequal levels: a child takes as near candidates the
 * children of the internal cells of its parent's near set and that set's
 * leaves as they are; far candidates are its Partners (M2L sources, any
 * level); at a leaf, near leaves are nearPartners (Eq. H2) and a near
 * internal cell is refined against the leaf (far descendants -> Partners,
 * near leaves -> nearPartners).  The expansions are those of Sec. III
 * (P2M Eq. multipolemoments, M2M Eq. momentshift, M2L Eq. taylorcalc at any
 * pair of levels, L2L Eq. taylorshift, L2P Eq. H).
 *
 * Several independent samples may share one handle (an ensemble): each gets
 * its own box and tree; one evaluation covers all of them.
 *   positions, moments  concatenated samples, total x 3 float64, host or
 *                       device; sample i is rows offsets[i] .. offsets[i+1].
 *   offsets             nsamples + 1 host int64, offsets[0] = 0, strictly
 *                       increasing (every sample holds a dipole).
 *   p                   1 .. 8; theta in (0, 1).
 *   split               nsamples thresholds s >= 1 (host), or NULL for
 *                       Eq. so: s = 0.74 p^2 (p > 3), else 8.
 *   box                 NULL (bounding box widened by 2^-20 of its largest
 *                       extent) or, for one sample only, 6 host doubles
 *                       (lo, hi); points outside are clamped to it.
 *   prec                CCFMM_FP64: every stage in FP64 with FP64 atomic
 *                       M2L accumulation; CCFMM_MIXED: FP32 P2M/M2M/M2L/P2P
 *                       with FP64 D tensors, M2L accumulated in FP32 per
 *                       cell and L2L in FP64.
 * Creation builds the trees, lists and D tensors on the handle's stream and
 * synchronises it.  M2L contributions are added with atomics, so results
 * may vary in the last bits from run to run.  Errors: CCFMM_ERR_ARG (bad
 * arguments, non-finite positions, a tree deeper or a box more elongated
 * than the 40-level keys and 30-bit cell coordinates allow, lists beyond
 * 2^31 entries), CCFMM_ERR_ALLOC, CCFMM_ERR_CUDA.
 * ---------------------------------------------------------------------- */
typedef struct ccfmm_adaptive_s *ccfmm_adaptive_t;

typedef struct {
    int64_t n;                /* dipoles over all samples */
    int32_t nsamples, p;
    double theta;
    int64_t ncells, nleaves;  /* over all samples */
    int32_t max_level, pad;
    int64_t far_pairs;        /* (cell, Partner) pairs */
    int64_t near_entries;     /* (leaf, nearPartner) pairs, the leaf itself included */
    int64_t near_pairs;       /* dipole pairs of the near field, sum n_leaf n_partner */
    int64_t d_rows;           /* distinct separations (one D tensor each) */
    int64_t m2l_items;        /* M2L work items */
    int64_t kernels_per_eval; /* kernels of one evaluation */
    double ms_build;          /* wall time of the build */
} ccfmm_adaptive_stats;

ccfmm_status fmm_adaptive_create(const double *positions, const double *moments,
                                 const int64_t *offsets, int nsamples, int p, double theta,
                                 const double *split, const double *box, ccfmm_prec prec,
                                 void *stream, ccfmm_adaptive_t *out);

/* Options of fmm_adaptive_create_ex (fmm_adaptive_create = autotune off).
 *   autotune  nonzero: the library picks the split threshold per sample-size
 *             class (floor(log2 N)): for each class, up to 16 of its samples
 *             (spread over its sizes) are built and evaluated as a trial
 *             forest for s = s0 x {1, sqrt2, 2, 2 sqrt2, 4} (s0: the given
 *             threshold of the class's median sample, or Eq. so), and the
 *             fastest mean evaluation time over `trials` timed evaluations
 *             (after one warm-up) wins.  Trials run on the handle's stream
 *             at creation.
 *   trials    timed evaluations per candidate (<= 0: 3).
 *   persistent  nonzero: every evaluation (and step) is one launch of a
 *             persistent kernel whose blocks take the stages' tiles of all
 *             samples from one task queue (rotation, permutation, P2M, M2M
 *             level by level, fold, M2L items, L2L level by level, near field,
 *             L2P, unpermute, energies), a task waiting for the phases it
 *             depends on with bounded polls; a wait that runs out ends the
 *             launch and the call returns CCFMM_ERR_TIMEOUT.  Needs the mixed
 *             path with the tensor-core M2L (p in 2..6): CCFMM_ERR_ARG
 *             otherwise.  Zero: the stages as separate kernels in one CUDA
 *             graph (the near field beside the far chain). */
typedef struct {
    int32_t autotune;
    int32_t trials;
    int32_t persistent;
} ccfmm_adaptive_opts;

ccfmm_status fmm_adaptive_create_ex(const double *positions, const double *moments,
                                    const int64_t *offsets, int nsamples, int p, double theta,
                                    const double *split, const double *box, ccfmm_prec prec,
                                    const ccfmm_adaptive_opts *opts, void *stream,
                                    ccfmm_adaptive_t *out);

/* The autotuner's choice: nclasses size classes (0 without autotune); for
 * class i < capacity its smallest N and its split threshold (either output
 * array may be NULL). */
ccfmm_status fmm_adaptive_tuning(ccfmm_adaptive_t a, int32_t *nclasses, int64_t *class_nmin,
                                 double *class_split, int32_t capacity);

/* Field at every dipole and the energy of every sample for the current
 * moments (one CUDA graph launch; synchronises).
 *   H_out  total x 3 float64 in input order (host, device or NULL).
 *   E_out  nsamples float64, E = -1/2 sum m.H per sample (host, device or
 *          NULL). */
ccfmm_status fmm_adaptive_evaluate(ccfmm_adaptive_t a, double *H_out, double *E_out);

/* The ensemble time step of fmm_batch_step (the same Philox4x64-10 rotation
 * of every moment, key (seed, step), counter (row, 0, 0, 0)), then an
 * evaluation. */
ccfmm_status fmm_adaptive_step(ccfmm_adaptive_t a, uint64_t seed, uint64_t step,
                               double max_angle, double *H_out, double *E_out);

ccfmm_status fmm_adaptive_set_moments(ccfmm_adaptive_t a, const double *moments);
ccfmm_status fmm_adaptive_get_moments(ccfmm_adaptive_t a, double *out);
ccfmm_status fmm_adaptive_info(ccfmm_adaptive_t a, ccfmm_adaptive_stats *out);

/* Cells in creation order (each sample's root, then depth first, lower
 * child first), 8 int64 per cell: level, parent, child0, child1 (-1 when
 * absent), first sorted dipole, dipole count, leaf flag, sample. */
ccfmm_status fmm_adaptive_cells(ccfmm_adaptive_t a, int64_t *out);

/* Sorted dipole order: out[i] = input row of the i-th sorted dipole (the
 * dipoles of a cell are rows first .. first + count - 1 of it). */
ccfmm_status fmm_adaptive_perm(ccfmm_adaptive_t a, int64_t *out);

/* Interaction pairs (cell, partner) as cell numbers: kind 0 nearPartners of
 * the leaves, kind 1 Partners (far).  *count receives the number; out
 * (2 x count int64, host) may be NULL to query it; capacity in pairs. */
ccfmm_status fmm_adaptive_pairs(ccfmm_adaptive_t a, int kind, int64_t *out, int64_t capacity,
                                int64_t *count);

/* Multipole moments Q and Taylor coefficients V of every cell after an
 * evaluation, ncells x (T(p) - 1) float64 each in the library's
 * multi-index order (host; either may be NULL). */
ccfmm_status fmm_adaptive_expansions(ccfmm_adaptive_t a, double *Q_out, double *V_out);

void fmm_adaptive_destroy(ccfmm_adaptive_t a);

/* The persistent step's task queue for a forest of the given shape, as
 * fmm_adaptive_create_ex with opts->persistent builds it (host only, no GPU;
 * for inspection and tests).
 *   N, nsamples, nleaf, ncells  dipoles, samples, leaf cells, cells
 *   max_level      deepest level; level_offsets: max_level + 2 offsets of
 *                  each level's cells in the level-ordered cell list
 *                  (nondecreasing, 0 first, ncells last)
 *   n_big, n_small M2L items of more than 16 pairs / of at most 16
 *   tasks          4 int32 per task in queue order: type | phase << 8, y, z,
 *                  (wait1 + 1) | (wait2 + 1) << 16 (0: no wait); types 0..11
 *                  = rotation, permutation, P2M, M2M, fold, big M2L item,
 *                  small M2L items, L2L, near field, L2P, unpermute, energy;
 *                  a tile of a warp-per-cell stage is [y, min(z, y + tiles[1]))
 *                  of its list (leaves, the level's cells, cells; small M2L:
 *                  groups of four items [y, min(z, y + tiles[2]))), a dipole
 *                  chunk is [y tiles[0], (y + 1) tiles[0]), a big item, a near-
 *                  field leaf or a sample is y.  May be NULL (count only).
 *   capacity       tasks room (in tasks); *ntasks receives the count
 *   need           tasks of each phase (may be NULL); need_capacity its room;
 *                  *nphases receives the phase count
 *   tiles          3 int32 (may be NULL): dipoles per chunk, cells per tile,
 *                  small-item groups per tile
 * Errors: CCFMM_ERR_ARG on an inconsistent shape; nothing is written past a
 * capacity (the counts are still returned). */
ccfmm_status fmm_adaptive_queue(int64_t N, int32_t nsamples, int32_t nleaf, int32_t ncells,
                                int32_t max_level, const int32_t *level_offsets, int32_t n_big,
                                int32_t n_small, int32_t *tasks, int64_t capacity,
                                int64_t *ntasks, int32_t *need, int32_t need_capacity,
                                int32_t *nphases, int32_t *tiles);

#ifdef __cplusplus
}
#endif

#endif /* CCFMM_H */
