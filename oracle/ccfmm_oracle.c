/*
 * ccfmm_oracle.c -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, FP64 CPU statement of the Cartesian-coordinates fast
 * multipole method for point dipoles of Zhang & Haas ("Adaptation and
 * Performance of the Cartesian Coordinates Fast Multipole Method for
 * Nanomagnetic Simulations"), together with the O(N^2) direct dipole sum that
 * the method approximates.  It exists only to check the GPU library: the test
 * suite, the package smoke check and the benchmark's CPU-baseline leg are the
 * only callers.  It shares no code, table or header with the GPU path.
 *
 * Every routine follows one passage of the paper, cited in its comment, in the
 * paper's order and notation: n = (nx,ny,nz), |n| = nx+ny+nz,
 * r^n = x^nx y^ny z^nz, n! = nx! ny! nz!  (Sec. III, shorthand definitions).
 * Where the printed text is garbled or ambiguous the reading taken is stated
 * at the point of use:
 *   - Eq. H2 (near field) is read as the field of dipole j at i,
 *     [3 (m_j . u) u - m_j] / r^3 with u = (r_i - r_j)/|r_i - r_j|, i.e.
 *     -grad of the dipole potential that Eq. multipolemoments implies.
 *   - Eq. H drops the minus sign of H = -grad V; the sign is restored.
 *   - The energy is E = -1/2 sum_i m_i . H_i (Appendix, updateField halves
 *     the leaf energy against double counting), in units of mu0/4pi.
 *   - "alpha_m == 2r/d" (Sec. II) is read as alpha == 2r/d; a pair is near
 *     when alpha > alpha_m strictly, so alpha == alpha_m is far.
 *   - Truncation of Eq. taylorcalc is "square" by default: every stored Q_k
 *     (1<=|k|<=p) feeds every stored V_n (1<=|n|<=p); V_0 never reaches H and
 *     is skipped.  The error discussion of Sec. II ("terms after the p_m-th
 *     order") also admits a total-degree reading, kept as an option: the term
 *     (n, k) is taken only when |n|+|k| <= P for a bound P in [2, 2p]; P = 2p
 *     is the square truncation and P = p+1 keeps exactly the Taylor polynomial
 *     of degree p-1 of each far field in (target - source) offsets.
 *   - The tree splits the currently longest axis, ties x<y<z; its depth L
 *     minimises |N / (non-empty leaves) - s| (ties to the smaller L); a point
 *     on a cell boundary belongs to the upper cell.
 *
 * Threads: OpenMP over independent cells / leaves / targets only; the
 * arithmetic for any one output is done in the plain order written here.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_MAXP 8
#define ORC_MAXL 40

typedef int64_t i64;

/* ------------------------------------------------------------------------- */
/* Multi-indices (Sec. III shorthand).  Enumeration: order k = 0,1,2,...;     */
/* inside an order, nx from k down to 0, then ny from k-nx down to 0.         */
/* ------------------------------------------------------------------------- */

int orc_nterms(int order)
{
    if (order < 0) return 0;
    return (order + 1) * (order + 2) * (order + 3) / 6;
}

int orc_index(int nx, int ny, int nz)
{
    int k = nx + ny + nz, m = ny + nz;
    return orc_nterms(k - 1) + m * (m + 1) / 2 + nz;
}

void orc_multi_indices(int order, int *out)
{
    int t = 0;
    for (int k = 0; k <= order; ++k)
        for (int nx = k; nx >= 0; --nx)
            for (int ny = k - nx; ny >= 0; --ny) {
                out[3 * t + 0] = nx;
                out[3 * t + 1] = ny;
                out[3 * t + 2] = k - nx - ny;
                ++t;
            }
}

static double factorial(int n)
{
    double f = 1.0;
    for (int i = 2; i <= n; ++i) f *= (double)i;
    return f;
}

static double ipow(double x, int n)
{
    double r = 1.0;
    for (int i = 0; i < n; ++i) r *= x;
    return r;
}

/* r^n / n!  for n = (a,b,c) */
static double mono(const double r[3], int a, int b, int c)
{
    return ipow(r[0], a) * ipow(r[1], b) * ipow(r[2], c) /
           (factorial(a) * factorial(b) * factorial(c));
}

typedef struct {
    int order, T;
    int *n; /* T x 3 */
} mlist;

static void mlist_make(mlist *m, int order)
{
    m->order = order;
    m->T = orc_nterms(order);
    m->n = (int *)malloc(sizeof(int) * 3 * (size_t)m->T);
    orc_multi_indices(order, m->n);
}

static void mlist_free(mlist *m) { free(m->n); m->n = NULL; }

/* ------------------------------------------------------------------------- */
/* F table of Eqs. Dn and Dnr.                                               */
/*   D_n(r) = r^-(2|n|+1) sum_{|q|=|n|} F_n(q) r^q                           */
/*   D_{n+e_v} = -d/dx_v D_n gives, for every q with F_n(q) != 0,            */
/*     F_{n+e_v}(q+e_v)         += (2|n|+1-q_v) F_n(q)                       */
/*     F_{n+e_v}(q-e_v+2e_mu)   += -q_v F_n(q)     (mu = the two other axes) */
/*   starting from F_0(0) = 1, with v the first axis such that n_v > 0.      */
/* Only the non-zero F_n(q) are kept, as the paper recommends.               */
/* ------------------------------------------------------------------------- */

typedef struct {
    int order, T;
    int *start;   /* T+1 */
    int *q;       /* nnz: index of q */
    double *val;  /* nnz */
    mlist ml;
} ftable;

static void ftable_make(ftable *F, int order)
{
    F->order = order;
    mlist_make(&F->ml, order);
    int T = F->ml.T;
    F->T = T;
    double *dense = (double *)calloc((size_t)T * (size_t)T, sizeof(double));
    dense[0] = 1.0; /* F_0(0) = 1 */
    for (int t = 1; t < T; ++t) {
        const int *n = &F->ml.n[3 * t];
        int v = (n[0] > 0) ? 0 : ((n[1] > 0) ? 1 : 2);
        int m[3] = {n[0], n[1], n[2]};
        m[v] -= 1;
        int km = m[0] + m[1] + m[2];
        int tm = orc_index(m[0], m[1], m[2]);
        for (int s = 0; s < T; ++s) {
            double f = dense[(size_t)tm * T + s];
            if (f == 0.0) continue;
            const int *q = &F->ml.n[3 * s];
            /* q + e_v */
            int a[3] = {q[0], q[1], q[2]};
            a[v] += 1;
            dense[(size_t)t * T + orc_index(a[0], a[1], a[2])] += (double)(2 * km + 1 - q[v]) * f;
            if (q[v] > 0) {
                for (int mu = 0; mu < 3; ++mu) {
                    if (mu == v) continue;
                    int b[3] = {q[0], q[1], q[2]};
                    b[v] -= 1;
                    b[mu] += 2;
                    dense[(size_t)t * T + orc_index(b[0], b[1], b[2])] += -(double)q[v] * f;
                }
            }
        }
    }
    F->start = (int *)malloc(sizeof(int) * (size_t)(T + 1));
    int nnz = 0;
    for (int t = 0; t < T; ++t)
        for (int s = 0; s < T; ++s)
            if (dense[(size_t)t * T + s] != 0.0) ++nnz;
    F->q = (int *)malloc(sizeof(int) * (size_t)(nnz > 0 ? nnz : 1));
    F->val = (double *)malloc(sizeof(double) * (size_t)(nnz > 0 ? nnz : 1));
    nnz = 0;
    for (int t = 0; t < T; ++t) {
        F->start[t] = nnz;
        for (int s = 0; s < T; ++s) {
            double f = dense[(size_t)t * T + s];
            if (f != 0.0) {
                F->q[nnz] = s;
                F->val[nnz] = f;
                ++nnz;
            }
        }
    }
    F->start[T] = nnz;
    free(dense);
}

static void ftable_free(ftable *F)
{
    free(F->start);
    free(F->q);
    free(F->val);
    mlist_free(&F->ml);
}

/* Eq. Dn: D_n(r) for every |n| <= F->order. */
static void dtensors(const ftable *F, const double r[3], double *D)
{
    double r2 = r[0] * r[0] + r[1] * r[1] + r[2] * r[2];
    double rr = sqrt(r2);
    for (int t = 0; t < F->T; ++t) {
        const int *n = &F->ml.n[3 * t];
        int k = n[0] + n[1] + n[2];
        double s = 0.0;
        for (int e = F->start[t]; e < F->start[t + 1]; ++e) {
            const int *q = &F->ml.n[3 * F->q[e]];
            s += F->val[e] * ipow(r[0], q[0]) * ipow(r[1], q[1]) * ipow(r[2], q[2]);
        }
        D[t] = s / ipow(rr, 2 * k + 1);
    }
}

void orc_D_tensors(int order, const double r[3], double *out)
{
    ftable F;
    ftable_make(&F, order);
    dtensors(&F, r, out);
    ftable_free(&F);
}

/* number of non-zero F_n(q) for the multi-index with enumeration index t */
int orc_F_nnz(int order, int t)
{
    ftable F;
    ftable_make(&F, order);
    int c = F.start[t + 1] - F.start[t];
    ftable_free(&F);
    return c;
}

/* ------------------------------------------------------------------------- */
/* Expansion operators (Sec. III).  Arrays hold T(p) coefficients in the     */
/* enumeration order above; entry 0 (Q_0, V_0) stays zero.                   */
/* ------------------------------------------------------------------------- */

/* Eq. multipolemoments: Q_n = (1/n!) sum_i m_i . grad r_i^n, with r_i taken
 * from the expansion centre c.  Since d/dx_a r^n = n_a r^(n-e_a),
 * Q_n = sum_i sum_a m_ia r_i^(n-e_a) / (n-e_a)!.  Accumulates into Q. */
static void p2m_one(const mlist *ml, int p, const double c[3], const double pos[3],
                    const double m[3], double *Q)
{
    double r[3] = {pos[0] - c[0], pos[1] - c[1], pos[2] - c[2]};
    int T = orc_nterms(p);
    for (int t = 1; t < T; ++t) {
        const int *n = &ml->n[3 * t];
        double s = 0.0;
        if (n[0] > 0) s += m[0] * mono(r, n[0] - 1, n[1], n[2]);
        if (n[1] > 0) s += m[1] * mono(r, n[0], n[1] - 1, n[2]);
        if (n[2] > 0) s += m[2] * mono(r, n[0], n[1], n[2] - 1);
        Q[t] += s;
    }
}

void orc_p2m(int p, const double c[3], i64 n, const double *pos, const double *mom, double *Q)
{
    mlist ml;
    mlist_make(&ml, p);
    for (int t = 0; t < ml.T; ++t) Q[t] = 0.0;
    for (i64 i = 0; i < n; ++i) p2m_one(&ml, p, c, &pos[3 * i], &mom[3 * i], Q);
    mlist_free(&ml);
}

/* Eq. momentshift: moments Q about the parent centre O from moments Q'
 * about the child centre c (c relative to O):  Q_n += sum_{k<=n} c^k/k! Q'_{n-k}.
 * Exact (no truncation): every term has |n-k| <= |n| <= p. */
static void m2m_one(const mlist *ml, int p, const double c[3], const double *Qc, double *Qp)
{
    int T = orc_nterms(p);
    for (int t = 0; t < T; ++t) {
        const int *n = &ml->n[3 * t];
        double s = 0.0;
        for (int kx = 0; kx <= n[0]; ++kx)
            for (int ky = 0; ky <= n[1]; ++ky)
                for (int kz = 0; kz <= n[2]; ++kz)
                    s += mono(c, kx, ky, kz) * Qc[orc_index(n[0] - kx, n[1] - ky, n[2] - kz)];
        Qp[t] += s;
    }
}

void orc_m2m(int p, const double c[3], const double *Qchild, double *Qparent)
{
    mlist ml;
    mlist_make(&ml, p);
    m2m_one(&ml, p, c, Qchild, Qparent);
    mlist_free(&ml);
}

/* Eq. taylorshift: the child's V'_n about c (c relative to the parent
 * centre) from the parent's V:  V'_n += sum_k c^k/k! V_{n+k}, over the
 * stored terms |n+k| <= p. */
static void l2l_one(const mlist *ml, int p, const double c[3], const double *Vp, double *Vc)
{
    int T = orc_nterms(p);
    for (int t = 1; t < T; ++t) {
        const int *n = &ml->n[3 * t];
        int kn = n[0] + n[1] + n[2];
        double s = 0.0;
        for (int u = 0; u < orc_nterms(p - kn); ++u) {
            const int *k = &ml->n[3 * u];
            s += mono(c, k[0], k[1], k[2]) * Vp[orc_index(n[0] + k[0], n[1] + k[1], n[2] + k[2])];
        }
        Vc[t] += s;
    }
}

void orc_l2l(int p, const double c[3], const double *Vparent, double *Vchild)
{
    mlist ml;
    mlist_make(&ml, p);
    l2l_one(&ml, p, c, Vparent, Vchild);
    mlist_free(&ml);
}

/* Eq. taylorcalc: V_n += (-1)^|n| sum_k D_{n+k}(c) Q_k, where c is the
 * centre of this (field) cell relative to the centre of the partner whose
 * moments are Q.  1<=|n|<=p, 1<=|k|<=p, and the term (n, k) only when
 * |n|+|k| <= maxdeg (maxdeg = 2p: the square truncation); D to order 2p. */
static void m2l_one(const ftable *F, int p, int maxdeg, const double c[3], const double *Q,
                    double *V, double *Dbuf)
{
    dtensors(F, c, Dbuf);
    int T = orc_nterms(p);
    const mlist *ml = &F->ml;
    for (int t = 1; t < T; ++t) {
        const int *n = &ml->n[3 * t];
        int kn = n[0] + n[1] + n[2];
        double s = 0.0;
        for (int u = 1; u < T; ++u) {
            const int *k = &ml->n[3 * u];
            if (kn + k[0] + k[1] + k[2] > maxdeg) continue;
            s += Dbuf[orc_index(n[0] + k[0], n[1] + k[1], n[2] + k[2])] * Q[u];
        }
        V[t] += ((kn % 2) ? -1.0 : 1.0) * s;
    }
}

/* maxdeg <= 0: the square truncation (2p) */
void orc_m2l_degree(int p, int maxdeg, const double c[3], const double *Q, double *V)
{
    ftable F;
    ftable_make(&F, 2 * p);
    double *D = (double *)malloc(sizeof(double) * (size_t)F.T);
    m2l_one(&F, p, maxdeg > 0 ? maxdeg : 2 * p, c, Q, V, D);
    free(D);
    ftable_free(&F);
}

void orc_m2l(int p, const double c[3], const double *Q, double *V)
{
    orc_m2l_degree(p, 2 * p, c, Q, V);
}

/* Eq. H, with the sign of H = -grad V restored:
 * H_a += -sum_{n: n_a>=1} V_n r^(n-e_a)/(n-e_a)!, r relative to the centre. */
static void l2p_one(const mlist *ml, int p, const double r[3], const double *V, double H[3])
{
    int T = orc_nterms(p);
    for (int t = 1; t < T; ++t) {
        const int *n = &ml->n[3 * t];
        if (n[0] > 0) H[0] -= V[t] * mono(r, n[0] - 1, n[1], n[2]);
        if (n[1] > 0) H[1] -= V[t] * mono(r, n[0], n[1] - 1, n[2]);
        if (n[2] > 0) H[2] -= V[t] * mono(r, n[0], n[1], n[2] - 1);
    }
}

void orc_l2p(int p, const double r[3], const double *V, double H[3])
{
    mlist ml;
    mlist_make(&ml, p);
    l2p_one(&ml, p, r, V, H);
    mlist_free(&ml);
}

/* ------------------------------------------------------------------------- */
/* Direct dipole sum (Sec. I, the O(N^2) brute force; Eq. H2 read as the     */
/* field of dipole j at i).  A source located at the field point is skipped  */
/* (Appendix, updateField), as is j == i.                                    */
/* ------------------------------------------------------------------------- */

static void pair_field(const double ri[3], const double rj[3], const double mj[3], double H[3])
{
    double d[3] = {ri[0] - rj[0], ri[1] - rj[1], ri[2] - rj[2]};
    double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
    if (r2 == 0.0) return;
    double r = sqrt(r2);
    double u[3] = {d[0] / r, d[1] / r, d[2] / r};
    double mu = mj[0] * u[0] + mj[1] * u[1] + mj[2] * u[2];
    double r3 = r2 * r;
    H[0] += (3.0 * mu * u[0] - mj[0]) / r3;
    H[1] += (3.0 * mu * u[1] - mj[1]) / r3;
    H[2] += (3.0 * mu * u[2] - mj[2]) / r3;
}

/* H at targets tgt[0..nt) (all points when tgt is NULL, nt == n). */
void orc_direct_field(i64 n, const double *pos, const double *mom, i64 nt, const i64 *tgt, double *H)
{
#pragma omp parallel for schedule(dynamic, 16)
    for (i64 t = 0; t < nt; ++t) {
        i64 i = tgt ? tgt[t] : t;
        double h[3] = {0.0, 0.0, 0.0};
        for (i64 j = 0; j < n; ++j) {
            if (j == i) continue;
            pair_field(&pos[3 * i], &pos[3 * j], &mom[3 * j], h);
        }
        H[3 * t + 0] = h[0];
        H[3 * t + 1] = h[1];
        H[3 * t + 2] = h[2];
    }
}

/* E = -1/2 sum_i m_i . H_i  (units of mu0/4pi; Appendix halves it). */
double orc_energy_from_field(i64 n, const double *mom, const double *H)
{
    double e = 0.0;
    for (i64 i = 0; i < n; ++i)
        e += mom[3 * i] * H[3 * i] + mom[3 * i + 1] * H[3 * i + 1] + mom[3 * i + 2] * H[3 * i + 2];
    return -0.5 * e;
}

/* Eq. so: the rule of thumb for the mean number of dipoles in a leaf. */
double orc_leaf_size_rule(int p)
{
    return (p > 3) ? 0.74 * (double)p * (double)p : 8.0;
}

/* Sec. IV: the error estimate e = [alpha/(2-alpha)]^p. */
double orc_error_estimate(int p, double alpha)
{
    return ipow(alpha / (2.0 - alpha), p);
}

int orc_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void orc_set_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

/* ------------------------------------------------------------------------- */
/* The tree (Sec. II, Sec. IV rule of thumb): recursive bisection into a     */
/* complete binary tree.  Cells are numbered heap-style: root 1, children    */
/* of cell c are 2c (lower half along the split axis) and 2c+1.  Level l     */
/* holds cells [2^l, 2^(l+1)); all leaves are at level L.                    */
/* ------------------------------------------------------------------------- */

typedef struct {
    i64 *v;
    i64 n, cap;
} ivec;

static void ivec_push(ivec *a, i64 x)
{
    if (a->n == a->cap) {
        a->cap = a->cap ? 2 * a->cap : 8;
        a->v = (i64 *)realloc(a->v, sizeof(i64) * (size_t)a->cap);
    }
    a->v[a->n++] = x;
}

typedef struct orc_fmm {
    i64 n;
    int p;
    int maxdeg;                 /* M2L terms with |n|+|k| <= maxdeg (2p: square) */
    double theta, leaf_size;
    double *pos, *mom;          /* copies, n x 3 */
    double lo[3], ext[3];
    int L;
    int axis[ORC_MAXL + 1];     /* axis[l]: axis split to make level l (l >= 1) */
    int nsplit[ORC_MAXL + 1][3];/* splits of each axis in the first l levels */
    i64 ncell;                  /* 2^(L+1); index 0 unused */
    i64 *leaf_of;               /* per point: leaf key in [0, 2^L) */
    i64 *leaf_start, *leaf_pts; /* CSR of points per leaf, ascending index */
    ivec *partners;             /* per cell: far list after createPartners */
    ivec *nearp;                /* per leaf cell: nearPartners */
    ftable F;                   /* to order 2p */
    double *Q, *V;              /* ncell x T(p) */
    double *H;                  /* n x 3 */
    unsigned char *have_H;      /* n */
} orc_fmm;

static int cell_level(i64 c)
{
    int l = 0;
    while ((c >> (l + 1)) != 0) ++l;
    return l;
}

/* widths of a level-l cell */
static void level_widths(const orc_fmm *f, int l, double w[3])
{
    for (int a = 0; a < 3; ++a) w[a] = f->ext[a] / ipow(2.0, f->nsplit[l][a]);
}

/* integer coordinates of cell c along each axis at its level */
static void cell_coords(const orc_fmm *f, i64 c, i64 ic[3])
{
    int l = cell_level(c);
    i64 key = c - ((i64)1 << l);
    ic[0] = ic[1] = ic[2] = 0;
    for (int j = 1; j <= l; ++j) {
        int bit = (int)((key >> (l - j)) & 1);
        int a = f->axis[j];
        ic[a] = 2 * ic[a] + bit;
    }
}

static void cell_center(const orc_fmm *f, i64 c, double cen[3])
{
    i64 ic[3];
    double w[3];
    cell_coords(f, c, ic);
    level_widths(f, cell_level(c), w);
    for (int a = 0; a < 3; ++a) cen[a] = f->lo[a] + ((double)ic[a] + 0.5) * w[a];
}

/* leaf key at depth l for one point: c_a = min(floor((x_a-lo_a)*n_a/ext_a), n_a-1) */
static i64 point_key(const orc_fmm *f, int l, const double x[3])
{
    i64 c[3];
    for (int a = 0; a < 3; ++a) {
        i64 na = (i64)1 << f->nsplit[l][a];
        double t = (x[a] - f->lo[a]) * (double)na / f->ext[a];
        i64 ca = (i64)floor(t);
        if (ca > na - 1) ca = na - 1;
        if (ca < 0) ca = 0;
        c[a] = ca;
    }
    /* interleave: level j contributes the next bit of axis[j] */
    i64 key = 0;
    int used[3] = {0, 0, 0};
    for (int j = 1; j <= l; ++j) {
        int a = f->axis[j];
        int nb = f->nsplit[l][a];
        int bit = (int)((c[a] >> (nb - 1 - used[a])) & 1);
        used[a]++;
        key = 2 * key + bit;
    }
    return key;
}

static int cmp_i64(const void *a, const void *b)
{
    i64 x = *(const i64 *)a, y = *(const i64 *)b;
    return (x > y) - (x < y);
}

static i64 count_nonempty(const orc_fmm *f, int l, i64 *scratch)
{
    for (i64 i = 0; i < f->n; ++i) scratch[i] = point_key(f, l, &f->pos[3 * i]);
    qsort(scratch, (size_t)f->n, sizeof(i64), cmp_i64);
    i64 c = 0;
    for (i64 i = 0; i < f->n; ++i)
        if (i == 0 || scratch[i] != scratch[i - 1]) ++c;
    return c;
}

/* near iff alpha = 2r/d > theta with r = |w|/2, i.e. |w|^2 > theta^2 d^2;
 * the factor (1 + 1e-12) makes a computed tie alpha == theta count as far. */
static int is_near(const orc_fmm *f, i64 a, i64 b)
{
    double w[3], ca[3], cb[3];
    level_widths(f, cell_level(a), w);
    cell_center(f, a, ca);
    cell_center(f, b, cb);
    double w2 = w[0] * w[0] + w[1] * w[1] + w[2] * w[2];
    double d2 = (ca[0] - cb[0]) * (ca[0] - cb[0]) + (ca[1] - cb[1]) * (ca[1] - cb[1]) +
                (ca[2] - cb[2]) * (ca[2] - cb[2]);
    return w2 > f->theta * f->theta * d2 * (1.0 + 1e-12);
}

/* Appendix, cell::createPartners() */
static void create_partners(orc_fmm *f, i64 c)
{
    int l = cell_level(c);
    int has_children = l < f->L;
    ivec keep = {NULL, 0, 0};
    ivec *P = &f->partners[c];
    for (i64 e = 0; e < P->n; ++e) {
        i64 A = P->v[e];
        if (is_near(f, A, c)) {
            if (has_children) {
                /* children of A into the Partners list of the children of c */
                ivec_push(&f->partners[2 * c], 2 * A);
                ivec_push(&f->partners[2 * c], 2 * A + 1);
                ivec_push(&f->partners[2 * c + 1], 2 * A);
                ivec_push(&f->partners[2 * c + 1], 2 * A + 1);
            } else {
                ivec_push(&f->nearp[c], A);
            }
            /* A is erased from the Partners list of c */
        } else {
            ivec_push(&keep, A);
        }
    }
    free(P->v);
    *P = keep;
    if (has_children) {
        ivec_push(&f->partners[2 * c], 2 * c + 1);
        ivec_push(&f->partners[2 * c + 1], 2 * c);
        create_partners(f, 2 * c);
        create_partners(f, 2 * c + 1);
    } else {
        ivec_push(&f->nearp[c], c);
    }
}

/* The box (given, or the bounding box widened by 2^-20 of its largest
 * extent) and the split sequence: at each level halve the currently widest
 * axis, ties x<y<z (Sec. IV examples).  Shared by the complete and the
 * adaptive tree. */
static void tree_geometry(i64 n, const double *pos, const double *box, double lo[3], double ext[3],
                          int axis[ORC_MAXL + 1], int nsplit[ORC_MAXL + 1][3])
{
    /* box: given, or the bounding box widened by 2^-20 of the largest extent */
    if (box) {
        for (int a = 0; a < 3; ++a) {
            lo[a] = box[a];
            ext[a] = box[3 + a] - box[a];
        }
    } else {
        double blo[3], bhi[3];
        for (int a = 0; a < 3; ++a) blo[a] = bhi[a] = pos[a];
        for (i64 i = 1; i < n; ++i)
            for (int a = 0; a < 3; ++a) {
                if (pos[3 * i + a] < blo[a]) blo[a] = pos[3 * i + a];
                if (pos[3 * i + a] > bhi[a]) bhi[a] = pos[3 * i + a];
            }
        double m = 0.0;
        for (int a = 0; a < 3; ++a)
            if (bhi[a] - blo[a] > m) m = bhi[a] - blo[a];
        if (m == 0.0) m = 1.0;
        double pad = m * ipow(0.5, 20);
        for (int a = 0; a < 3; ++a) {
            double l0 = blo[a] - pad, h0 = bhi[a] + pad;
            lo[a] = l0;
            ext[a] = h0 - l0;
        }
    }

    /* split sequence: at each level halve the currently widest axis, ties x<y<z */
    nsplit[0][0] = nsplit[0][1] = nsplit[0][2] = 0;
    axis[0] = -1;
    for (int l = 1; l <= ORC_MAXL; ++l) {
        double w[3];
        for (int b = 0; b < 3; ++b) w[b] = ext[b] / ipow(2.0, nsplit[l - 1][b]);
        int a = 0;
        if (w[1] > w[a]) a = 1;
        if (w[2] > w[a]) a = 2;
        axis[l] = a;
        for (int b = 0; b < 3; ++b) nsplit[l][b] = nsplit[l - 1][b];
        nsplit[l][a] += 1;
    }
}

orc_fmm *orc_fmm_new(i64 n, const double *pos, const double *mom, int p, double theta,
                     double leaf_size, const double *box)
{
    if (n < 1 || p < 1 || p > ORC_MAXP || !(theta > 0.0 && theta < 1.0)) return NULL;
    orc_fmm *f = (orc_fmm *)calloc(1, sizeof(orc_fmm));
    f->n = n;
    f->p = p;
    f->maxdeg = 2 * p;
    f->theta = theta;
    f->leaf_size = (leaf_size > 0.0) ? leaf_size : orc_leaf_size_rule(p);
    f->pos = (double *)malloc(sizeof(double) * 3 * (size_t)n);
    f->mom = (double *)malloc(sizeof(double) * 3 * (size_t)n);
    memcpy(f->pos, pos, sizeof(double) * 3 * (size_t)n);
    memcpy(f->mom, mom, sizeof(double) * 3 * (size_t)n);

    tree_geometry(n, pos, box, f->lo, f->ext, f->axis, f->nsplit);

    /* depth: L minimising |N/nonempty_L - s|; N/nonempty_L never increases with
     * L, so the scan stops at the first L where it is <= s. */
    i64 *scratch = (i64 *)malloc(sizeof(i64) * (size_t)n);
    double best = INFINITY;
    int bestL = 0;
    for (int l = 0; l <= ORC_MAXL; ++l) {
        double avg = (double)n / (double)count_nonempty(f, l, scratch);
        double dev = fabs(avg - f->leaf_size);
        if (dev < best) {
            best = dev;
            bestL = l;
        }
        if (avg <= f->leaf_size) break;
    }
    free(scratch);
    f->L = bestL;
    f->ncell = (i64)1 << (f->L + 1);

    /* leaf membership and per-leaf point lists */
    i64 nleaf = (i64)1 << f->L;
    f->leaf_of = (i64 *)malloc(sizeof(i64) * (size_t)n);
    f->leaf_start = (i64 *)calloc((size_t)nleaf + 1, sizeof(i64));
    f->leaf_pts = (i64 *)malloc(sizeof(i64) * (size_t)n);
    for (i64 i = 0; i < n; ++i) {
        f->leaf_of[i] = point_key(f, f->L, &pos[3 * i]);
        f->leaf_start[f->leaf_of[i] + 1]++;
    }
    for (i64 k = 0; k < nleaf; ++k) f->leaf_start[k + 1] += f->leaf_start[k];
    i64 *fill = (i64 *)malloc(sizeof(i64) * (size_t)nleaf);
    for (i64 k = 0; k < nleaf; ++k) fill[k] = f->leaf_start[k];
    for (i64 i = 0; i < n; ++i) f->leaf_pts[fill[f->leaf_of[i]]++] = i;
    free(fill);

    /* interaction lists: Appendix createPartners from the root, whose
     * Partners list starts empty */
    f->partners = (ivec *)calloc((size_t)f->ncell, sizeof(ivec));
    f->nearp = (ivec *)calloc((size_t)f->ncell, sizeof(ivec));
    create_partners(f, 1);

    ftable_make(&f->F, 2 * p);
    int T = orc_nterms(p);
    f->Q = (double *)calloc((size_t)f->ncell * T, sizeof(double));
    f->V = (double *)calloc((size_t)f->ncell * T, sizeof(double));
    f->H = (double *)calloc(3 * (size_t)n, sizeof(double));
    f->have_H = (unsigned char *)calloc((size_t)n, 1);
    return f;
}

void orc_fmm_free(orc_fmm *f)
{
    if (!f) return;
    for (i64 c = 0; c < f->ncell; ++c) {
        free(f->partners[c].v);
        free(f->nearp[c].v);
    }
    free(f->partners);
    free(f->nearp);
    free(f->pos);
    free(f->mom);
    free(f->leaf_of);
    free(f->leaf_start);
    free(f->leaf_pts);
    ftable_free(&f->F);
    free(f->Q);
    free(f->V);
    free(f->H);
    free(f->have_H);
    free(f);
}

/* Truncation of Eq. taylorcalc for later downward passes: maxdeg <= 0 is the
 * square truncation; otherwise the bound P on |n|+|k|, 2 <= P <= 2p.
 * Returns 0, or -1 (unchanged) for a bound outside that range. */
int orc_fmm_set_truncation(orc_fmm *f, int maxdeg)
{
    if (maxdeg <= 0) maxdeg = 2 * f->p;
    if (maxdeg < 2 || maxdeg > 2 * f->p) return -1;
    f->maxdeg = maxdeg;
    return 0;
}

int orc_fmm_depth(const orc_fmm *f) { return f->L; }
double orc_fmm_leaf_target(const orc_fmm *f) { return f->leaf_size; }

void orc_fmm_box(const orc_fmm *f, double out[6])
{
    for (int a = 0; a < 3; ++a) {
        out[a] = f->lo[a];
        out[3 + a] = f->lo[a] + f->ext[a];
    }
}

/* axis[1..L] into out[0..L) */
void orc_fmm_axes(const orc_fmm *f, int *out)
{
    for (int l = 1; l <= f->L; ++l) out[l - 1] = f->axis[l];
}

void orc_fmm_leaf_widths(const orc_fmm *f, double w[3]) { level_widths(f, f->L, w); }

void orc_fmm_leaf_of(const orc_fmm *f, i64 *out)
{
    memcpy(out, f->leaf_of, sizeof(i64) * (size_t)f->n);
}

i64 orc_fmm_nonempty_leaves(const orc_fmm *f)
{
    i64 c = 0, nleaf = (i64)1 << f->L;
    for (i64 k = 0; k < nleaf; ++k)
        if (f->leaf_start[k + 1] > f->leaf_start[k]) ++c;
    return c;
}

void orc_fmm_cell_center(const orc_fmm *f, i64 c, double out[3]) { cell_center(f, c, out); }

/* far pairs (cell, partner) as heap ids; returns the count, fills out when non-NULL */
i64 orc_fmm_far_pairs(const orc_fmm *f, i64 *out)
{
    i64 k = 0;
    for (i64 c = 1; c < f->ncell; ++c)
        for (i64 e = 0; e < f->partners[c].n; ++e) {
            if (out) {
                out[2 * k] = c;
                out[2 * k + 1] = f->partners[c].v[e];
            }
            ++k;
        }
    return k;
}

/* near pairs (leaf, nearPartner) as heap ids */
i64 orc_fmm_near_pairs(const orc_fmm *f, i64 *out)
{
    i64 k = 0;
    for (i64 c = 1; c < f->ncell; ++c)
        for (i64 e = 0; e < f->nearp[c].n; ++e) {
            if (out) {
                out[2 * k] = c;
                out[2 * k + 1] = f->nearp[c].v[e];
            }
            ++k;
        }
    return k;
}

/* Appendix, cell::updateMoment(): leaves by Eq. multipolemoments, other
 * cells by shifting their children's moments (Eq. momentshift). */
void orc_fmm_upward(orc_fmm *f)
{
    int T = orc_nterms(f->p);
    mlist ml;
    mlist_make(&ml, f->p);
    memset(f->Q, 0, sizeof(double) * (size_t)f->ncell * T);
    i64 nleaf = (i64)1 << f->L;
#pragma omp parallel for schedule(dynamic, 8)
    for (i64 k = 0; k < nleaf; ++k) {
        i64 c = nleaf + k;
        double cen[3];
        cell_center(f, c, cen);
        for (i64 e = f->leaf_start[k]; e < f->leaf_start[k + 1]; ++e) {
            i64 i = f->leaf_pts[e];
            p2m_one(&ml, f->p, cen, &f->pos[3 * i], &f->mom[3 * i], &f->Q[(size_t)c * T]);
        }
    }
    for (int l = f->L - 1; l >= 0; --l) {
        i64 c0 = (i64)1 << l, c1 = (i64)1 << (l + 1);
#pragma omp parallel for schedule(dynamic, 8)
        for (i64 c = c0; c < c1; ++c) {
            double cp[3];
            cell_center(f, c, cp);
            for (int b = 0; b < 2; ++b) {
                i64 ch = 2 * c + b;
                double cc[3], rel[3];
                cell_center(f, ch, cc);
                for (int a = 0; a < 3; ++a) rel[a] = cc[a] - cp[a];
                m2m_one(&ml, f->p, rel, &f->Q[(size_t)ch * T], &f->Q[(size_t)c * T]);
            }
        }
    }
    mlist_free(&ml);
}

/* Appendix, cell::updateField(): top-down, each cell inherits its parent's
 * Taylor coefficients (Eq. taylorshift) and adds its Partners' moments
 * (Eq. taylorcalc); each leaf then evaluates the smooth field (Eq. H) and the
 * near field over its nearPartners (Eq. H2).  When leaf_mask is not NULL only
 * the masked leaves (and the cells above them) are evaluated. */
void orc_fmm_downward(orc_fmm *f, const unsigned char *leaf_mask)
{
    int T = orc_nterms(f->p);
    mlist ml;
    mlist_make(&ml, f->p);
    i64 nleaf = (i64)1 << f->L;
    unsigned char *need = (unsigned char *)calloc((size_t)f->ncell, 1);
    for (i64 k = 0; k < nleaf; ++k)
        if (!leaf_mask || leaf_mask[k])
            for (i64 c = nleaf + k; c >= 1; c >>= 1) need[c] = 1;
    memset(f->V, 0, sizeof(double) * (size_t)f->ncell * T);
    memset(f->have_H, 0, (size_t)f->n);
    for (int l = 0; l <= f->L; ++l) {
        i64 c0 = (i64)1 << l, c1 = (i64)1 << (l + 1);
#pragma omp parallel for schedule(dynamic, 4)
        for (i64 c = c0; c < c1; ++c) {
            if (!need[c]) continue;
            double *V = &f->V[(size_t)c * T];
            double cen[3];
            cell_center(f, c, cen);
            if (c > 1) {
                double cpar[3], rel[3];
                cell_center(f, c / 2, cpar);
                for (int a = 0; a < 3; ++a) rel[a] = cen[a] - cpar[a];
                l2l_one(&ml, f->p, rel, &f->V[(size_t)(c / 2) * T], V);
            }
            double *Dbuf = (double *)malloc(sizeof(double) * (size_t)f->F.T);
            for (i64 e = 0; e < f->partners[c].n; ++e) {
                i64 A = f->partners[c].v[e];
                double ca[3], rel[3];
                cell_center(f, A, ca);
                for (int a = 0; a < 3; ++a) rel[a] = cen[a] - ca[a];
                m2l_one(&f->F, f->p, f->maxdeg, rel, &f->Q[(size_t)A * T], V, Dbuf);
            }
            free(Dbuf);
        }
    }
#pragma omp parallel for schedule(dynamic, 8)
    for (i64 k = 0; k < nleaf; ++k) {
        if (leaf_mask && !leaf_mask[k]) continue;
        i64 c = nleaf + k;
        double cen[3];
        cell_center(f, c, cen);
        for (i64 e = f->leaf_start[k]; e < f->leaf_start[k + 1]; ++e) {
            i64 i = f->leaf_pts[e];
            double h[3] = {0.0, 0.0, 0.0};
            double r[3] = {f->pos[3 * i] - cen[0], f->pos[3 * i + 1] - cen[1], f->pos[3 * i + 2] - cen[2]};
            l2p_one(&ml, f->p, r, &f->V[(size_t)c * T], h);
            for (i64 a = 0; a < f->nearp[c].n; ++a) {
                i64 kA = f->nearp[c].v[a] - nleaf;
                for (i64 s = f->leaf_start[kA]; s < f->leaf_start[kA + 1]; ++s) {
                    i64 j = f->leaf_pts[s];
                    if (j == i) continue;
                    pair_field(&f->pos[3 * i], &f->pos[3 * j], &f->mom[3 * j], h);
                }
            }
            f->H[3 * i] = h[0];
            f->H[3 * i + 1] = h[1];
            f->H[3 * i + 2] = h[2];
            f->have_H[i] = 1;
        }
    }
    free(need);
    mlist_free(&ml);
}

/* moments / local coefficients of every cell: ncell x T(p), heap order */
void orc_fmm_moments(const orc_fmm *f, double *out)
{
    memcpy(out, f->Q, sizeof(double) * (size_t)f->ncell * orc_nterms(f->p));
}

void orc_fmm_locals(const orc_fmm *f, double *out)
{
    memcpy(out, f->V, sizeof(double) * (size_t)f->ncell * orc_nterms(f->p));
}

/* fields in input order; points not evaluated by the last downward pass get NaN */
void orc_fmm_field(const orc_fmm *f, double *H)
{
    for (i64 i = 0; i < f->n; ++i)
        for (int a = 0; a < 3; ++a) H[3 * i + a] = f->have_H[i] ? f->H[3 * i + a] : NAN;
}

/* Appendix: the leaf energy summed over the evaluated points, halved. */
double orc_fmm_energy(const orc_fmm *f)
{
    double e = 0.0;
    for (i64 i = 0; i < f->n; ++i)
        if (f->have_H[i])
            e += f->mom[3 * i] * f->H[3 * i] + f->mom[3 * i + 1] * f->H[3 * i + 1] +
                 f->mom[3 * i + 2] * f->H[3 * i + 2];
    return -0.5 * e;
}

/* ------------------------------------------------------------------------- */
/* Ensemble time step (a project addition, not in the paper): every moment  */
/* is turned about a random axis by a random angle.  The random numbers come */
/* from the counter-based generator Philox4x64-10 (Salmon, Moraes, Dror,     */
/* Shaw, "Parallel random numbers: as easy as 1, 2, 3", SC 2011): key =      */
/* (seed, step), counter = (dipole index, 0, 0, 0).  From the four 64-bit    */
/* outputs x0..x3, u_i = (x_i >> 11) 2^-53; axis z = 1 - 2 u0,               */
/* phi = 2 pi u1, axis = (sqrt(1-z^2) cos phi, sqrt(1-z^2) sin phi, z);      */
/* angle = max_angle * u2.  The turn is Rodrigues' formula                   */
/* m' = m cos a + (k x m) sin a + k (k.m)(1 - cos a).                        */
/* ------------------------------------------------------------------------- */

static void mulhilo64(uint64_t a, uint64_t b, uint64_t *hi, uint64_t *lo)
{
    unsigned __int128 p = (unsigned __int128)a * (unsigned __int128)b;
    *hi = (uint64_t)(p >> 64);
    *lo = (uint64_t)p;
}

void orc_philox4x64(const uint64_t ctr_in[4], const uint64_t key_in[2], uint64_t out[4])
{
    const uint64_t M0 = 0xD2E7470EE14C6C93ull, M1 = 0xCA5A826395121157ull;
    const uint64_t W0 = 0x9E3779B97F4A7C15ull, W1 = 0xBB67AE8584CAA73Bull;
    uint64_t c[4] = {ctr_in[0], ctr_in[1], ctr_in[2], ctr_in[3]};
    uint64_t k[2] = {key_in[0], key_in[1]};
    for (int r = 0; r < 10; ++r) {
        uint64_t hi0, lo0, hi1, lo1;
        mulhilo64(M0, c[0], &hi0, &lo0);
        mulhilo64(M1, c[2], &hi1, &lo1);
        uint64_t n0 = hi1 ^ c[1] ^ k[0], n2 = hi0 ^ c[3] ^ k[1];
        c[0] = n0;
        c[1] = lo1;
        c[2] = n2;
        c[3] = lo0;
        k[0] += W0;
        k[1] += W1;
    }
    for (int i = 0; i < 4; ++i) out[i] = c[i];
}

/* turn moments mom[0..n) (rows of 3) in place; dipole i has global index first + i */
void orc_rotate_moments(i64 n, double *mom, uint64_t seed, uint64_t step, double max_angle, i64 first)
{
    const double two53 = 1.0 / 9007199254740992.0;
    const double pi = 3.14159265358979323846;
    for (i64 i = 0; i < n; ++i) {
        uint64_t ctr[4] = {(uint64_t)(first + i), 0, 0, 0}, key[2] = {seed, step}, x[4];
        orc_philox4x64(ctr, key, x);
        double u0 = (double)(x[0] >> 11) * two53, u1 = (double)(x[1] >> 11) * two53;
        double u2 = (double)(x[2] >> 11) * two53;
        double z = 1.0 - 2.0 * u0, phi = 2.0 * pi * u1, s = sqrt(1.0 - z * z);
        double k[3] = {s * cos(phi), s * sin(phi), z};
        double a = max_angle * u2, ca = cos(a), sa = sin(a);
        double *m = &mom[3 * i];
        double kxm[3] = {k[1] * m[2] - k[2] * m[1], k[2] * m[0] - k[0] * m[2], k[0] * m[1] - k[1] * m[0]};
        double km = k[0] * m[0] + k[1] * m[1] + k[2] * m[2];
        double r[3];
        for (int d = 0; d < 3; ++d) r[d] = m[d] * ca + kxm[d] * sa + k[d] * km * (1.0 - ca);
        m[0] = r[0];
        m[1] = r[1];
        m[2] = r[2];
    }
}

/* ------------------------------------------------------------------------- */
/* Adaptive-depth tree (a project extension; the paper's tree is complete,  */
/* Sec. II and Appendix).  Readings taken here:                             */
/*   - Cells are the uniform tree's cells (same box, split sequence and     */
/*     point membership), but a cell is split only while it holds more than */
/*     s points; empty children are not created.                             */
/*   - Two cells of different levels are near when (r_A + r_B) / d > theta, */
/*     r = half the cell diagonal, d = distance of the centres; for equal   */
/*     levels this is the paper's 2r/d > alpha_m, evaluated exactly as the  */
/*     uniform tree does.                                                   */
/*   - createPartners with unequal levels: the near candidates N(c) of a    */
/*     cell are cells of its level or coarser leaves.  A child of c takes   */
/*     as candidates the children of every internal member of N(c) (its own */
/*     sibling pair from c itself) and every leaf member as it is; a far    */
/*     candidate goes to its Partners (M2L source), a near one stays in its  */
/*     N.  At a leaf, near leaves become nearPartners (the finer cell keeps */
/*     the coarser near leaf), and a near internal cell is refined against  */
/*     the leaf: its far descendants become Partners of the leaf, its near  */
/*     leaves nearPartners.                                                 */
/* ------------------------------------------------------------------------- */

typedef struct {
    int level;
    i64 ic[3];            /* integer coordinates at its level */
    i64 parent, child[2]; /* -1 when absent */
    i64 p0, np;           /* points perm[p0 .. p0+np) */
    ivec cand, farp, nearp;
} acell;

typedef struct orc_afmm {
    i64 n;
    int p;
    double theta, s;
    double *pos, *mom;
    double lo[3], ext[3];
    int axis[ORC_MAXL + 1];
    int nsplit[ORC_MAXL + 1][3];
    acell *c;
    i64 nc, cap;
    i64 *perm;
    ftable F;
    double *Q, *V, *H;    /* nc x T(p), nc x T(p), n x 3 */
} orc_afmm;

static void a_widths(const orc_afmm *f, int l, double w[3])
{
    for (int a = 0; a < 3; ++a) w[a] = f->ext[a] / ipow(2.0, f->nsplit[l][a]);
}

static void a_center(const orc_afmm *f, i64 c, double cen[3])
{
    double w[3];
    a_widths(f, f->c[c].level, w);
    for (int a = 0; a < 3; ++a) cen[a] = f->lo[a] + ((double)f->c[c].ic[a] + 0.5) * w[a];
}

/* coordinate of x along axis a at a level with n_a = 2^ns cells (the uniform
 * tree's membership rule) */
static i64 a_coord(const orc_afmm *f, int a, int ns, double x)
{
    i64 na = (i64)1 << ns;
    double t = (x - f->lo[a]) * (double)na / f->ext[a];
    i64 ca = (i64)floor(t);
    if (ca > na - 1) ca = na - 1;
    if (ca < 0) ca = 0;
    return ca;
}

static i64 a_new_cell(orc_afmm *f)
{
    if (f->nc == f->cap) {
        f->cap = f->cap ? 2 * f->cap : 64;
        f->c = (acell *)realloc(f->c, sizeof(acell) * (size_t)f->cap);
    }
    memset(&f->c[f->nc], 0, sizeof(acell));
    f->c[f->nc].parent = f->c[f->nc].child[0] = f->c[f->nc].child[1] = -1;
    return f->nc++;
}

/* split cell c while it holds more than s points */
static void a_split(orc_afmm *f, i64 c)
{
    if ((double)f->c[c].np <= f->s || f->c[c].level >= ORC_MAXL) return;
    const int l = f->c[c].level + 1, a = f->axis[l];
    const i64 p0 = f->c[c].p0, np = f->c[c].np;
    /* stable partition by the child bit along the split axis: the lower
     * child's points, then the upper child's, each in their old order */
    i64 *tmp = (i64 *)malloc(sizeof(i64) * (size_t)np);
    i64 nlo = 0, k = 0;
    for (i64 e = 0; e < np; ++e) {
        i64 i = f->perm[p0 + e];
        if ((a_coord(f, a, f->nsplit[l][a], f->pos[3 * i + a]) & 1) == 0) tmp[k++] = i;
    }
    nlo = k;
    for (i64 e = 0; e < np; ++e) {
        i64 i = f->perm[p0 + e];
        if ((a_coord(f, a, f->nsplit[l][a], f->pos[3 * i + a]) & 1) == 1) tmp[k++] = i;
    }
    memcpy(&f->perm[p0], tmp, sizeof(i64) * (size_t)np);
    free(tmp);
    for (int side = 0; side < 2; ++side) {
        i64 cnt = side == 0 ? nlo : np - nlo;
        if (cnt == 0) continue;
        i64 ch = a_new_cell(f);
        acell *C = &f->c[c], *H = &f->c[ch];
        H->level = l;
        H->parent = c;
        for (int b = 0; b < 3; ++b) H->ic[b] = C->ic[b];
        H->ic[a] = 2 * C->ic[a] + side;
        H->p0 = side == 0 ? p0 : p0 + nlo;
        H->np = cnt;
        C->child[side] = ch;
        a_split(f, ch);
    }
}

static int a_is_leaf(const orc_afmm *f, i64 c) { return f->c[c].child[0] < 0 && f->c[c].child[1] < 0; }

static int a_near(const orc_afmm *f, i64 x, i64 y)
{
    double cx[3], cy[3], wx[3], wy[3];
    a_center(f, x, cx);
    a_center(f, y, cy);
    a_widths(f, f->c[x].level, wx);
    a_widths(f, f->c[y].level, wy);
    double d2 = 0.0;
    for (int a = 0; a < 3; ++a) d2 += (cx[a] - cy[a]) * (cx[a] - cy[a]);
    if (f->c[x].level == f->c[y].level) {
        double w2 = wx[0] * wx[0] + wx[1] * wx[1] + wx[2] * wx[2];
        return w2 > f->theta * f->theta * d2 * (1.0 + 1e-12);
    }
    double rx = 0.5 * sqrt(wx[0] * wx[0] + wx[1] * wx[1] + wx[2] * wx[2]);
    double ry = 0.5 * sqrt(wy[0] * wy[0] + wy[1] * wy[1] + wy[2] * wy[2]);
    return (rx + ry) * (rx + ry) > f->theta * f->theta * d2 * (1.0 + 1e-12);
}

static void a_consider(orc_afmm *f, i64 ci, i64 b)
{
    if (b == ci || a_near(f, ci, b))
        ivec_push(&f->c[ci].cand, b);
    else
        ivec_push(&f->c[ci].farp, b);
}

/* leaf c against the subtree of a near internal cell a */
static void a_resolve(orc_afmm *f, i64 c, i64 a)
{
    for (int s = 0; s < 2; ++s) {
        i64 b = f->c[a].child[s];
        if (b < 0) continue;
        if (!a_near(f, c, b))
            ivec_push(&f->c[c].farp, b);
        else if (a_is_leaf(f, b))
            ivec_push(&f->c[c].nearp, b);
        else
            a_resolve(f, c, b);
    }
}

static void a_partners(orc_afmm *f, i64 c)
{
    if (a_is_leaf(f, c)) {
        for (i64 e = 0; e < f->c[c].cand.n; ++e) {
            i64 a = f->c[c].cand.v[e];
            if (a == c || a_is_leaf(f, a))
                ivec_push(&f->c[c].nearp, a);
            else
                a_resolve(f, c, a);
        }
        return;
    }
    for (int s = 0; s < 2; ++s) {
        i64 ci = f->c[c].child[s];
        if (ci < 0) continue;
        for (i64 e = 0; e < f->c[c].cand.n; ++e) {
            i64 a = f->c[c].cand.v[e];
            if (a == c) {
                for (int t = 0; t < 2; ++t)
                    if (f->c[c].child[t] >= 0) a_consider(f, ci, f->c[c].child[t]);
            } else if (a_is_leaf(f, a)) {
                a_consider(f, ci, a);
            } else {
                for (int t = 0; t < 2; ++t)
                    if (f->c[a].child[t] >= 0) a_consider(f, ci, f->c[a].child[t]);
            }
        }
    }
    for (int s = 0; s < 2; ++s)
        if (f->c[c].child[s] >= 0) a_partners(f, f->c[c].child[s]);
}

/* Tree and lists for n points; s: split while a cell holds more than s
 * points; box as for the uniform tree (NULL: widened bounding box). */
orc_afmm *orc_afmm_new(i64 n, const double *pos, const double *mom, int p, double theta, double s,
                       const double *box)
{
    if (n < 1 || p < 1 || p > ORC_MAXP || !(theta > 0.0 && theta < 1.0) || !(s >= 1.0)) return NULL;
    orc_afmm *f = (orc_afmm *)calloc(1, sizeof(orc_afmm));
    f->n = n;
    f->p = p;
    f->theta = theta;
    f->s = s;
    f->pos = (double *)malloc(sizeof(double) * 3 * (size_t)n);
    f->mom = (double *)malloc(sizeof(double) * 3 * (size_t)n);
    memcpy(f->pos, pos, sizeof(double) * 3 * (size_t)n);
    memcpy(f->mom, mom, sizeof(double) * 3 * (size_t)n);
    /* the complete tree's box and split sequence */
    tree_geometry(n, pos, box, f->lo, f->ext, f->axis, f->nsplit);

    f->perm = (i64 *)malloc(sizeof(i64) * (size_t)n);
    for (i64 i = 0; i < n; ++i) f->perm[i] = i;
    i64 root = a_new_cell(f);
    f->c[root].level = 0;
    f->c[root].p0 = 0;
    f->c[root].np = n;
    a_split(f, root);
    /* lists: the root is its own near candidate */
    ivec_push(&f->c[root].cand, root);
    a_partners(f, root);

    ftable_make(&f->F, 2 * p);
    int T = orc_nterms(p);
    f->Q = (double *)calloc((size_t)f->nc * T, sizeof(double));
    f->V = (double *)calloc((size_t)f->nc * T, sizeof(double));
    f->H = (double *)calloc(3 * (size_t)n, sizeof(double));
    return f;
}

void orc_afmm_free(orc_afmm *f)
{
    if (!f) return;
    for (i64 c = 0; c < f->nc; ++c) {
        free(f->c[c].cand.v);
        free(f->c[c].farp.v);
        free(f->c[c].nearp.v);
    }
    free(f->c);
    free(f->perm);
    free(f->pos);
    free(f->mom);
    ftable_free(&f->F);
    free(f->Q);
    free(f->V);
    free(f->H);
    free(f);
}

/* children are created after their parent, so index order is top-down and
 * reverse index order bottom-up */
static void a_upward(orc_afmm *f, const mlist *ml)
{
    int T = orc_nterms(f->p);
    memset(f->Q, 0, sizeof(double) * (size_t)f->nc * T);
    for (i64 c = f->nc - 1; c >= 0; --c) {
        double cen[3];
        a_center(f, c, cen);
        double *Q = &f->Q[(size_t)c * T];
        if (a_is_leaf(f, c)) {
            /* Eq. multipolemoments about the leaf centre */
            for (i64 e = 0; e < f->c[c].np; ++e) {
                i64 i = f->perm[f->c[c].p0 + e];
                p2m_one(ml, f->p, cen, &f->pos[3 * i], &f->mom[3 * i], Q);
            }
        } else {
            /* Eq. momentshift from each child */
            for (int s = 0; s < 2; ++s) {
                i64 ch = f->c[c].child[s];
                if (ch < 0) continue;
                double cc[3], rel[3];
                a_center(f, ch, cc);
                for (int a = 0; a < 3; ++a) rel[a] = cc[a] - cen[a];
                m2m_one(ml, f->p, rel, &f->Q[(size_t)ch * T], Q);
            }
        }
    }
}

static void a_downward(orc_afmm *f, const mlist *ml)
{
    int T = orc_nterms(f->p);
    memset(f->V, 0, sizeof(double) * (size_t)f->nc * T);
    double *Dbuf = (double *)malloc(sizeof(double) * (size_t)f->F.T);
    for (i64 c = 0; c < f->nc; ++c) {
        double cen[3];
        a_center(f, c, cen);
        double *V = &f->V[(size_t)c * T];
        i64 par = f->c[c].parent;
        if (par >= 0) {
            /* Eq. taylorshift from the parent */
            double cp[3], rel[3];
            a_center(f, par, cp);
            for (int a = 0; a < 3; ++a) rel[a] = cen[a] - cp[a];
            l2l_one(ml, f->p, rel, &f->V[(size_t)par * T], V);
        }
        /* Eq. taylorcalc from every Partner (any level) */
        for (i64 e = 0; e < f->c[c].farp.n; ++e) {
            i64 b = f->c[c].farp.v[e];
            double cb[3], rel[3];
            a_center(f, b, cb);
            for (int a = 0; a < 3; ++a) rel[a] = cen[a] - cb[a];
            m2l_one(&f->F, f->p, 2 * f->p, rel, &f->Q[(size_t)b * T], V, Dbuf);
        }
        if (!a_is_leaf(f, c)) continue;
        /* Eq. H (L2P) and the near field over nearPartners, j != i */
        for (i64 e = 0; e < f->c[c].np; ++e) {
            i64 i = f->perm[f->c[c].p0 + e];
            double h[3] = {0.0, 0.0, 0.0};
            double r[3] = {f->pos[3 * i] - cen[0], f->pos[3 * i + 1] - cen[1], f->pos[3 * i + 2] - cen[2]};
            l2p_one(ml, f->p, r, V, h);
            for (i64 q = 0; q < f->c[c].nearp.n; ++q) {
                i64 b = f->c[c].nearp.v[q];
                for (i64 g = 0; g < f->c[b].np; ++g) {
                    i64 j = f->perm[f->c[b].p0 + g];
                    if (j == i) continue;
                    pair_field(&f->pos[3 * i], &f->pos[3 * j], &f->mom[3 * j], h);
                }
            }
            for (int a = 0; a < 3; ++a) f->H[3 * i + a] = h[a];
        }
    }
    free(Dbuf);
}

void orc_afmm_run(orc_afmm *f)
{
    mlist ml;
    mlist_make(&ml, f->p);
    a_upward(f, &ml);
    a_downward(f, &ml);
    mlist_free(&ml);
}

void orc_afmm_field(const orc_afmm *f, double *H) { memcpy(H, f->H, sizeof(double) * 3 * (size_t)f->n); }

double orc_afmm_energy(const orc_afmm *f)
{
    double e = 0.0;
    for (i64 i = 0; i < f->n; ++i)
        e += f->mom[3 * i] * f->H[3 * i] + f->mom[3 * i + 1] * f->H[3 * i + 1] +
             f->mom[3 * i + 2] * f->H[3 * i + 2];
    return -0.5 * e;
}

i64 orc_afmm_ncells(const orc_afmm *f) { return f->nc; }

/* multipole moments Q and Taylor coefficients V of every cell (nc x T(p),
 * the oracle's multi-index order), after orc_afmm_run */
void orc_afmm_moments(const orc_afmm *f, double *out)
{
    memcpy(out, f->Q, sizeof(double) * (size_t)f->nc * orc_nterms(f->p));
}

void orc_afmm_locals(const orc_afmm *f, double *out)
{
    memcpy(out, f->V, sizeof(double) * (size_t)f->nc * orc_nterms(f->p));
}

/* the box (lo, hi) and the level widths w[l][a], l = 0 .. ORC_MAXL */
void orc_afmm_box(const orc_afmm *f, double out[6])
{
    for (int a = 0; a < 3; ++a) {
        out[a] = f->lo[a];
        out[3 + a] = f->lo[a] + f->ext[a];
    }
}

void orc_afmm_widths(const orc_afmm *f, double *out)
{
    for (int l = 0; l <= ORC_MAXL; ++l) a_widths(f, l, &out[3 * l]);
}

/* level, parent, child0, child1, first point, point count, leaf flag */
void orc_afmm_cell(const orc_afmm *f, i64 c, i64 out[7])
{
    out[0] = f->c[c].level;
    out[1] = f->c[c].parent;
    out[2] = f->c[c].child[0];
    out[3] = f->c[c].child[1];
    out[4] = f->c[c].p0;
    out[5] = f->c[c].np;
    out[6] = a_is_leaf(f, c);
}

void orc_afmm_perm(const orc_afmm *f, i64 *out) { memcpy(out, f->perm, sizeof(i64) * (size_t)f->n); }

/* (cell, partner) pairs: kind 0 nearPartners of leaves, 1 Partners (far);
 * returns the count, fills out when non-NULL */
i64 orc_afmm_pairs(const orc_afmm *f, int kind, i64 *out)
{
    i64 k = 0;
    for (i64 c = 0; c < f->nc; ++c) {
        const ivec *v = kind ? &f->c[c].farp : &f->c[c].nearp;
        for (i64 e = 0; e < v->n; ++e) {
            if (out) {
                out[2 * k] = c;
                out[2 * k + 1] = v->v[e];
            }
            ++k;
        }
    }
    return k;
}
