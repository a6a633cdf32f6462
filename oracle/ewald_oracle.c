/*
 * Plain FP64 CPU oracle for periodic Ewald summation (TEST INFRASTRUCTURE).
 *
 * This file is the correctness reference for the GPU library.  Only the
 * tests, the package smoke check and the benchmark's CPU-baseline leg may
 * load it; the product path never calls it.  It shares no code, header,
 * table or constant with the CUDA path.
 *
 * What it computes (Thorpe, Smith, Hasnip & Drummond, "Acceleration of the
 * CASINO quantum Monte Carlo software using GPUs and OpenACC", Sec. 2.2:
 * Eqs. (2)-(4) for 3D, Eqs. (5)-(6) for 2D with every charge at z = 0):
 *
 *   V = sum_{i<j} q_i q_j v_E(r_i - r_j) + 1/2 sum_j q_j^2 v_M
 *
 * written with alpha = sqrt(paper gamma) so that the screening function is
 * erfc(alpha r).  Expanding v_E and v_M and collecting terms gives five
 * pieces, each returned separately:
 *
 *   E_real  = sum_{i<j} q_i q_j sum_{R : |d_ij+R| < r_c} erfc(alpha|d_ij+R|)/|d_ij+R|
 *   E_madR  = 1/2 sum_i q_i^2 sum_{R != 0, |R| < r_c} erfc(alpha|R|)/|R|
 *   E_recip = C sum_{G != 0, |G| <= g_c} f(G) |rho(G)|^2,  rho(G) = sum_i q_i e^{iG.r_i}
 *             3D: C = 2 pi / Omega,  f(G) = exp(-G^2/(4 alpha^2)) / G^2
 *             2D: C = pi / A,        f(G) = erfc(G/(2 alpha)) / G
 *   E_self  = -(alpha/sqrt(pi)) sum_i q_i^2
 *   E_bg    = 3D: -pi Q^2 / (2 Omega alpha^2);   2D: -sqrt(pi) Q^2 / (A alpha)
 *
 * (Q = sum_i q_i.)  The reciprocal pieces of v_E and v_M combine into
 * (C) sum_G f |rho|^2 because |rho|^2 = sum_j q_j^2 + 2 sum_{i<j} q_i q_j cos(G.r_ij);
 * the constant -pi/(Omega gamma) of 3D v_E and v_M sums to the background
 * term; -2 sqrt(gamma/pi) of v_M is the self term.  In 2D at z = 0 the two
 * erfc terms of the reciprocal sum coincide and the bracket of v_E reduces
 * to 1/(alpha sqrt(pi)).
 *
 * oracle_energy_z / oracle_delta_e_z (end of the file) take 2D cells whose
 * charges sit at heights z != 0 (layers), from the pair definition.
 *
 * The single-particle move (Sec. 2.1: VMC and DMC sampling keep asking for the
 * potential-energy change of a one-particle move) is computed by
 * oracle_delta_e straight from its definition, with its own rho(G).
 *
 * Everything is a literal double loop: every lattice vector R whose integer
 * coordinates could place d+R inside the cutoff sphere is visited, and every
 * G vector (both +G and -G) inside the G sphere is summed with direct
 * cos/sin per particle.  No blocking, no recurrences, no symmetry tricks.
 *
 * Parity status: pinned (bcc and hexagonal Wigner-crystal Madelung energies,
 * rocksalt Madelung constant, alpha independence, invariances, supercell
 * consistency, continuity of v_E - 1/r, brute-force rho identity, move dE
 * against two full energies).
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#define ORC_OK 0
#define ORC_ERR_ARG 1
#define ORC_ERR_LATTICE 2
#define ORC_ERR_COINCIDENT 3

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

typedef struct {
    int dim;
    double a[3][3]; /* a[i] = lattice vector i (rows), unused components 0 */
    double b[3][3]; /* b[j] = reciprocal vector j, a_i . b_j = 2 pi delta_ij */
    double vol;     /* |volume| (3D) or |area| (2D) */
} cell_t;

/*
 * Compensated (Neumaier) running sum.  The long sums of the energy (over
 * ~5e5 particle pairs, over thousands of G vectors) would otherwise carry a
 * rounding error of ~1e-10 of their size, above the 1e-12 relative parity
 * gate; compensation keeps the oracle's own error near one rounding.
 */
typedef struct { double s, c; } ksum_t;

static void kadd(ksum_t *k, double x) {
    double t = k->s + x;
    if (fabs(k->s) >= fabs(x)) k->c += (k->s - t) + x;
    else k->c += (x - t) + k->s;
    k->s = t;
}

static double kval(const ksum_t *k) { return k->s + k->c; }

static double dot(int dim, const double *x, const double *y) {
    double s = 0.0;
    for (int k = 0; k < dim; ++k) s += x[k] * y[k];
    return s;
}

static double norm(int dim, const double *x) { return sqrt(dot(dim, x, x)); }

/* Reciprocal lattice from cross products (3D) or the 2D rotation. */
static int make_cell(int dim, const double *lat, cell_t *c) {
    if (dim != 2 && dim != 3) return ORC_ERR_ARG;
    memset(c, 0, sizeof(*c));
    c->dim = dim;
    for (int i = 0; i < dim; ++i)
        for (int k = 0; k < dim; ++k) c->a[i][k] = lat[i * dim + k];
    if (dim == 3) {
        double *a1 = c->a[0], *a2 = c->a[1], *a3 = c->a[2];
        double c23[3] = {a2[1] * a3[2] - a2[2] * a3[1], a2[2] * a3[0] - a2[0] * a3[2],
                         a2[0] * a3[1] - a2[1] * a3[0]};
        double c31[3] = {a3[1] * a1[2] - a3[2] * a1[1], a3[2] * a1[0] - a3[0] * a1[2],
                         a3[0] * a1[1] - a3[1] * a1[0]};
        double c12[3] = {a1[1] * a2[2] - a1[2] * a2[1], a1[2] * a2[0] - a1[0] * a2[2],
                         a1[0] * a2[1] - a1[1] * a2[0]};
        double v = a1[0] * c23[0] + a1[1] * c23[1] + a1[2] * c23[2];
        if (!(fabs(v) > 0.0)) return ORC_ERR_LATTICE;
        for (int k = 0; k < 3; ++k) {
            c->b[0][k] = 2.0 * M_PI * c23[k] / v;
            c->b[1][k] = 2.0 * M_PI * c31[k] / v;
            c->b[2][k] = 2.0 * M_PI * c12[k] / v;
        }
        c->vol = fabs(v);
    } else {
        double *a1 = c->a[0], *a2 = c->a[1];
        double s = a1[0] * a2[1] - a1[1] * a2[0];
        if (!(fabs(s) > 0.0)) return ORC_ERR_LATTICE;
        c->b[0][0] = 2.0 * M_PI * a2[1] / s;
        c->b[0][1] = -2.0 * M_PI * a2[0] / s;
        c->b[1][0] = -2.0 * M_PI * a1[1] / s;
        c->b[1][1] = 2.0 * M_PI * a1[0] / s;
        c->vol = fabs(s);
    }
    return ORC_OK;
}

/* Displacement d brought to fractional coordinates in [-1/2, 1/2]. */
static void wrap(const cell_t *c, const double *d, double *dw) {
    int dim = c->dim;
    double f[3] = {0, 0, 0};
    for (int k = 0; k < dim; ++k) {
        f[k] = dot(dim, c->b[k], d) / (2.0 * M_PI);
        f[k] -= nearbyint(f[k]);
    }
    for (int x = 0; x < dim; ++x) {
        dw[x] = 0.0;
        for (int k = 0; k < dim; ++k) dw[x] += f[k] * c->a[k][x];
    }
}

/*
 * Sum over lattice vectors R of erfc(alpha|d+R|)/|d+R| for |d+R| < r_c.
 * d is wrapped first; any R with |d+R| < r_c has |R| < r_c + |d| and hence
 * integer coordinates |m_k| = |R.b_k|/2pi <= (r_c + |d|)|b_k|/2pi, so the box
 * below contains every contributing R.  skip_origin drops R = 0 (used for the
 * Madelung self-image sum).  Returns ORC_ERR_COINCIDENT if some |d+R| is
 * below 1e-10 of the cell's length scale (two particles on top of each other
 * up to the rounding of the wrap).
 */
static int image_sum(const cell_t *c, const double *d, double alpha, double r_c,
                     int skip_origin, double *out) {
    int dim = c->dim;
    double dw[3] = {0, 0, 0};
    wrap(c, d, dw);
    double dn = norm(dim, dw);
    int mmax[3] = {0, 0, 0};
    for (int k = 0; k < dim; ++k)
        mmax[k] = (int)ceil((r_c + dn) * norm(dim, c->b[k]) / (2.0 * M_PI));
    double s = 0.0;
    int m[3];
    for (m[0] = -mmax[0]; m[0] <= mmax[0]; ++m[0])
        for (m[1] = -mmax[1]; m[1] <= mmax[1]; ++m[1])
            for (m[2] = -mmax[2]; m[2] <= mmax[2]; ++m[2]) {
                if (skip_origin && m[0] == 0 && m[1] == 0 && m[2] == 0) continue;
                double x[3] = {0, 0, 0};
                for (int y = 0; y < dim; ++y) {
                    x[y] = dw[y];
                    for (int k = 0; k < dim; ++k) x[y] += m[k] * c->a[k][y];
                }
                double r = norm(dim, x);
                if (r < r_c) {
                    if (r < 1e-10 * pow(c->vol, 1.0 / dim)) return ORC_ERR_COINCIDENT;
                    s += erfc(alpha * r) / r;
                }
            }
    *out = s;
    return ORC_OK;
}

/* Reciprocal weight f(G) of the 3D and 2D sums. */
static double recip_weight(int dim, double g, double alpha) {
    if (dim == 3) return exp(-g * g / (4.0 * alpha * alpha)) / (g * g);
    return erfc(g / (2.0 * alpha)) / g;
}

static double recip_prefactor(const cell_t *c) {
    return c->dim == 3 ? 2.0 * M_PI / c->vol : M_PI / c->vol;
}

/*
 * Visit every G = sum_k n_k b_k with 0 < |G| <= g_c.  Since n_k = G.a_k/2pi,
 * |n_k| <= g_c |a_k| / 2pi bounds the box.  The callback gets G and |G|.
 */
typedef void (*gvisit_fn)(const double *G, double g, const int *n, void *ctx);

static void for_each_g(const cell_t *c, double g_c, gvisit_fn fn, void *ctx) {
    int dim = c->dim;
    int nmax[3] = {0, 0, 0};
    for (int k = 0; k < dim; ++k)
        nmax[k] = (int)ceil(g_c * norm(dim, c->a[k]) / (2.0 * M_PI));
    int n[3];
    for (n[0] = -nmax[0]; n[0] <= nmax[0]; ++n[0])
        for (n[1] = -nmax[1]; n[1] <= nmax[1]; ++n[1])
            for (n[2] = -nmax[2]; n[2] <= nmax[2]; ++n[2]) {
                if (n[0] == 0 && n[1] == 0 && n[2] == 0) continue;
                double G[3] = {0, 0, 0};
                for (int y = 0; y < dim; ++y)
                    for (int k = 0; k < dim; ++k) G[y] += n[k] * c->b[k][y];
                double g = norm(dim, G);
                if (g <= g_c) fn(G, g, n, ctx);
            }
}

typedef struct {
    int dim, n;
    const double *pos, *q;
    double alpha;
    ksum_t sum;
    long count;
} recip_ctx;

/* f(G) |rho(G)|^2 with rho summed directly with cos and sin. */
static void visit_recip(const double *G, double g, const int *nvec, void *vctx) {
    (void)nvec;
    recip_ctx *r = (recip_ctx *)vctx;
    double re = 0.0, im = 0.0;
    for (int i = 0; i < r->n; ++i) {
        double ph = dot(r->dim, G, r->pos + (size_t)i * r->dim);
        re += r->q[i] * cos(ph);
        im += r->q[i] * sin(ph);
    }
    kadd(&r->sum, recip_weight(r->dim, g, r->alpha) * (re * re + im * im));
    r->count += 1;
}

/* f(G) sum_{i,j} q_i q_j cos(G.(r_i - r_j)): the same sum without rho. */
static void visit_recip_pairs(const double *G, double g, const int *nvec, void *vctx) {
    (void)nvec;
    recip_ctx *r = (recip_ctx *)vctx;
    double s = 0.0;
    for (int i = 0; i < r->n; ++i)
        for (int j = 0; j < r->n; ++j) {
            double d[3] = {0, 0, 0};
            for (int y = 0; y < r->dim; ++y)
                d[y] = r->pos[(size_t)i * r->dim + y] - r->pos[(size_t)j * r->dim + y];
            s += r->q[i] * r->q[j] * cos(dot(r->dim, G, d));
        }
    kadd(&r->sum, recip_weight(r->dim, g, r->alpha) * s);
    r->count += 1;
}

static void visit_count(const double *G, double g, const int *nvec, void *vctx) {
    (void)G; (void)g; (void)nvec;
    ((recip_ctx *)vctx)->count += 1;
}

static int check_common(int dim, const double *lattice, int n, const double *pos,
                        const double *q, double alpha, double r_c, double g_c) {
    if ((dim != 2 && dim != 3) || !lattice || n < 1 || !pos || !q) return ORC_ERR_ARG;
    if (!(alpha > 0.0) || !(r_c > 0.0) || !(g_c > 0.0)) return ORC_ERR_ARG;
    return ORC_OK;
}

/*
 * Full Ewald energy of one configuration.  comp (may be NULL) receives
 * {E_real, E_madR, E_recip, E_self, E_bg}; *e receives their sum.
 */
int oracle_energy(int dim, const double *lattice, int n, const double *pos, const double *q,
                  double alpha, double r_c, double g_c, double *comp, double *e) {
    int st = check_common(dim, lattice, n, pos, q, alpha, r_c, g_c);
    if (st) return st;
    cell_t c;
    if ((st = make_cell(dim, lattice, &c))) return st;

    ksum_t e_real_sum = {0.0, 0.0};
    for (int i = 0; i < n; ++i)
        for (int j = i + 1; j < n; ++j) {
            double d[3] = {0, 0, 0}, s;
            for (int y = 0; y < dim; ++y)
                d[y] = pos[(size_t)i * dim + y] - pos[(size_t)j * dim + y];
            if ((st = image_sum(&c, d, alpha, r_c, 0, &s))) return st;
            kadd(&e_real_sum, q[i] * q[j] * s);
        }
    double e_real = kval(&e_real_sum);

    double zero[3] = {0, 0, 0}, smad, q2 = 0.0, qsum = 0.0;
    if ((st = image_sum(&c, zero, alpha, r_c, 1, &smad))) return st;
    for (int i = 0; i < n; ++i) {
        q2 += q[i] * q[i];
        qsum += q[i];
    }
    double e_madR = 0.5 * q2 * smad;

    recip_ctx rc = {dim, n, pos, q, alpha, {0.0, 0.0}, 0};
    for_each_g(&c, g_c, visit_recip, &rc);
    double e_recip = recip_prefactor(&c) * kval(&rc.sum);

    double e_self = -alpha / sqrt(M_PI) * q2;
    double e_bg = dim == 3 ? -M_PI * qsum * qsum / (2.0 * c.vol * alpha * alpha)
                           : -sqrt(M_PI) * qsum * qsum / (c.vol * alpha);
    if (comp) {
        comp[0] = e_real;
        comp[1] = e_madR;
        comp[2] = e_recip;
        comp[3] = e_self;
        comp[4] = e_bg;
    }
    *e = e_real + e_madR + e_recip + e_self + e_bg;
    return ORC_OK;
}

/*
 * Change of the Ewald energy when particle k moves to r_new, computed
 * directly: the pair terms of k with every other particle at the new and old
 * positions, and the reciprocal sum with rho and rho + delta, where
 * delta(G) = q_k (e^{iG.r_new} - e^{iG.r_k}).  The Madelung, self and
 * background pieces do not depend on positions and cancel.
 */
typedef struct {
    int dim, n, k;
    const double *pos, *q, *r_new;
    double alpha;
    ksum_t sum;
} move_ctx;

static void visit_move(const double *G, double g, const int *nvec, void *vctx) {
    (void)nvec;
    move_ctx *m = (move_ctx *)vctx;
    double re = 0.0, im = 0.0;
    for (int i = 0; i < m->n; ++i) {
        double ph = dot(m->dim, G, m->pos + (size_t)i * m->dim);
        re += m->q[i] * cos(ph);
        im += m->q[i] * sin(ph);
    }
    double ph_new = dot(m->dim, G, m->r_new);
    double ph_old = dot(m->dim, G, m->pos + (size_t)m->k * m->dim);
    double dre = m->q[m->k] * (cos(ph_new) - cos(ph_old));
    double dim_ = m->q[m->k] * (sin(ph_new) - sin(ph_old));
    double after = (re + dre) * (re + dre) + (im + dim_) * (im + dim_);
    double before = re * re + im * im;
    kadd(&m->sum, recip_weight(m->dim, g, m->alpha) * (after - before));
}

/* The move's real-space and reciprocal-space parts separately (their sum is
 * oracle_delta_e's result); the parts set the scale of a move's energy
 * change against which its rounding is judged. */
int oracle_delta_e_parts(int dim, const double *lattice, int n, const double *pos, const double *q,
                         int k, const double *r_new, double alpha, double r_c, double g_c,
                         double *de_real, double *de_recip) {
    int st = check_common(dim, lattice, n, pos, q, alpha, r_c, g_c);
    if (st) return st;
    if (k < 0 || k >= n || !r_new || !de_real || !de_recip) return ORC_ERR_ARG;
    cell_t c;
    if ((st = make_cell(dim, lattice, &c))) return st;

    ksum_t d_real = {0.0, 0.0};
    for (int j = 0; j < n; ++j) {
        if (j == k) continue;
        double dn[3] = {0, 0, 0}, dold[3] = {0, 0, 0}, sn, so;
        for (int y = 0; y < dim; ++y) {
            dn[y] = r_new[y] - pos[(size_t)j * dim + y];
            dold[y] = pos[(size_t)k * dim + y] - pos[(size_t)j * dim + y];
        }
        if ((st = image_sum(&c, dn, alpha, r_c, 0, &sn))) return st;
        if ((st = image_sum(&c, dold, alpha, r_c, 0, &so))) return st;
        kadd(&d_real, q[k] * q[j] * (sn - so));
    }
    move_ctx mc = {dim, n, k, pos, q, r_new, alpha, {0.0, 0.0}};
    for_each_g(&c, g_c, visit_move, &mc);
    *de_real = kval(&d_real);
    *de_recip = recip_prefactor(&c) * kval(&mc.sum);
    return ORC_OK;
}

int oracle_delta_e(int dim, const double *lattice, int n, const double *pos, const double *q,
                   int k, const double *r_new, double alpha, double r_c, double g_c,
                   double *de) {
    if (!de) return ORC_ERR_ARG;
    double re = 0.0, rc = 0.0;
    int st = oracle_delta_e_parts(dim, lattice, n, pos, q, k, r_new, alpha, r_c, g_c, &re, &rc);
    if (st) return st;
    *de = re + rc;
    return ORC_OK;
}

/* rho(G) = sum_i q_i e^{iG.r_i} at the integer G coordinates nvec[g][dim]. */
int oracle_rho_at(int dim, const double *lattice, int n, const double *pos, const double *q,
                  int n_g, const int *nvec, double *rho /* [n_g][2] */) {
    if ((dim != 2 && dim != 3) || !lattice || n < 0 || n_g < 0 || !nvec || !rho)
        return ORC_ERR_ARG;
    cell_t c;
    int st = make_cell(dim, lattice, &c);
    if (st) return st;
    for (int g = 0; g < n_g; ++g) {
        double G[3] = {0, 0, 0};
        for (int y = 0; y < dim; ++y)
            for (int k = 0; k < dim; ++k) G[y] += nvec[(size_t)g * dim + k] * c.b[k][y];
        double re = 0.0, im = 0.0;
        for (int i = 0; i < n; ++i) {
            double ph = dot(dim, G, pos + (size_t)i * dim);
            re += q[i] * cos(ph);
            im += q[i] * sin(ph);
        }
        rho[2 * g] = re;
        rho[2 * g + 1] = im;
    }
    return ORC_OK;
}

/* E_recip written as the double sum over particle pairs (no rho). */
int oracle_recip_pairsum(int dim, const double *lattice, int n, const double *pos,
                         const double *q, double alpha, double g_c, double *e_recip) {
    if ((dim != 2 && dim != 3) || !lattice || n < 1 || !pos || !q || !(alpha > 0) ||
        !(g_c > 0) || !e_recip)
        return ORC_ERR_ARG;
    cell_t c;
    int st = make_cell(dim, lattice, &c);
    if (st) return st;
    recip_ctx rc = {dim, n, pos, q, alpha, {0.0, 0.0}, 0};
    for_each_g(&c, g_c, visit_recip_pairs, &rc);
    *e_recip = recip_prefactor(&c) * kval(&rc.sum);
    return ORC_OK;
}

/* Number of G != 0 with |G| <= g_c (both members of each +-G pair). */
long oracle_gcount(int dim, const double *lattice, double g_c) {
    cell_t c;
    if (make_cell(dim, lattice, &c)) return -1;
    recip_ctx rc = {dim, 0, NULL, NULL, 1.0, {0.0, 0.0}, 0};
    for_each_g(&c, g_c, visit_count, &rc);
    return rc.count;
}

/*
 * Cutoffs from a tolerance: erfc(alpha r_c) = tol for real space; for
 * reciprocal space exp(-g_c^2/(4 alpha^2)) = tol in 3D and
 * erfc(g_c/(2 alpha)) = tol in 2D.  erfc is inverted by bisection.
 */
static double erfc_inverse(double tol) {
    double lo = 0.0, hi = 30.0;
    for (int it = 0; it < 200; ++it) {
        double mid = 0.5 * (lo + hi);
        if (erfc(mid) > tol) lo = mid; else hi = mid;
    }
    return 0.5 * (lo + hi);
}

int oracle_cutoffs(int dim, double alpha, double tol, double *r_c, double *g_c) {
    if ((dim != 2 && dim != 3) || !(alpha > 0) || !(tol > 0 && tol < 1) || !r_c || !g_c)
        return ORC_ERR_ARG;
    double x = erfc_inverse(tol);
    *r_c = x / alpha;
    *g_c = dim == 3 ? 2.0 * alpha * sqrt(-log(tol)) : 2.0 * alpha * x;
    return ORC_OK;
}

/* ------------------------------------------------------------------------
 * Two-body plane-wave Jastrow term p (paper Sec. 2.3, Eqs. (7), (9)):
 *
 *   J_p = sum_{i<j} p(r_i - r_j),   p(r) = sum_{m=1}^{N_p} a_m sum_{G in star_m^+} cos(G.r)
 *
 * A star is read here as a shell of simulation-cell reciprocal-lattice
 * vectors of equal length (relative tolerance 1e-9), shells counted from the
 * shortest nonzero |G|; star_m^+ holds one of each +-G pair, so the oracle
 * sums the whole shell (both signs) with a factor 1/2.  cos is periodic, so
 * r_i - r_j needs no wrapping.  Derivatives by particle i:
 *
 *   grad_i J_p = sum_{j != i} sum_m a_m sum_{G in star_m^+} (-sin(G.(r_i - r_j))) G
 *   lap_i  J_p = sum_{j != i} sum_m a_m sum_{G in star_m^+} (-|G|^2) cos(G.(r_i - r_j))
 *
 * Plain double loops over pairs and G vectors, cos and sin of each phase.
 * ---------------------------------------------------------------------- */

typedef struct {
    double *g;
    long n, cap;
} glist_t;

static void visit_collect(const double *G, double g, const int *nvec, void *vctx) {
    (void)G;
    (void)nvec;
    glist_t *l = (glist_t *)vctx;
    if (l->n == l->cap) {
        l->cap = l->cap ? 2 * l->cap : 256;
        l->g = (double *)realloc(l->g, (size_t)l->cap * sizeof(double));
    }
    l->g[l->n++] = g;
}

static int cmp_double(const void *a, const void *b) {
    double x = *(const double *)a, y = *(const double *)b;
    return (x > y) - (x < y);
}

/* Shell radii: radius[m] for m = 0 .. n_stars-1.  Grows the search sphere
 * until it holds n_stars shells completely (all G with |G| <= g are visited). */
static int star_radii(const cell_t *c, int n_stars, double *radius) {
    double g = 0.0;
    for (int k = 0; k < c->dim; ++k) g = fmax(g, norm(c->dim, c->b[k]));
    for (int iter = 0; iter < 40; ++iter, g *= 1.5) {
        glist_t l = {NULL, 0, 0};
        for_each_g(c, g, visit_collect, &l);
        qsort(l.g, (size_t)l.n, sizeof(double), cmp_double);
        int m = 0;
        for (long i = 0; i < l.n && m < n_stars; ++i)
            if (m == 0 || l.g[i] > radius[m - 1] * (1.0 + 1e-9)) radius[m++] = l.g[i];
        free(l.g);
        if (m >= n_stars) return ORC_OK;
    }
    return ORC_ERR_ARG;
}

static int star_of(const double *radius, int n_stars, double g) {
    for (int m = 0; m < n_stars; ++m)
        if (fabs(g / radius[m] - 1.0) <= 1e-9) return m;
    return -1;
}

/* Every G of the first n_stars shells (both signs): nvec[i][dim] integer
 * coordinates on the reciprocal basis and star[i] (0-based shell index).
 * *n_g receives the count; at most max_g entries are written. */
typedef struct {
    int dim, n_stars, max_g, count;
    const double *radius;
    int *nvec, *star;
} starlist_t;

static void visit_star_list(const double *G, double g, const int *nvec, void *vctx) {
    (void)G;
    starlist_t *s = (starlist_t *)vctx;
    int m = star_of(s->radius, s->n_stars, g);
    if (m < 0) return;
    if (s->count < s->max_g) {
        for (int k = 0; k < s->dim; ++k) s->nvec[s->count * s->dim + k] = nvec[k];
        s->star[s->count] = m;
    }
    s->count++;
}

int oracle_jastrow_stars(int dim, const double *lattice, int n_stars, int max_g, int *n_g, int *nvec,
                         int *star) {
    cell_t c;
    if (n_stars < 1 || !n_g) return ORC_ERR_ARG;
    int st = make_cell(dim, lattice, &c);
    if (st) return st;
    double *radius = (double *)malloc((size_t)n_stars * sizeof(double));
    st = star_radii(&c, n_stars, radius);
    if (!st) {
        starlist_t s = {dim, n_stars, max_g, 0, radius, nvec, star};
        for_each_g(&c, radius[n_stars - 1] * (1.0 + 1e-9), visit_star_list, &s);
        *n_g = s.count;
    }
    free(radius);
    return st;
}

typedef struct {
    int dim, n, n_stars;
    const double *pos, *a, *radius;
    ksum_t j;
    ksum_t *grad, *lap;
} jp_ctx;

static void visit_jastrow(const double *G, double g, const int *nvec, void *vctx) {
    (void)nvec;
    jp_ctx *c = (jp_ctx *)vctx;
    int m = star_of(c->radius, c->n_stars, g);
    if (m < 0) return;
    const double w = 0.5 * c->a[m];  /* the whole shell, both signs */
    const int dim = c->dim;
    for (int i = 0; i < c->n; ++i)
        for (int j = 0; j < c->n; ++j) {
            if (i == j) continue;
            double ph = 0.0;
            for (int k = 0; k < dim; ++k) ph += G[k] * (c->pos[i * dim + k] - c->pos[j * dim + k]);
            const double cs = cos(ph), sn = sin(ph);
            if (i < j) kadd(&c->j, w * cs);
            if (c->grad)
                for (int k = 0; k < dim; ++k) kadd(&c->grad[i * dim + k], -w * sn * G[k]);
            if (c->lap) kadd(&c->lap[i], -w * g * g * cs);
        }
}

int oracle_jastrow_p(int dim, const double *lattice, int n, const double *pos, int n_stars, const double *a,
                     double *j_out, double *grad, double *lap) {
    cell_t c;
    if (n < 1 || n_stars < 1 || !pos || !a || !j_out) return ORC_ERR_ARG;
    int st = make_cell(dim, lattice, &c);
    if (st) return st;
    double *radius = (double *)malloc((size_t)n_stars * sizeof(double));
    ksum_t *gs = grad ? (ksum_t *)calloc((size_t)n * dim, sizeof(ksum_t)) : NULL;
    ksum_t *ls = lap ? (ksum_t *)calloc((size_t)n, sizeof(ksum_t)) : NULL;
    st = star_radii(&c, n_stars, radius);
    if (!st) {
        jp_ctx ctx = {dim, n, n_stars, pos, a, radius, {0, 0}, gs, ls};
        for_each_g(&c, radius[n_stars - 1] * (1.0 + 1e-9), visit_jastrow, &ctx);
        *j_out = kval(&ctx.j);
        for (int i = 0; grad && i < n * dim; ++i) grad[i] = kval(&gs[i]);
        for (int i = 0; lap && i < n; ++i) lap[i] = kval(&ls[i]);
    }
    free(radius);
    free(gs);
    free(ls);
    return st;
}

/* ===================================================================== */
/*
 * Two-dimensional cell with every charge at a height z above the plane
 * (Sec. 2.2, Eqs. (5)-(6) with z != 0: layered systems such as bilayers).
 * Positions are in-plane [n][2], heights z[n].  The energy is the pair sum
 * of the definition, pair by pair:
 *
 *   V = sum_{i<j} q_i q_j v_E(rho_ij, z_ij) + 1/2 sum_j q_j^2 v_M
 *
 *   v_E(rho, z) = (pi/A) sum_{G != 0} F(G, z) e^{iG.rho}
 *               + sum_R erfc(alpha |(rho + R, z)|) / |(rho + R, z)|
 *               - (2 pi/A) [z erf(alpha z) + e^{-alpha^2 z^2} / (alpha sqrt(pi))]
 *   F(G, z)     = [e^{zG} erfc(G/(2 alpha) + z alpha) + e^{-zG} erfc(G/(2 alpha) - z alpha)] / G
 *   v_M         = Eq. (6), as in oracle_energy's 2D case.
 *
 * The five pieces returned (same order as oracle_energy):
 *   E_real  = sum_{i<j} q_i q_j sum_R erfc(alpha r)/r,  r = |(rho_ij + R, z_ij)| < r_c
 *   E_madR  = 1/2 sum q^2 sum_{R != 0, |R| < r_c} erfc(alpha R)/R
 *   E_recip = (pi/A) sum_{G != 0, |G| <= g_c} [sum_{i<j} q_i q_j F(G, z_ij) cos(G.rho_ij)
 *                                               + 1/2 sum_i q_i^2 F(G, 0)]
 *   E_self  = -(alpha/sqrt(pi)) sum q^2
 *   E_bg    = -(2 pi/A) [sum_{i<j} q_i q_j g(z_ij) + 1/2 sum_i q_i^2 g(0)],
 *             g(z) = z erf(alpha z) + e^{-alpha^2 z^2} / (alpha sqrt(pi))
 *
 * (F(G, 0) = 2 erfc(G/2alpha)/G and g(0) = 1/(alpha sqrt(pi)) give v_M's
 * reciprocal and background constants.)  With every z equal this is
 * oracle_energy's 2D result.  F is evaluated as printed, which needs
 * e^{|z|G} to stay finite: the call refuses |z_ij| g_c > 600.
 *
 * Parity status: pinned (reduction to the z = 0 energy, alpha independence
 * with z != 0, the Fourier series of a charged sheet lattice for z != 0,
 * the charged-sheet limit at large separation, invariances, move dE).
 */
static double parry_f(double g, double z, double alpha) {
    z = fabs(z);
    double a = g / (2.0 * alpha), b = z * alpha;
    return (exp(z * g) * erfc(a + b) + exp(-z * g) * erfc(a - b)) / g;
}

static double sheet_g(double z, double alpha) {
    return z * erf(alpha * z) + exp(-alpha * alpha * z * z) / (alpha * sqrt(M_PI));
}

/* Sum over in-plane lattice vectors R of erfc(alpha r)/r, r = |(d + R, z)| < r_c. */
static int image_sum_z(const cell_t *c, const double *d, double z, double alpha, double r_c, double *out) {
    double dw[3] = {0, 0, 0};
    wrap(c, d, dw);
    double dn = norm(2, dw);
    int mmax[2];
    for (int k = 0; k < 2; ++k) mmax[k] = (int)ceil((r_c + dn) * norm(2, c->b[k]) / (2.0 * M_PI));
    double s = 0.0;
    for (int m0 = -mmax[0]; m0 <= mmax[0]; ++m0)
        for (int m1 = -mmax[1]; m1 <= mmax[1]; ++m1) {
            double x0 = dw[0] + m0 * c->a[0][0] + m1 * c->a[1][0];
            double x1 = dw[1] + m0 * c->a[0][1] + m1 * c->a[1][1];
            double r = sqrt(x0 * x0 + x1 * x1 + z * z);
            if (r < r_c) {
                if (r < 1e-10 * sqrt(c->vol)) return ORC_ERR_COINCIDENT;
                s += erfc(alpha * r) / r;
            }
        }
    *out = s;
    return ORC_OK;
}

typedef struct {
    int n, k;          /* k >= 0: only pairs (k, j) for a move, with r_new */
    const double *pos, *z, *q, *r_new;
    double alpha;
    ksum_t sum;
} zrecip_ctx;

/* sum_{i<j} q_i q_j F(G, z_ij) cos(G.rho_ij) + 1/2 sum q_i^2 F(G, 0) */
static void visit_recip_z(const double *G, double g, const int *nvec, void *vctx) {
    (void)nvec;
    zrecip_ctx *r = (zrecip_ctx *)vctx;
    double s = 0.0, f0 = parry_f(g, 0.0, r->alpha), zl = 0.0, fl = f0;
    for (int i = 0; i < r->n; ++i) {
        s += 0.5 * r->q[i] * r->q[i] * f0;
        for (int j = i + 1; j < r->n; ++j) {
            double z = r->z[i] - r->z[j];
            if (z != zl) {  /* F of the last height difference is reused */
                zl = z;
                fl = parry_f(g, z, r->alpha);
            }
            double ph = G[0] * (r->pos[2 * i] - r->pos[2 * j]) + G[1] * (r->pos[2 * i + 1] - r->pos[2 * j + 1]);
            s += r->q[i] * r->q[j] * fl * cos(ph);
        }
    }
    kadd(&r->sum, s);
}

static int check_z(const double *lattice, int n, const double *pos, const double *z, const double *q,
                   double alpha, double r_c, double g_c, double *zmax) {
    int st = check_common(2, lattice, n, pos, q, alpha, r_c, g_c);
    if (st) return st;
    if (!z) return ORC_ERR_ARG;
    double lo = z[0], hi = z[0];
    for (int i = 0; i < n; ++i) {
        if (!isfinite(z[i])) return ORC_ERR_ARG;
        lo = fmin(lo, z[i]);
        hi = fmax(hi, z[i]);
    }
    *zmax = hi - lo;
    if (*zmax * g_c > 600.0) return ORC_ERR_ARG;
    return ORC_OK;
}

int oracle_energy_z(const double *lattice, int n, const double *pos, const double *z, const double *q,
                    double alpha, double r_c, double g_c, double *comp, double *e) {
    double zmax;
    int st = check_z(lattice, n, pos, z, q, alpha, r_c, g_c, &zmax);
    if (st) return st;
    cell_t c;
    if ((st = make_cell(2, lattice, &c))) return st;

    ksum_t real = {0.0, 0.0}, bg = {0.0, 0.0};
    double q2 = 0.0;
    for (int i = 0; i < n; ++i) {
        q2 += q[i] * q[i];
        for (int j = i + 1; j < n; ++j) {
            double d[2] = {pos[2 * i] - pos[2 * j], pos[2 * i + 1] - pos[2 * j + 1]}, s;
            if ((st = image_sum_z(&c, d, z[i] - z[j], alpha, r_c, &s))) return st;
            kadd(&real, q[i] * q[j] * s);
            kadd(&bg, q[i] * q[j] * sheet_g(z[i] - z[j], alpha));
        }
    }
    double zero[3] = {0, 0, 0}, smad;
    if ((st = image_sum(&c, zero, alpha, r_c, 1, &smad))) return st;

    zrecip_ctx rc = {n, -1, pos, z, q, NULL, alpha, {0.0, 0.0}};
    for_each_g(&c, g_c, visit_recip_z, &rc);

    double pa = M_PI / c.vol;
    double e_real = kval(&real);
    double e_madR = 0.5 * q2 * smad;
    double e_recip = pa * kval(&rc.sum);
    double e_self = -alpha / sqrt(M_PI) * q2;
    double e_bg = -2.0 * pa * (kval(&bg) + 0.5 * q2 * sheet_g(0.0, alpha));
    if (comp) {
        comp[0] = e_real;
        comp[1] = e_madR;
        comp[2] = e_recip;
        comp[3] = e_self;
        comp[4] = e_bg;
    }
    *e = e_real + e_madR + e_recip + e_self + e_bg;
    return ORC_OK;
}

/* v_E of one pair without the height term (it does not change in a move):
 * the image sum and (pi/A) sum_G F(G, z) cos(G.rho), for every G. */
typedef struct {
    double rho[2], z, alpha;
    ksum_t sum;
} zpair_ctx;

static void visit_pair_z(const double *G, double g, const int *nvec, void *vctx) {
    (void)nvec;
    zpair_ctx *p = (zpair_ctx *)vctx;
    kadd(&p->sum, parry_f(g, p->z, p->alpha) * cos(G[0] * p->rho[0] + G[1] * p->rho[1]));
}

/*
 * Energy change when particle k moves in the plane to r_new (its height
 * stays z[k]), straight from the pair definition:
 *   dE = q_k sum_{j != k} q_j [v_E(r_new - rho_j, z_kj) - v_E(rho_k - rho_j, z_kj)].
 * The height term of v_E depends on z_kj only and cancels.
 */
int oracle_delta_e_z(const double *lattice, int n, const double *pos, const double *z, const double *q, int k,
                     const double *r_new, double alpha, double r_c, double g_c, double *de) {
    double zmax;
    int st = check_z(lattice, n, pos, z, q, alpha, r_c, g_c, &zmax);
    if (st) return st;
    if (k < 0 || k >= n || !r_new || !de) return ORC_ERR_ARG;
    cell_t c;
    if ((st = make_cell(2, lattice, &c))) return st;
    ksum_t tot = {0.0, 0.0};
    for (int j = 0; j < n; ++j) {
        if (j == k) continue;
        double v[2];
        for (int which = 0; which < 2; ++which) {
            const double *rk = which ? r_new : pos + 2 * k;
            double d[2] = {rk[0] - pos[2 * j], rk[1] - pos[2 * j + 1]}, s;
            if ((st = image_sum_z(&c, d, z[k] - z[j], alpha, r_c, &s))) return st;
            zpair_ctx pc = {{d[0], d[1]}, z[k] - z[j], alpha, {0.0, 0.0}};
            for_each_g(&c, g_c, visit_pair_z, &pc);
            v[which] = s + M_PI / c.vol * kval(&pc.sum);
        }
        kadd(&tot, q[k] * q[j] * (v[1] - v[0]));
    }
    *de = kval(&tot);
    return ORC_OK;
}

/* ===================================================================== */
/*
 * Two-body polynomial Jastrow term u (Sec. 2.3, Eq. (8)):
 *
 *   J_u = sum_{i<j} u_{s_i s_j}(r_ij),
 *   u(r) = (r - L_u)^C sum_{l=0}^{N_u} alpha_l r^l  for r < L_u, 0 beyond,
 *
 * r_ij being the distance from i to the nearest image of j.  L_u must lie
 * below half the shortest nonzero lattice vector, so at most one image of
 * j is inside L_u; the sum below visits every image inside L_u, which is
 * that definition.  Particles 0 .. n_up-1 have spin up, the others spin
 * down; like spins take the coefficients alpha_like, unlike spins
 * alpha_unlike.  alpha_1 of each set is not an input: the Kato cusp
 * condition u'(0) = Gamma fixes it,
 *
 *   alpha_1 = Gamma / (-L_u)^C + C alpha_0 / L_u,
 *
 * Gamma = 1/2 (unlike spins) and 1/4 (like spins) in 3D, 1 and 1/3 in 2D.
 * Gradient and Laplacian with respect to particle i's position:
 *
 *   grad_i = sum_{j != i} u'(r_ij) x_ij / r_ij,
 *   lap_i  = sum_{j != i} [u''(r_ij) + (d - 1) u'(r_ij) / r_ij],
 *
 * with x_ij = r_i - (nearest image of r_j).  u' and u'' by the product
 * rule on (r - L_u)^C P(r), each power sum written out term by term.
 *
 * Parity status: pinned (cusp value of u', vanishing of u and its first
 * C - 1 derivatives at L_u, finite differences of J_u, a two-particle
 * closed form, image and spin bookkeeping, invariances).
 */
static double cusp_alpha1(int dim, int like, double L, int C, double a0) {
    double gamma = dim == 3 ? (like ? 0.25 : 0.5) : (like ? 1.0 / 3.0 : 1.0);
    return gamma / pow(-L, C) + C * a0 / L;
}

/* u, u', u'' of one set at r < L (alpha[1] already the cusp value) */
static void u_terms(double r, double L, int C, int n_u, const double *alpha, double *u, double *du, double *d2u) {
    double P = 0.0, dP = 0.0, d2P = 0.0;
    for (int l = 0; l <= n_u; ++l) {
        P += alpha[l] * pow(r, l);
        if (l >= 1) dP += l * alpha[l] * pow(r, l - 1);
        if (l >= 2) d2P += l * (l - 1) * alpha[l] * pow(r, l - 2);
    }
    double t = r - L;
    double tC = pow(t, C), tC1 = pow(t, C - 1), tC2 = C >= 2 ? pow(t, C - 2) : 0.0;
    *u = tC * P;
    *du = C * tC1 * P + tC * dP;
    *d2u = C * (C - 1) * tC2 * P + 2.0 * C * tC1 * dP + tC * d2P;
}

int oracle_jastrow_u(int dim, const double *lattice, int n, const double *pos, int n_up, double L, int C, int n_u,
                     const double *alpha_like, const double *alpha_unlike, double *j_out, double *grad, double *lap) {
    cell_t c;
    if (n < 1 || !pos || !alpha_like || !alpha_unlike || !j_out || n_up < 0 || n_up > n) return ORC_ERR_ARG;
    if (C < 1 || C > 8 || n_u < 1 || n_u > 24 || !(L > 0.0)) return ORC_ERR_ARG;
    int st = make_cell(dim, lattice, &c);
    if (st) return st;
    /* L below half of every nonzero lattice vector of a box of small vectors */
    for (int m0 = -2; m0 <= 2; ++m0)
        for (int m1 = -2; m1 <= 2; ++m1)
            for (int m2 = (dim == 3 ? -2 : 0); m2 <= (dim == 3 ? 2 : 0); ++m2) {
                if (!m0 && !m1 && !m2) continue;
                double R[3] = {0, 0, 0};
                for (int y = 0; y < dim; ++y) R[y] = m0 * c.a[0][y] + m1 * c.a[1][y] + (dim == 3 ? m2 * c.a[2][y] : 0);
                if (!(2.0 * L < norm(dim, R))) return ORC_ERR_ARG;
            }
    double al[2][25];
    for (int l = 0; l <= n_u; ++l) {
        al[0][l] = alpha_unlike[l];
        al[1][l] = alpha_like[l];
    }
    al[0][1] = cusp_alpha1(dim, 0, L, C, al[0][0]);
    al[1][1] = cusp_alpha1(dim, 1, L, C, al[1][0]);
    ksum_t js = {0.0, 0.0};
    ksum_t *gs = (ksum_t *)calloc((size_t)n * dim, sizeof(ksum_t));
    ksum_t *ls = (ksum_t *)calloc((size_t)n, sizeof(ksum_t));
    for (int i = 0; i < n && !st; ++i)
        for (int j = 0; j < n && !st; ++j) {
            if (i == j) continue;
            const int like = (i < n_up) == (j < n_up);
            double d[3] = {0, 0, 0}, dw[3] = {0, 0, 0};
            for (int y = 0; y < dim; ++y) d[y] = pos[i * dim + y] - pos[j * dim + y];
            wrap(&c, d, dw);
            int mmax[3] = {0, 0, 0};
            for (int k = 0; k < dim; ++k)
                mmax[k] = (int)ceil((L + norm(dim, dw)) * norm(dim, c.b[k]) / (2.0 * M_PI));
            int m[3];
            for (m[0] = -mmax[0]; m[0] <= mmax[0]; ++m[0])
                for (m[1] = -mmax[1]; m[1] <= mmax[1]; ++m[1])
                    for (m[2] = -mmax[2]; m[2] <= mmax[2]; ++m[2]) {
                        double x[3] = {0, 0, 0};
                        for (int y = 0; y < dim; ++y) {
                            x[y] = dw[y];
                            for (int k = 0; k < dim; ++k) x[y] += m[k] * c.a[k][y];
                        }
                        const double r = norm(dim, x);
                        if (r >= L) continue;
                        if (r < 1e-10 * pow(c.vol, 1.0 / dim)) {
                            st = ORC_ERR_COINCIDENT;
                            continue;
                        }
                        double u, du, d2u;
                        u_terms(r, L, C, n_u, al[like], &u, &du, &d2u);
                        if (i < j) kadd(&js, u);
                        for (int y = 0; y < dim; ++y) kadd(&gs[i * dim + y], du * x[y] / r);
                        kadd(&ls[i], d2u + (dim - 1) * du / r);
                    }
        }
    if (!st) {
        *j_out = kval(&js);
        for (int k = 0; grad && k < n * dim; ++k) grad[k] = kval(&gs[k]);
        for (int k = 0; lap && k < n; ++k) lap[k] = kval(&ls[k]);
    }
    free(gs);
    free(ls);
    return st;
}
