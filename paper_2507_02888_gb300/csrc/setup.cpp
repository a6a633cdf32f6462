// Host set-up of a periodic system, in FP64 (paper Sec. 6.1: the Ewald
// set-up tables are numerically sensitive and stay in double precision even
// when the rest runs in single precision).
//
// Builds, from the lattice, the charges and alpha:
//   - the reciprocal basis b_k (a_i . b_j = 2 pi delta_ij) and the volume;
//   - the cutoffs (erfc(alpha r_c) = 1e-16, or kMixedRealTol in the mixed
//     path; exp(-G^2/4alpha^2) = 1e-16 in 3D, erfc(G/2alpha) = 1e-16 in 2D)
//     unless the caller gives them;
//   - the G vectors of one half-space (one of each +-G pair), grouped in rows
//     of consecutive n1 and split into runs for the structure-factor kernel,
//     with weights 2 C f(G) (paper Eq. (3) and Eq. (5) at z = 0);
//   - the lattice vectors that can bring a wrapped displacement inside r_c,
//     and per displacement cell the short list of those that can for any
//     displacement in that cell;
//   - the position-independent energies: Madelung self-image, self,
//     background and the real-space sum among fixed particles (Eqs. (2)-(6)),
//     and the fixed particles' rho(G).
#include <algorithm>
#include <cmath>
#include <cstring>

#include "ewald_internal.h"

namespace ewald {

static const double kPi = 3.14159265358979323846;

static bool all_finite(const double *p, size_t n) {
    for (size_t i = 0; i < n; ++i)
        if (!std::isfinite(p[i])) return false;
    return true;
}

// x with erfc(x) = y (0 < y < 1), Newton's method on log erfc.
static double inverse_erfc(double y) {
    double x = std::sqrt(-std::log(y));
    for (int it = 0; it < 100; ++it) {
        double e = std::erfc(x);
        double g = std::log(e) - std::log(y);
        double gp = -2.0 / std::sqrt(kPi) * std::exp(-x * x) / e;
        double dx = g / gp;
        x -= dx;
        if (std::fabs(dx) < 1e-15 * std::fabs(x)) break;
    }
    return x;
}

static double norm_n(const double *v, int dim) {
    double s = 0;
    for (int k = 0; k < dim; ++k) s += v[k] * v[k];
    return std::sqrt(s);
}

// Cartesian vector of integer or fractional lattice coordinates m: sum_k m_k a_k.
static void lat_to_cart(const HostTables &t, const double *m, double *x) {
    for (int y = 0; y < 3; ++y) x[y] = 0;
    for (int y = 0; y < t.dim; ++y)
        for (int k = 0; k < t.dim; ++k) x[y] += m[k] * t.A[k][y];
}

// Fractional coordinates f_k = b_k . r / 2pi.
static void cart_to_frac(const HostTables &t, const double *r, double *f) {
    for (int k = 0; k < t.dim; ++k) {
        f[k] = 0;
        for (int y = 0; y < t.dim; ++y) f[k] += t.Ainv[y][k] * r[y];
    }
}

static int setup_lattice(HostTables *t, const double *lat, std::string *why) {
    int dim = t->dim;
    for (int i = 0; i < dim; ++i)
        for (int k = 0; k < dim; ++k) t->A[i][k] = lat[i * dim + k];
    double det;
    if (dim == 3) {
        double(*a)[3] = t->A;
        double c[3][3];  // cofactors
        c[0][0] = a[1][1] * a[2][2] - a[1][2] * a[2][1];
        c[0][1] = a[1][2] * a[2][0] - a[1][0] * a[2][2];
        c[0][2] = a[1][0] * a[2][1] - a[1][1] * a[2][0];
        c[1][0] = a[0][2] * a[2][1] - a[0][1] * a[2][2];
        c[1][1] = a[0][0] * a[2][2] - a[0][2] * a[2][0];
        c[1][2] = a[0][1] * a[2][0] - a[0][0] * a[2][1];
        c[2][0] = a[0][1] * a[1][2] - a[0][2] * a[1][1];
        c[2][1] = a[0][2] * a[1][0] - a[0][0] * a[1][2];
        c[2][2] = a[0][0] * a[1][1] - a[0][1] * a[1][0];
        det = a[0][0] * c[0][0] + a[0][1] * c[0][1] + a[0][2] * c[0][2];
        if (!(det > 0)) {
            *why = "lattice is singular or left-handed (det <= 0)";
            return EWALD_ERR_LATTICE;
        }
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) t->Ainv[i][j] = c[j][i] / det;  // inverse = adj / det
    } else {
        double(*a)[3] = t->A;
        det = a[0][0] * a[1][1] - a[0][1] * a[1][0];
        if (!(det > 0)) {
            *why = "lattice is singular or left-handed (det <= 0)";
            return EWALD_ERR_LATTICE;
        }
        t->Ainv[0][0] = a[1][1] / det;
        t->Ainv[0][1] = -a[0][1] / det;
        t->Ainv[1][0] = -a[1][0] / det;
        t->Ainv[1][1] = a[0][0] / det;
    }
    // scale-free conditioning check: reject nearly flat cells
    double prod = 1;
    for (int i = 0; i < dim; ++i) prod *= norm_n(t->A[i], dim);
    if (det < 1e-10 * prod) {
        *why = "lattice is (numerically) singular";
        return EWALD_ERR_LATTICE;
    }
    t->volume = det;
    for (int k = 0; k < dim; ++k)
        for (int y = 0; y < dim; ++y) t->B[k][y] = 2 * kPi * t->Ainv[y][k];
    return EWALD_OK;
}

// Largest |A^T f| over the corners of [-1/2, 1/2]^dim: the longest wrapped displacement.
static double max_wrapped_norm(const HostTables &t) {
    double best = 0;
    for (int c = 0; c < (1 << t.dim); ++c) {
        double f[3] = {0, 0, 0}, x[3];
        for (int k = 0; k < t.dim; ++k) f[k] = (c >> k & 1) ? 0.5 : -0.5;
        lat_to_cart(t, f, x);
        best = std::max(best, norm_n(x, t.dim));
    }
    return best;
}

// Close radius of the FP32 path and the coarsest displacement cells that go
// with it.  A displacement within r_close of an image R (a physically close
// pair, possibly across the cell boundary) has its term evaluated in FP64.
// The FP32 loop tests only candidate 0 of each cell for this, which is
// enough when no two images can come within r_close of one cell: two such
// images are less than 2 (r_close + cell radius) apart, so it suffices that
// 2 (r_close + max_wrapped_norm / 2^bits) < |R_min|.  r_close = 0.3 of the
// mean spacing of all charges, lowered if the cell is very flat.
static void set_close_radius(HostTables *t) {
    const int dim = t->dim;
    double rmin = 1e300;
    for (int m0 = -2; m0 <= 2; ++m0)
        for (int m1 = -2; m1 <= 2; ++m1)
            for (int m2 = (dim == 3 ? -2 : 0); m2 <= (dim == 3 ? 2 : 0); ++m2) {
                if (!m0 && !m1 && !m2) continue;
                double m[3] = {(double)m0, (double)m1, (double)m2}, x[3];
                lat_to_cart(*t, m, x);
                rmin = std::min(rmin, norm_n(x, dim));
            }
    const double spacing = std::pow(t->volume / (double)(t->n_mob + t->n_fix), 1.0 / dim);
    double rc = std::min(0.3 * spacing, 0.25 * rmin);
    const double wn = max_wrapped_norm(*t);
    const int max_bits = dim == 3 ? 4 : 6;
    int b = 0;
    while (b < max_bits && 2 * (rc + wn / (1 << b)) >= rmin) ++b;
    rc = std::min(rc, 0.999 * (0.5 * rmin - wn / (1 << b)));
    t->r_close = std::max(rc, 0.0);
    t->min_bits = b;
}

static void build_images(HostTables *t) {
    int dim = t->dim;
    double reach = t->r_c + max_wrapped_norm(*t);
    int mb[3] = {0, 0, 0};
    for (int k = 0; k < dim; ++k) mb[k] = (int)std::ceil(reach * norm_n(t->B[k], dim) / (2 * kPi));
    struct Img { double r, x[3]; };
    std::vector<Img> v;
    for (int m0 = -mb[0]; m0 <= mb[0]; ++m0)
        for (int m1 = -mb[1]; m1 <= mb[1]; ++m1)
            for (int m2 = -mb[2]; m2 <= mb[2]; ++m2) {
                double m[3] = {(double)m0, (double)m1, (double)m2}, x[3];
                lat_to_cart(*t, m, x);
                double r = norm_n(x, dim);
                if (r < reach * (1 + 1e-9)) v.push_back({r, {x[0], x[1], x[2]}});
            }
    std::sort(v.begin(), v.end(), [](const Img &a, const Img &b) { return a.r < b.r; });
    t->img.clear();
    for (auto &i : v) t->img.insert(t->img.end(), {i.x[0], i.x[1], i.x[2]});
}

// Candidate lists for 2^bits displacement cells per axis, in image-table
// order except that the image nearest to the cell's centre comes first.
// Returns the longest list.  A displacement cell is the parallelepiped [-1/2 + s/M,
// -1/2 + (s+1)/M) of fractional coordinates; every point in it is within
// d_max / M of its centre, so R can contribute only if |c + R| < r_c + d_max/M.
static int cand_lists(const HostTables &t, const std::vector<double> &imgs, double cutoff, int bits,
                      std::vector<unsigned short> *cand, std::vector<int> *len) {
    int dim = t.dim, M = 1 << bits, n_sub = 1;
    for (int k = 0; k < dim; ++k) n_sub *= M;
    double rad = max_wrapped_norm(t) / M;
    double lim = (cutoff + rad) * (1 + 1e-9);
    int n_img = (int)imgs.size() / 3;
    std::vector<std::vector<unsigned short>> lists(n_sub);
    int longest = 0;
    for (int s = 0; s < n_sub; ++s) {
        double f[3] = {0, 0, 0}, c[3];
        for (int k = 0; k < dim; ++k) f[k] = -0.5 + (((s >> (k * bits)) & (M - 1)) + 0.5) / M;
        lat_to_cart(t, f, c);
        int nearest = -1;
        double dn = 1e300;
        for (int i = 0; i < n_img; ++i) {
            double x[3];
            for (int y = 0; y < 3; ++y) x[y] = c[y] + imgs[3 * i + y];
            const double r = norm_n(x, dim);
            if (r < lim) {
                if (r < dn) dn = r, nearest = (int)lists[s].size();
                lists[s].push_back((unsigned short)i);
            }
        }
        // the image nearest to the cell's centre first: with at least
        // min_bits bits it is the only one that can bring a displacement of
        // the cell within r_close (see set_close_radius)
        if (nearest > 0) std::rotate(lists[s].begin(), lists[s].begin() + nearest, lists[s].begin() + nearest + 1);
        longest = std::max(longest, (int)lists[s].size());
    }
    if (cand) {
        // pad every list to the longest with the sentinel image n_img (far away)
        cand->assign((size_t)n_sub * std::max(longest, 1), (unsigned short)n_img);
        len->assign(n_sub, 0);
        for (int s = 0; s < n_sub; ++s) {
            (*len)[s] = (int)lists[s].size();
            std::copy(lists[s].begin(), lists[s].end(), cand->begin() + (size_t)s * longest);
        }
    }
    return longest;
}

// Position in list l (of length len) of the image second nearest to the
// point c, after the nearest, which t.cand already puts first.
static int second_nearest(const HostTables &t, const unsigned short *l, int len, const double *c) {
    const int n_img = (int)t.img.size() / 3;
    int best = 1;
    double db = 1e300;
    for (int p = 1; p < len; ++p) {
        if (l[p] >= n_img) continue;
        double x[3];
        for (int y = 0; y < 3; ++y) x[y] = c[y] + t.img[3 * l[p] + y];
        const double r = norm_n(x, t.dim);
        if (r < db) db = r, best = p;
    }
    return best;
}

static void cell_centre(const HostTables &t, int s, double *c) {
    const int M = 1 << t.sub_bits;
    double f[3] = {0, 0, 0};
    for (int k = 0; k < t.dim; ++k) f[k] = -0.5 + (((s >> (k * t.sub_bits)) & (M - 1)) + 0.5) / M;
    lat_to_cart(t, f, c);
}

// Whether the mixed form's energy loop should take the first two images of
// every list as one unconditional paired evaluation (terms outside r_c
// masked): where lists hold 3 to 8 images and the second nearest image to a
// cell's centre lies inside r_c for at least 3/4 of the displacements, the
// masked evaluation costs less than testing and queueing the two images.
// Estimated on 4^dim stratified points of every displacement cell.
bool mixed_direct_pays(const HostTables &t) {
    if (t.cand_max < 3 || t.cand_max > 8) return false;
    const int dim = t.dim, M = 1 << t.sub_bits, L = t.cand_max, n_sub = (int)(t.cand.size() / L);
    const int per = 1 << (2 * dim);
    long inside = 0, total = 0;
    for (int s = 0; s < n_sub; ++s) {
        const int len = t.cand_len.empty() ? L : t.cand_len[s];
        double c[3];
        cell_centre(t, s, c);
        const unsigned short *l = t.cand.data() + (size_t)s * L;
        const int p2 = len >= 2 ? second_nearest(t, l, len, c) : -1;
        for (int q = 0; q < per; ++q) {
            total++;
            if (p2 < 0 || l[p2] >= (int)t.img.size() / 3) continue;
            double f[3] = {0, 0, 0}, x[3];
            for (int k = 0; k < dim; ++k) {
                const int cell_k = (s >> (k * t.sub_bits)) & (M - 1), sub_k = (q >> (2 * k)) & 3;
                f[k] = -0.5 + (cell_k + (sub_k + 0.5) / 4) / M;
            }
            lat_to_cart(t, f, x);
            for (int y = 0; y < 3; ++y) x[y] += t.img[3 * l[p2] + y];
            if (norm_n(x, dim) < t.r_c) inside++;
        }
    }
    return total > 0 && inside * 4 >= total * 3;
}

// The candidate lists in the order of the mixed form's pair loop: as in
// t.cand (the image nearest to the cell's centre first, the rest in
// image-table order), and with direct evaluation the second nearest image
// moved to the second place, so that the unconditional pair holds the two
// images most often inside r_c.
std::vector<unsigned short> mixed_cand_order(const HostTables &t, bool direct) {
    std::vector<unsigned short> out = t.cand;
    if (!direct) return out;
    const int L = std::max(t.cand_max, 1), n_sub = (int)(t.cand.size() / L);
    for (int s = 0; s < n_sub; ++s) {
        const int len = t.cand_len.empty() ? L : t.cand_len[s];
        if (len < 3) continue;
        double c[3];
        cell_centre(t, s, c);
        unsigned short *l = out.data() + (size_t)s * L;
        const int p2 = second_nearest(t, l, len, c);
        std::rotate(l + 1, l + p2, l + p2 + 1);
    }
    return out;
}

static int build_cand(const HostTables &t, int bits, std::vector<unsigned short> *cand, std::vector<int> *len) {
    return cand_lists(t, t.img, t.r_c, bits, cand, len);
}

int set_subcells(HostTables *t, int bits) {
    t->sub_bits = bits;
    t->cand_max = build_cand(*t, bits, &t->cand, &t->cand_len);
    return t->cand_max;
}

// Bytes of shared memory the candidate lists of 2^bits cells per axis need.
size_t subcell_bytes(const HostTables &t, int bits) {
    int n_sub = 1 << (bits * t.dim);
    return (size_t)n_sub * build_cand(t, bits, nullptr, nullptr) * 2;
}

// Choose the number of displacement cells: the shortest longest-list whose
// table fits in max_bytes of shared memory.
int pick_subcells(HostTables *t, int max_bytes) {
    int best_bits = t->min_bits, best_len = 1 << 30;
    int max_bits = t->dim == 3 ? 4 : 6;
    for (int b = t->min_bits; b <= max_bits; ++b) {
        int n_sub = 1 << (b * t->dim);
        int L = build_cand(*t, b, nullptr, nullptr);
        size_t bytes = (size_t)n_sub * L * 2 + (size_t)n_sub * 4;
        if (bytes > (size_t)max_bytes && b > t->min_bits) break;
        if (L < best_len) {
            best_len = L;
            best_bits = b;
        }
    }
    t->sub_bits = best_bits;
    t->cand_max = build_cand(*t, best_bits, &t->cand, &t->cand_len);
    return best_bits;
}

// erfcx(x) = exp(x^2) erfc(x) for x >= 0: directly while exp(x^2) stays
// finite, else the asymptotic series 1/(x sqrt(pi)) sum_k (-1)^k (2k-1)!! /
// (2x^2)^k (Abramowitz & Stegun 7.1.23), whose terms at x >= 26 fall below
// 1e-19 by k = 8.
static double erfcx_pos(double x) {
    if (x < 26.0) return std::exp(x * x) * std::erfc(x);
    const double v = 1.0 / (2.0 * x * x);
    double term = 1.0, sum = 1.0;
    for (int k = 1; k <= 8; ++k) {
        term *= -(2.0 * k - 1.0) * v;
        sum += term;
    }
    return sum / (x * std::sqrt(kPi));
}

// F(G, z) of the 2D reciprocal sum at height difference z (paper Eq. (5)):
// [e^{zG} erfc(G/2alpha + z alpha) + e^{-zG} erfc(G/2alpha - z alpha)] / G.
// With a = G/2alpha and b = |z| alpha (zG = 2ab) each product is written
// without the large factor e^{|z|G}: e^{-a^2-b^2} erfcx(a + b), and
// e^{-a^2-b^2} erfcx(a - b) if a >= b, else e^{-|z|G} erfc(a - b).
static double parry_f(double g, double z, double alpha) {
    const double a = g / (2 * alpha), b = std::fabs(z) * alpha;
    const double e = std::exp(-a * a - b * b);
    const double t1 = e * erfcx_pos(a + b);
    const double t2 = a >= b ? e * erfcx_pos(a - b) : std::exp(-std::fabs(z) * g) * std::erfc(a - b);
    return (t1 + t2) / g;
}

// z erf(alpha z) + exp(-alpha^2 z^2) / (alpha sqrt(pi)): the G = 0 term of
// paper Eq. (5) at height difference z (divided by -2 pi / A)
static double sheet_g(double z, double alpha) {
    return z * std::erf(alpha * z) + std::exp(-alpha * alpha * z * z) / (alpha * std::sqrt(kPi));
}

static void build_gvectors(HostTables *t) {
    int dim = t->dim;
    int nb[3] = {0, 0, 0};
    for (int k = 0; k < dim; ++k) nb[k] = (int)std::ceil(t->g_c * norm_n(t->A[k], dim) / (2 * kPi));
    struct Row { int n2, n3, lo, hi; };
    std::vector<Row> rows;
    int n3lo = 0, n3hi = dim == 3 ? nb[2] : 0;
    for (int n3 = n3lo; n3 <= n3hi; ++n3)
        for (int n2 = -nb[1]; n2 <= nb[1]; ++n2) {
            if (n3 == 0 && n2 < 0) continue;  // half-space: first nonzero of (n3, n2, n1) > 0
            int lo = 1 << 30, hi = -(1 << 30);
            for (int n1 = -nb[0]; n1 <= nb[0]; ++n1) {
                if (n3 == 0 && n2 == 0 && n1 <= 0) continue;
                double G[3] = {0, 0, 0};
                for (int y = 0; y < dim; ++y)
                    G[y] = n1 * t->B[0][y] + n2 * t->B[1][y] + (dim == 3 ? n3 * t->B[2][y] : 0);
                if (norm_n(G, dim) <= t->g_c) {
                    lo = std::min(lo, n1);
                    hi = std::max(hi, n1);
                }
            }
            if (lo <= hi) rows.push_back({n2, n3, lo, hi});
        }
    // Split every row at its smallest |G| and walk outward in both directions,
    // in runs of <= run_len consecutive n1 (lengths as equal as possible).  A
    // run is (n1 start, n2, n3, dir * length), dir = +1 or -1.  The FP32
    // recurrence error grows along a run; starting each run at the small-|G|
    // end keeps it smallest where the weights f(G) are largest.
    t->runs.clear();
    t->gn.clear();
    t->n1max = t->n2max = t->n3max = 0;
    auto split = [&](int start, int L, int dir, int n2, int n3) {
        if (L <= 0) return;
        int nr = (L + t->run_len - 1) / t->run_len;
        for (int j = 0; j < nr; ++j) {
            int len = L / nr + (j < L % nr ? 1 : 0);
            t->runs.insert(t->runs.end(), {start, n2, n3, dir * len});
            start += dir * len;
        }
    };
    for (auto &r : rows) {
        int mid = r.lo;
        double best = 1e300;
        for (int n1 = r.lo; n1 <= r.hi; ++n1) {
            double G[3] = {0, 0, 0};
            for (int y = 0; y < dim; ++y)
                G[y] = n1 * t->B[0][y] + r.n2 * t->B[1][y] + (dim == 3 ? r.n3 * t->B[2][y] : 0);
            double g = norm_n(G, dim);
            if (g < best) { best = g; mid = n1; }
        }
        split(mid, r.hi - mid + 1, +1, r.n2, r.n3);
        split(mid - 1, mid - r.lo, -1, r.n2, r.n3);
        t->n1max = std::max(t->n1max, std::max(std::abs(r.lo), std::abs(r.hi)));
        t->n2max = std::max(t->n2max, std::abs(r.n2));
        t->n3max = std::max(t->n3max, std::abs(r.n3));
    }
    // Longest runs first (stable): the structure-factor kernel's warps then
    // hold runs of nearly one length and stop at their own longest.
    {
        const int nr = (int)t->runs.size() / 4;
        std::vector<int> order(nr);
        for (int i = 0; i < nr; ++i) order[i] = i;
        std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
            return std::abs(t->runs[4 * a + 3]) > std::abs(t->runs[4 * b + 3]);
        });
        std::vector<int> sorted;
        sorted.reserve(t->runs.size());
        for (int i : order) sorted.insert(sorted.end(), t->runs.begin() + 4 * i, t->runs.begin() + 4 * i + 4);
        t->runs.swap(sorted);
    }
    int n_runs = (int)t->runs.size() / 4;
    int slots = n_runs * t->run_len;
    t->gw.assign(slots, 0.0);
    t->g2slot.clear();
    double C = dim == 3 ? 2 * kPi / t->volume : kPi / t->volume;
    for (int run = 0; run < n_runs; ++run) {
        const int *rn = &t->runs[4 * run];
        const int dir = rn[3] > 0 ? 1 : -1, len = std::abs(rn[3]);
        for (int j = 0; j < len; ++j) {
            int n[3] = {rn[0] + dir * j, rn[1], rn[2]};
            double G[3] = {0, 0, 0};
            for (int y = 0; y < dim; ++y)
                for (int k = 0; k < dim; ++k) G[y] += n[k] * t->B[k][y];
            double g = norm_n(G, dim);
            double f = dim == 3 ? std::exp(-g * g / (4 * t->alpha * t->alpha)) / (g * g)
                                : std::erfc(g / (2 * t->alpha)) / g;
            int slot = j * n_runs + run;
            t->gw[slot] = 2 * C * f;  // half-space: +G and -G give equal terms
            t->g2slot.push_back(slot);
            for (int k = 0; k < dim; ++k) t->gn.push_back(n[k]);
        }
    }
    // layered 2D: weight (pi/A) F(G, z_L - z_L') of Re(rho_L conj(rho_L')),
    // every ordered layer pair (half-space: +G and -G give equal terms)
    t->gwl.clear();
    if (t->n_layers > 1) {
        const int nl = t->n_layers;
        t->gwl.assign((size_t)nl * nl * slots, 0.0);
        for (int run = 0; run < n_runs; ++run) {
            const int *rn = &t->runs[4 * run];
            const int dir = rn[3] > 0 ? 1 : -1, len = std::abs(rn[3]);
            for (int j = 0; j < len; ++j) {
                int n[3] = {rn[0] + dir * j, rn[1], rn[2]};
                double G[3] = {0, 0, 0};
                for (int y = 0; y < dim; ++y)
                    for (int k = 0; k < dim; ++k) G[y] += n[k] * t->B[k][y];
                const double g = norm_n(G, dim);
                const int slot = j * n_runs + run;
                for (int L = 0; L < nl; ++L)
                    for (int M = 0; M < nl; ++M)
                        t->gwl[((size_t)L * nl + M) * slots + slot] =
                            C * parry_f(g, t->layer_z[L] - t->layer_z[M], t->alpha);
            }
        }
    }
}

static void build_constants(HostTables *t) {
    int dim = t->dim;
    double q2 = 0, Q = 0;
    for (double q : t->q_mob) { q2 += q * q; Q += q; }
    for (double q : t->q_fix) { q2 += q * q; Q += q; }
    t->e_self = -t->alpha / std::sqrt(kPi) * q2;
    t->e_bg = dim == 3 ? -kPi * Q * Q / (2 * t->volume * t->alpha * t->alpha)
                       : -std::sqrt(kPi) * Q * Q / (t->volume * t->alpha);
    if (t->n_layers > 1) {  // -(pi/A) sum_{L,L'} Q_L Q_L' g(z_L - z_L')
        std::vector<double> QL(t->n_layers, 0.0);
        for (int i = 0; i < t->n_mob; ++i) QL[t->mob_layer[i]] += t->q_mob[i];
        for (int i = 0; i < t->n_fix; ++i) QL[t->fix_layer[i]] += t->q_fix[i];
        double sg = 0;
        for (int L = 0; L < t->n_layers; ++L)
            for (int M = 0; M < t->n_layers; ++M) sg += QL[L] * QL[M] * sheet_g(t->layer_z[L] - t->layer_z[M], t->alpha);
        t->e_bg = -kPi / t->volume * sg;
    }
    // Madelung self-image sum over R != 0 inside r_c: the image list covers |R| < r_c.
    int n_img = (int)t->img.size() / 3;
    double smad = 0;
    for (int i = 0; i < n_img; ++i) {
        double r = norm_n(&t->img[3 * i], dim);
        if (r > 0 && r < t->r_c) smad += std::erfc(t->alpha * r) / r;
    }
    t->e_madR = 0.5 * q2 * smad;
    // fixed-fixed real-space pairs, wrapped displacement + candidate images
    double eII = 0;
    for (int I = 0; I < t->n_fix; ++I)
        for (int J = I + 1; J < t->n_fix; ++J) {
            double d[3] = {0, 0, 0}, f[3], dw[3];
            for (int y = 0; y < dim; ++y) d[y] = t->fix_pos[I * dim + y] - t->fix_pos[J * dim + y];
            cart_to_frac(*t, d, f);
            for (int k = 0; k < dim; ++k) f[k] -= std::floor(f[k] + 0.5);
            lat_to_cart(*t, f, dw);
            const double dz = t->n_layers > 1 ? t->z_fix[I] - t->z_fix[J] : 0.0;
            double s = 0;
            for (int i = 0; i < n_img; ++i) {
                double x[3];
                for (int y = 0; y < 3; ++y) x[y] = dw[y] + t->img[3 * i + y];
                double r = std::sqrt(x[0] * x[0] + x[1] * x[1] + (dim == 3 ? x[2] * x[2] : dz * dz));
                if (r < t->r_c && r > 0) s += std::erfc(t->alpha * r) / r;
            }
            eII += t->q_fix[I] * t->q_fix[J] * s;
        }
    t->e_II = eII;
    // fixed particles' rho(G) per layer and slot: sum_I q_I exp(2 pi i n . f_I)
    int n_runs = (int)t->runs.size() / 4;
    const size_t slots = (size_t)n_runs * t->run_len;
    t->rho_fix.assign((size_t)t->n_layers * slots * 2, 0.0);
    if (t->n_fix == 0) return;
    std::vector<double> fr(t->n_fix * 3, 0.0);
    for (int I = 0; I < t->n_fix; ++I) cart_to_frac(*t, &t->fix_pos[I * dim], &fr[3 * I]);
    for (int run = 0; run < n_runs; ++run) {
        const int *rn = &t->runs[4 * run];
        const int dir = rn[3] > 0 ? 1 : -1, len = std::abs(rn[3]);
        for (int j = 0; j < len; ++j) {
            int n[3] = {rn[0] + dir * j, rn[1], rn[2]};
            const size_t slot = (size_t)j * n_runs + run;
            for (int I = 0; I < t->n_fix; ++I) {
                double ph = 0;
                for (int k = 0; k < dim; ++k) ph += n[k] * fr[3 * I + k];
                ph = 2 * kPi * (ph - std::floor(ph));
                const size_t o = 2 * ((t->n_layers > 1 ? (size_t)t->fix_layer[I] * slots : 0) + slot);
                t->rho_fix[o] += t->q_fix[I] * std::cos(ph);
                t->rho_fix[o + 1] += t->q_fix[I] * std::sin(ph);
            }
        }
    }
}

// Layers: the distinct heights among all particles, ascending.  One height
// (or none given) keeps n_layers = 1 and the plain 2D form: only height
// differences enter the energy.
static int setup_layers(HostTables *t, const ewald_desc *d, std::string *why) {
    t->n_layers = 1;
    t->layer_z.clear();
    t->z_mob.clear();
    t->z_fix.clear();
    t->mob_layer.clear();
    t->fix_layer.clear();
    t->lay_idx.clear();
    t->lay_start.clear();
    if (!d->mobile_z && !d->fixed_z) return EWALD_OK;
    std::vector<double> zm(t->n_mob, 0.0), zf(t->n_fix, 0.0);
    if (d->mobile_z) zm.assign(d->mobile_z, d->mobile_z + t->n_mob);
    if (d->fixed_z && t->n_fix) zf.assign(d->fixed_z, d->fixed_z + t->n_fix);
    std::vector<double> zs(zm);
    zs.insert(zs.end(), zf.begin(), zf.end());
    std::sort(zs.begin(), zs.end());
    zs.erase(std::unique(zs.begin(), zs.end()), zs.end());
    if (zs.size() == 1) return EWALD_OK;
    if ((int)zs.size() > EWALD_MAX_LAYERS) {
        *why = "more distinct particle heights than EWALD_MAX_LAYERS";
        return EWALD_ERR_ARG;
    }
    t->n_layers = (int)zs.size();
    t->layer_z = zs;
    t->z_mob = zm;
    t->z_fix = zf;
    auto layer_of = [&](double z) { return (int)(std::lower_bound(zs.begin(), zs.end(), z) - zs.begin()); };
    for (double z : zm) t->mob_layer.push_back(layer_of(z));
    for (double z : zf) t->fix_layer.push_back(layer_of(z));
    t->lay_start.assign(t->n_layers + 1, 0);
    for (int L = 0; L < t->n_layers; ++L) {
        t->lay_start[L] = (int)t->lay_idx.size();
        for (int i = 0; i < t->n_mob; ++i)
            if (t->mob_layer[i] == L) t->lay_idx.push_back(i);
    }
    t->lay_start[t->n_layers] = (int)t->lay_idx.size();
    return EWALD_OK;
}

// Shortest nonzero lattice vector (small integer combinations of a reduced
// basis reach it).
double shortest_lattice_vector(const HostTables &t) {
    double rmin = 1e300;
    const int r3 = t.dim == 3 ? 3 : 0;
    for (int m0 = -3; m0 <= 3; ++m0)
        for (int m1 = -3; m1 <= 3; ++m1)
            for (int m2 = -r3; m2 <= r3; ++m2) {
                if (!m0 && !m1 && !m2) continue;
                double m[3] = {(double)m0, (double)m1, (double)m2}, x[3];
                lat_to_cart(t, m, x);
                rmin = std::min(rmin, norm_n(x, t.dim));
            }
    return rmin;
}

// Images and displacement-cell candidate lists for a short cutoff (the
// Jastrow u term): every lattice vector within cutoff + the longest wrapped
// displacement, nearest first, and the lists for the cell count (2^bits per
// axis, bits <= max_bits) with the shortest longest list.  Returns that
// length; img is [n][3], cand [n_sub][cand_max] padded with index n.
int short_range_lists(const HostTables &t, double cutoff, int max_bits, std::vector<double> *img,
                      std::vector<unsigned short> *cand, int *bits_out) {
    const int dim = t.dim;
    const double reach = cutoff + max_wrapped_norm(t);
    int mb[3] = {0, 0, 0};
    for (int k = 0; k < dim; ++k) mb[k] = (int)std::ceil(reach * norm_n(t.B[k], dim) / (2 * kPi));
    struct Img { double r, x[3]; };
    std::vector<Img> v;
    for (int m0 = -mb[0]; m0 <= mb[0]; ++m0)
        for (int m1 = -mb[1]; m1 <= mb[1]; ++m1)
            for (int m2 = -mb[2]; m2 <= mb[2]; ++m2) {
                double m[3] = {(double)m0, (double)m1, (double)m2}, x[3];
                lat_to_cart(t, m, x);
                const double r = norm_n(x, dim);
                if (r < reach * (1 + 1e-9)) v.push_back({r, {x[0], x[1], x[2]}});
            }
    std::sort(v.begin(), v.end(), [](const Img &a, const Img &b) { return a.r < b.r; });
    img->clear();
    for (auto &i : v) img->insert(img->end(), {i.x[0], i.x[1], i.x[2]});
    int best = 1 << 30, best_bits = 0;
    for (int b = 0; b <= max_bits; ++b) {
        const int L = cand_lists(t, *img, cutoff, b, nullptr, nullptr);
        if (L < best) {
            best = L;
            best_bits = b;
        }
    }
    std::vector<int> len;
    *bits_out = best_bits;
    return cand_lists(t, *img, cutoff, best_bits, cand, &len);
}

int build_tables(const ewald_desc *d, HostTables *t, std::string *why) {
    if (!d) { *why = "desc is NULL"; return EWALD_ERR_ARG; }
    if (d->dim != 2 && d->dim != 3) { *why = "dim must be 2 or 3"; return EWALD_ERR_ARG; }
    if (!d->lattice) { *why = "lattice is NULL"; return EWALD_ERR_ARG; }
    if (d->n_mobile < 1 || !d->mobile_charge) { *why = "need n_mobile >= 1 and charges"; return EWALD_ERR_ARG; }
    if (d->n_fixed < 0 || (d->n_fixed > 0 && (!d->fixed_pos || !d->fixed_charge))) {
        *why = "bad fixed particles";
        return EWALD_ERR_ARG;
    }
    if (d->n_mobile > (1 << 20) || d->n_fixed > (1 << 20)) { *why = "too many particles"; return EWALD_ERR_ARG; }
    if (d->precision != EWALD_FP64 && d->precision != EWALD_MIXED && d->precision != EWALD_FP64_TIERED) {
        *why = "bad precision";
        return EWALD_ERR_ARG;
    }
    int dim = d->dim;
    if (!all_finite(d->lattice, dim * dim) || !all_finite(d->mobile_charge, d->n_mobile) ||
        (d->n_fixed && (!all_finite(d->fixed_pos, (size_t)d->n_fixed * dim) ||
                        !all_finite(d->fixed_charge, d->n_fixed))) ||
        !std::isfinite(d->gamma) || !std::isfinite(d->g_cutoff) || !std::isfinite(d->r_cutoff)) {
        *why = "non-finite input";
        return EWALD_ERR_ARG;
    }
    if ((d->mobile_z || d->fixed_z) && dim != 2) { *why = "particle heights need dim 2"; return EWALD_ERR_ARG; }
    if ((d->mobile_z && !all_finite(d->mobile_z, d->n_mobile)) ||
        (d->fixed_z && d->n_fixed && !all_finite(d->fixed_z, d->n_fixed))) {
        *why = "non-finite height";
        return EWALD_ERR_ARG;
    }
    t->dim = dim;
    t->n_mob = d->n_mobile;
    t->n_fix = d->n_fixed;
    // the tiered form is the FP64 form with a tiered real-space kernel
    t->tiered = d->precision == EWALD_FP64_TIERED;
    t->precision = t->tiered ? EWALD_FP64 : d->precision;
    t->resum_every = d->resum_every > 0 ? d->resum_every : 64;
    t->q_mob.assign(d->mobile_charge, d->mobile_charge + d->n_mobile);
    t->q_fix.assign(d->fixed_charge, d->fixed_charge + d->n_fixed);
    t->fix_pos.assign(d->fixed_pos, d->fixed_pos + (size_t)d->n_fixed * dim);
    int st = setup_lattice(t, d->lattice, why);
    if (st) return st;
    if ((st = setup_layers(t, d, why))) return st;

    // Cutoff tolerances.  The G side is 1e-16 in both precisions (the
    // reciprocal sum is cheap and sets the G count).  The real-space side is
    // 1e-16 in FP64; the mixed path re-expresses it for FP32 (as Sec. 6.1
    // does with CASINO's hard-wired tolerances): kMixedRealTol, far below
    // FP32 resolution but well above 1e-16, so that the pair sum skips the
    // images whose terms could not change an FP32 result.
    const double tol = 1e-16;
    double x_r = inverse_erfc(tol);
    const double x_rr = d->precision == EWALD_MIXED ? inverse_erfc(kMixedRealTol) : x_r;
    if (d->gamma > 0) {
        t->alpha = d->gamma;
    } else {
        // Balanced alpha: real-space and reciprocal work of the same order, with
        // N_G ~ sqrt(K N) reciprocal vectors (K from the trade-off between the
        // image count inside r_c and the G count inside g_c at 1e-16).
        double n = d->n_mobile + d->n_fixed;
        if (dim == 3) {
            double ng = std::sqrt(2.56e4 * n);
            double gc = std::cbrt(ng * 6 * kPi * kPi / t->volume);
            t->alpha = gc / (2 * std::sqrt(-std::log(tol)));
        } else {
            double ng = std::sqrt(1.19e3 * n);
            double gc = std::sqrt(ng * 4 * kPi / t->volume);
            t->alpha = gc / (2 * x_r);
        }
    }
    t->r_c = d->r_cutoff > 0 ? d->r_cutoff : x_rr / t->alpha;
    t->g_c = d->g_cutoff > 0 ? d->g_cutoff
                             : (dim == 3 ? 2 * t->alpha * std::sqrt(-std::log(tol)) : 2 * t->alpha * x_r);
    // guard against cutoffs that would need absurd tables
    double Lc = std::pow(t->volume, 1.0 / dim);
    if (t->r_c > 64 * Lc || t->g_c * Lc / (2 * kPi) > 256) {
        *why = "cutoff too large for the cell";
        return EWALD_ERR_ARG;
    }
    if (t->n_layers > 1 && (t->layer_z.back() - t->layer_z.front()) * t->g_c > 600) {
        *why = "layer separation too large for the G cutoff (|dz| g_c > 600)";
        return EWALD_ERR_ARG;
    }
    build_images(t);
    if (t->img.size() / 3 > 4000) {
        *why = "real-space cutoff needs more than 4000 candidate images";
        return EWALD_ERR_ARG;
    }
    set_close_radius(t);
    pick_subcells(t, 24 * 1024);
    build_gvectors(t);
    if (t->runs.empty()) {
        *why = "no G vector inside the cutoff";
        return EWALD_ERR_ARG;
    }
    build_constants(t);
    return EWALD_OK;
}

}  // namespace ewald
