/*
 * FP64 CPU oracle for Urchin reverse ray tracing (Altay & Theuns, arXiv:1304.4235).
 *
 * TEST INFRASTRUCTURE.  This file is the plain, slow, obviously-correct
 * restatement of what the paper defines, used only to check the CUDA library:
 * only the test-suite, the smoke check and the benchmark's CPU-baseline /
 * reference leg load it.  It shares no code, header, table or constant
 * generator with the CUDA path and never calls it.
 *
 * Every function below states the passage it follows.  Readings where the
 * paper is silent or garbled:
 *   - Verner et al. (1996) H I fit: the printed form lacks the exponent -P on
 *     (1 + sqrt(x/x_a)); the published fit has it, and only with it does
 *     sigma(13.6 eV) come out at sigma_th (App. C1, Eq. sigma_ver).
 *   - Rate coefficients (App. C3 points to fits in Theuns et al. 1998, not
 *     printed): alpha_A, alpha_B and collisional ionisation gamma from the
 *     Hui & Gnedin (1997) fits.
 *   - Root of the Riccati quadratic (Eq. xroots, x_-): evaluated as
 *     2P / (-Q + sqrt(Q^2 - 4PR)), the same root by Vieta's formula, which
 *     does not cancel when Gamma >> alpha n_H.
 *   - Update order: Jacobi (every Gamma of a sweep from the previous sweep's
 *     x), the order-independent variant Sec. 4 allows for parallel codes.
 *   - Rays start at the particle centre and sum every particle whose
 *     smoothing sphere they cross, the particle itself included (Eq. colden);
 *     periodic boxes add every periodic image within reach.
 *   - Frequency quadrature: w_j ~ J(nu_j) sigma(nu_j) / (h nu_j) (nu_{j+1/2}
 *     - nu_{j-1/2}) at geometric bin centres, rescaled so sum_j w_j =
 *     Gamma_thin (Eq. gamma and Sec. 3.3.3, ~100 bins).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_PI 3.14159265358979323846
#define OR_KERNEL_M4 0
#define OR_KERNEL_GT 1

/* ------------------------------------------------------------------------ */
/* Photoionisation cross sections, App. C1.                                 */
/* ------------------------------------------------------------------------ */

/* Eq. sigma_ana: sigma_th = 2^9 pi / (3 e^4) alpha_fs pi a_0^2 (CODATA 2018). */
double oracle_sigma_th(void)
{
    const double alpha_fs = 7.2973525693e-3;
    const double a0_cm = 5.29177210903e-9;
    return pow(2.0, 9.0) * OR_PI / (3.0 * exp(4.0)) * alpha_fs * OR_PI * a0_cm * a0_cm;
}

/* Ionisation threshold of H I in eV (13.6057 eV, Rydberg energy). */
double oracle_E_th(void) { return 13.605693122994; }

/* Eq. sigma_ana: exact hydrogenic cross section of an ion of charge Z,
 * threshold Z^2 E_th; zero below threshold. */
double oracle_sigma_hydrogenic(double E_eV, double Z)
{
    double Eth = Z * Z * oracle_E_th();
    if (E_eV < Eth) return 0.0;
    double r = E_eV / Eth;            /* nu / nu_th */
    double eps = sqrt(r - 1.0);
    double shape;
    if (eps < 1e-6) {
        shape = 1.0;                  /* limit eps -> 0 of the bracket */
    } else {
        shape = exp(4.0 - 4.0 * atan(eps) / eps) / (1.0 - exp(-2.0 * OR_PI / eps));
    }
    return oracle_sigma_th() / (Z * Z) * pow(1.0 / r, 4.0) * shape;
}

/* Eq. sigma_pwr: sigma_th (nu/nu_th)^-3. */
double oracle_sigma_powerlaw(double E_eV)
{
    if (E_eV < oracle_E_th()) return 0.0;
    return oracle_sigma_th() * pow(E_eV / oracle_E_th(), -3.0);
}

/* Eq. sigma_ver with the exponent -P restored (see header):
 * sigma = sigma_0 (x-1)^2 x^(0.5P-5.5) (1 + sqrt(x/x_a))^-P, x = E/E_0. */
double oracle_sigma_verner(double E_eV)
{
    if (E_eV < oracle_E_th()) return 0.0;
    const double E0 = 0.4298, sigma0 = 5.475e4 * 1e-18, xa = 32.88, P = 2.963;
    double x = E_eV / E0;
    return sigma0 * (x - 1.0) * (x - 1.0) * pow(x, 0.5 * P - 5.5) * pow(1.0 + sqrt(x / xa), -P);
}

double oracle_sigma(int which, double E_eV)
{
    if (which == 1) return oracle_sigma_hydrogenic(E_eV, 1.0);
    if (which == 2) return oracle_sigma_powerlaw(E_eV);
    return oracle_sigma_verner(E_eV);
}

/* Binned spectrum for Eq. gamma_shld: s_j = sigma_j / sigma_th and weights
 * w_j with sum_j w_j = Gamma_thin (Eq. gamma: Gamma = 4 pi int J sigma/(h nu)
 * dnu; 4 pi and h drop out of the normalisation). */
void oracle_spectrum(int F, const double* E_edges, const double* J, int xsec,
                     double gamma_thin, double* s_out, double* w_out)
{
    double sth = oracle_sigma_th(), tot = 0.0;
    for (int j = 0; j < F; ++j) {
        double Ej = sqrt(E_edges[j] * E_edges[j + 1]);
        double sj = oracle_sigma(xsec, Ej);
        s_out[j] = sj / sth;
        w_out[j] = J[j] * sj / Ej * (E_edges[j + 1] - E_edges[j]);
        tot += w_out[j];
    }
    for (int j = 0; j < F; ++j) w_out[j] *= gamma_thin / tot;
}

/* ------------------------------------------------------------------------ */
/* SPH kernels, Sec. 4.1.1.                                                  */
/* ------------------------------------------------------------------------ */

/* Eq. spline: M4 shape with the 8/(pi h^3) prefactor removed. */
double oracle_m4_shape(double q)
{
    if (q < 0.0) q = -q;
    if (q <= 0.5) return 1.0 - 6.0 * q * q + 6.0 * q * q * q;
    if (q <= 1.0) return 2.0 * (1.0 - q) * (1.0 - q) * (1.0 - q);
    return 0.0;
}

/* Eq. Gt constants: t = 2 pi^(1/6), A h = t, and the bracket
 * D = erf(t) - 2 t exp(-t^2)/sqrt(pi) so that N = 8/(pi h^3) / D. */
static double gt_t(void) { return 2.0 * pow(OR_PI, 1.0 / 6.0); }
static double gt_D(void)
{
    double t = gt_t();
    return erf(t) - 2.0 * t * exp(-t * t) / sqrt(OR_PI);
}

/* Eq. Gt shape with the 8/(pi h^3) prefactor removed: exp(-A^2 r^2) / D, r<=h. */
double oracle_gt_shape(double q)
{
    if (q < 0.0) q = -q;
    if (q > 1.0) return 0.0;
    double t = gt_t();
    return exp(-t * t * q * q) / gt_D();
}

/* Antiderivatives in u of q^n with q = sqrt(b^2 + u^2) (b, u in units of h):
 *   int q   du = (u q + b^2 asinh(u/b)) / 2
 *   int q^2 du = b^2 u + u^3 / 3
 *   int q^3 du = u q^3 / 4 + 3 b^2 u q / 8 + 3 b^4 asinh(u/b) / 8
 * (b^k asinh(u/b) -> 0 as b -> 0 for k >= 2). */
static double b2_asinh(double b, double u, int power)
{
    if (b <= 0.0) return 0.0;
    return pow(b, (double)power) * asinh(u / b);
}
static double Q1(double b, double u) { double q = sqrt(b * b + u * u); return 0.5 * (u * q + b2_asinh(b, u, 2)); }
static double Q2(double b, double u) { return b * b * u + u * u * u / 3.0; }
static double Q3(double b, double u)
{
    double q = sqrt(b * b + u * u);
    return u * q * q * q / 4.0 + 3.0 * b * b * u * q / 8.0 + 3.0 * b2_asinh(b, u, 4) / 8.0;
}
/* inner piece 1 - 6q^2 + 6q^3 (q <= 1/2) and outer piece 2(1-q)^3 (1/2 < q <= 1) */
static double m4_inner_prim(double b, double u) { return u - 6.0 * Q2(b, u) + 6.0 * Q3(b, u); }
static double m4_outer_prim(double b, double u) { return 2.0 * u - 6.0 * Q1(b, u) + 6.0 * Q2(b, u) - 2.0 * Q3(b, u); }

/* int_{u1}^{u2} M4shape(sqrt(b^2+u^2)) du for b in [0,1], u1 <= u2, both
 * inside the chord |u| <= sqrt(1-b^2).  Closed form of the line integral
 * through the M4 kernel used by Eq. colden. */
double oracle_chord_m4(double b, double u1, double u2)
{
    if (b >= 1.0 || u2 <= u1) return 0.0;
    double c = sqrt(1.0 - b * b);
    if (u1 < -c) u1 = -c;
    if (u2 > c) u2 = c;
    if (u2 <= u1) return 0.0;
    if (b >= 0.5) return m4_outer_prim(b, u2) - m4_outer_prim(b, u1);
    double s = sqrt(0.25 - b * b);   /* |u| at which q = 1/2 */
    double total = 0.0, lo, hi;
    lo = u1; hi = fmin(u2, -s);                 /* outer piece, u < -s */
    if (hi > lo) total += m4_outer_prim(b, hi) - m4_outer_prim(b, lo);
    lo = fmax(u1, -s); hi = fmin(u2, s);        /* inner piece, |u| <= s */
    if (hi > lo) total += m4_inner_prim(b, hi) - m4_inner_prim(b, lo);
    lo = fmax(u1, s); hi = u2;                  /* outer piece, u > s */
    if (hi > lo) total += m4_outer_prim(b, hi) - m4_outer_prim(b, lo);
    return total;
}

/* Eq. I(h,b,z1,z2) for the truncated Gaussian in units of h, prefactor
 * 8/(pi h^2) removed: exp(-t^2 b^2) sqrt(pi)/(2 t D) [erf(t z2) - erf(t z1)],
 * limits clipped to the chord inside r <= h. */
double oracle_chord_gt(double b, double u1, double u2)
{
    if (b >= 1.0 || u2 <= u1) return 0.0;
    double c = sqrt(1.0 - b * b);
    if (u1 < -c) u1 = -c;
    if (u2 > c) u2 = c;
    if (u2 <= u1) return 0.0;
    double t = gt_t();
    return exp(-t * t * b * b) * sqrt(OR_PI) / (2.0 * t * gt_D()) * (erf(t * u2) - erf(t * u1));
}

double oracle_chord(int kernel, double b, double u1, double u2)
{
    return kernel == OR_KERNEL_GT ? oracle_chord_gt(b, u1, u2) : oracle_chord_m4(b, u1, u2);
}

/* ------------------------------------------------------------------------ */
/* Columns, Eq. nhi / Eq. colden, brute force over all particles.           */
/* ------------------------------------------------------------------------ */

/* Threshold optical depth tau = sigma_th N_HI along the segment
 * o + t dir, t in [0, l_ray], by direct summation over every particle j
 * (and, for a periodic box of side L, over every periodic image of j that
 * can reach the segment):
 *     N_HI = sum_j (m_j x_j / m_p) int_0^L W(|r(t) - r_j| / h_j) dt.
 * Lengths are in the caller's unit; unit_cm converts them to cm. */
/* Term of particle j, shifted by (sx, sy, sz) (a periodic image offset, or
 * zero), in the column of the segment o + t dir, t in [0, l_ray], before
 * the factor sigma_th: (m_j x_j / m_p) (8/pi) / (h_j unit_cm)^2 times the
 * chord integral of the kernel; 0 when the segment misses the sphere. */
static double pair_term(double pxj, double pyj, double pzj, double hj, double mxj, double sx, double sy,
                        double sz, double unit_cm, const double* o, const double* dir, double l_ray, int kernel)
{
    double dx = pxj + sx - o[0];
    double dy = pyj + sy - o[1];
    double dz = pzj + sz - o[2];
    double tc = dx * dir[0] + dy * dir[1] + dz * dir[2];
    /* impact parameter from |d x dir| */
    double cx = dy * dir[2] - dz * dir[1];
    double cy = dz * dir[0] - dx * dir[2];
    double cz = dx * dir[1] - dy * dir[0];
    double b2 = cx * cx + cy * cy + cz * cz;
    if (b2 >= hj * hj) return 0.0;
    double half = sqrt(hj * hj - b2);
    double t1 = fmax(0.0, tc - half), t2 = fmin(l_ray, tc + half);
    if (t2 <= t1) return 0.0;
    double F = oracle_chord(kernel, sqrt(b2) / hj, (t1 - tc) / hj, (t2 - tc) / hj);
    double hcm = hj * unit_cm;
    return mxj * (8.0 / OR_PI) / (hcm * hcm) * F;
}

static double column_from_point(int64_t n, const double* px, const double* py, const double* pz,
                                const double* h, const double* mass_H, const double* x,
                                int periodic, double L, double unit_cm, int nimg,
                                const double* o, const double* dir, double l_ray, int kernel)
{
    double sum = 0.0;
    for (int64_t j = 0; j < n; ++j) {
        for (int a = -nimg; a <= nimg; ++a)
        for (int bb = -nimg; bb <= nimg; ++bb)
        for (int c = -nimg; c <= nimg; ++c)
            sum += pair_term(px[j], py[j], pz[j], h[j], mass_H[j] * x[j], periodic ? a * L : 0.0,
                             periodic ? bb * L : 0.0, periodic ? c * L : 0.0, unit_cm, o, dir, l_ray, kernel);
    }
    return oracle_sigma_th() * sum;
}

static int image_range(int periodic, double L, int64_t n, const double* h, double l_ray)
{
    if (!periodic) return 0;
    double hmax = 0.0;
    for (int64_t j = 0; j < n; ++j) hmax = fmax(hmax, h[j]);
    /* a segment of length l_ray starting inside [0,L)^3 reaches spheres whose
     * centres lie within l_ray + hmax of the box */
    return (int)ceil((l_ray + hmax) / L);
}

/* Rays from arbitrary points: tau_out[p*R + k] for point p, direction k. */
void oracle_columns_points(int64_t n, const double* px, const double* py, const double* pz,
                           const double* h, const double* mass_H, const double* x,
                           int periodic, double L, double unit_cm,
                           const double* points, int64_t n_points,
                           const double* dirs, int R, double l_ray, int kernel, double* tau_out)
{
    int nimg = image_range(periodic, L, n, h, l_ray);
    int64_t total = n_points * (int64_t)R;
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t r = 0; r < total; ++r) {
        int64_t p = r / R;
        int k = (int)(r % R);
        tau_out[r] = column_from_point(n, px, py, pz, h, mass_H, x, periodic, L, unit_cm, nimg,
                                       points + 3 * p, dirs + 3 * k, l_ray, kernel);
    }
}

/* Rays from particle centres (Sec. 3.2): origins[o] are particle indices
 * (NULL = all particles); tau_out[o*R + k]. */
void oracle_columns(int64_t n, const double* px, const double* py, const double* pz,
                    const double* h, const double* mass_H, const double* x,
                    int periodic, double L, double unit_cm,
                    const int64_t* origins, int64_t n_orig,
                    const double* dirs, int R, double l_ray, int kernel, double* tau_out)
{
    double* pts = (double*)malloc(sizeof(double) * 3 * (size_t)(n_orig > 0 ? n_orig : 1));
    for (int64_t o = 0; o < n_orig; ++o) {
        int64_t i = origins ? origins[o] : o;
        pts[3 * o] = px[i]; pts[3 * o + 1] = py[i]; pts[3 * o + 2] = pz[i];
    }
    oracle_columns_points(n, px, py, pz, h, mass_H, x, periodic, L, unit_cm,
                          pts, n_orig, dirs, R, l_ray, kernel, tau_out);
    free(pts);
}

/* ------------------------------------------------------------------------ */
/* Columns by a uniform-grid query: the same sum as oracle_columns          */
/* (Eq. colden), with the candidate particles of a ray taken from the grid  */
/* cells its segment passes through instead of from all n particles.        */
/* ------------------------------------------------------------------------ */

/* Every particle is listed in each cell of the box of cells that its
 * sphere's bounding box overlaps ("cell range" [lo, hi] per axis, in
 * unwrapped cell indices; a periodic grid stores cell i at i mod G).  A ray
 * walks the cells its segment crosses in order (3-D DDA in unwrapped
 * indices).  A candidate j met in unwrapped cell c belongs to the periodic
 * image a of j whose unwrapped range [lo + a G, hi + a G] contains c; that
 * image is evaluated once, in the first cell of the walk inside its range
 * (the cells of a range that a straight segment crosses are consecutive in
 * the walk, as the range is a box).  Every image whose sphere the segment
 * crosses has a crossed cell in its range, so the set of non-zero terms is
 * the brute force's; only the order of the sum differs. */
typedef struct {
    int periodic;
    double L, c;            /* box side, cell size */
    double lo[3];           /* grid origin */
    int64_t G[3];           /* cells per axis */
    int64_t* start;         /* [ncell + 1] first entry of each cell */
    int64_t* idx;           /* particle index per entry */
    int64_t* rlo;           /* [3 n] unwrapped cell range of each particle */
    int64_t* rhi;
    int64_t n;
} oracle_grid;

static int64_t floor_div(int64_t a, int64_t b) { int64_t q = a / b; return (a % b != 0 && (a < 0) != (b < 0)) ? q - 1 : q; }
static int64_t pos_mod(int64_t a, int64_t b) { int64_t r = a % b; return r < 0 ? r + b : r; }

void oracle_grid_free(oracle_grid* g)
{
    if (!g) return;
    free(g->start); free(g->idx); free(g->rlo); free(g->rhi); free(g);
}

/* Build the grid with cells of about `cell` (length unit).  Returns NULL when
 * a periodic sphere's cell range spans the whole box (2 h_j close to L),
 * where the image of a candidate would not be unique. */
oracle_grid* oracle_grid_build(int64_t n, const double* px, const double* py, const double* pz,
                               const double* h, int periodic, double L, double cell)
{
    oracle_grid* g = (oracle_grid*)calloc(1, sizeof(oracle_grid));
    const double* p[3] = {px, py, pz};
    g->periodic = periodic;
    g->L = L;
    g->n = n;
    if (periodic) {
        int64_t G = (int64_t)floor(L / cell);
        if (G < 1) G = 1;
        g->c = L / (double)G;
        for (int a = 0; a < 3; ++a) { g->lo[a] = 0.0; g->G[a] = G; }
    } else {
        g->c = cell;
        for (int a = 0; a < 3; ++a) {
            double mn = 1e300, mx = -1e300;
            for (int64_t j = 0; j < n; ++j) {
                mn = fmin(mn, p[a][j] - h[j]);
                mx = fmax(mx, p[a][j] + h[j]);
            }
            g->lo[a] = mn;
            g->G[a] = (int64_t)floor((mx - mn) / cell) + 1;
        }
    }
    g->rlo = (int64_t*)malloc(sizeof(int64_t) * 3 * (size_t)n);
    g->rhi = (int64_t*)malloc(sizeof(int64_t) * 3 * (size_t)n);
    for (int64_t j = 0; j < n; ++j)
        for (int a = 0; a < 3; ++a) {
            int64_t l = (int64_t)floor((p[a][j] - h[j] - g->lo[a]) / g->c);
            int64_t u = (int64_t)floor((p[a][j] + h[j] - g->lo[a]) / g->c);
            if (!periodic) {
                if (l < 0) l = 0;
                if (u > g->G[a] - 1) u = g->G[a] - 1;
            } else if (u - l + 1 >= g->G[a]) {
                oracle_grid_free(g);
                return NULL;
            }
            g->rlo[3 * j + a] = l;
            g->rhi[3 * j + a] = u;
        }
    const int64_t ncell = g->G[0] * g->G[1] * g->G[2];
    g->start = (int64_t*)calloc((size_t)ncell + 1, sizeof(int64_t));
    for (int pass = 0; pass < 2; ++pass) {
        int64_t* fill = NULL;
        if (pass == 1) {
            for (int64_t q = 0; q < ncell; ++q) g->start[q + 1] += g->start[q];
            g->idx = (int64_t*)malloc(sizeof(int64_t) * (size_t)(g->start[ncell] > 0 ? g->start[ncell] : 1));
            fill = (int64_t*)malloc(sizeof(int64_t) * (size_t)ncell);
            memcpy(fill, g->start, sizeof(int64_t) * (size_t)ncell);
        }
        for (int64_t j = 0; j < n; ++j)
            for (int64_t i = g->rlo[3 * j]; i <= g->rhi[3 * j]; ++i)
                for (int64_t k = g->rlo[3 * j + 1]; k <= g->rhi[3 * j + 1]; ++k)
                    for (int64_t m = g->rlo[3 * j + 2]; m <= g->rhi[3 * j + 2]; ++m) {
                        const int64_t q = (pos_mod(i, g->G[0]) * g->G[1] + pos_mod(k, g->G[1])) * g->G[2] +
                                          pos_mod(m, g->G[2]);
                        if (pass == 0) g->start[q + 1]++;
                        else g->idx[fill[q]++] = j;
                    }
        free(fill);
    }
    return g;
}

int64_t oracle_grid_entries(const oracle_grid* g) { return g ? g->start[g->G[0] * g->G[1] * g->G[2]] : -1; }

/* The column of the segment o + t dir, t in [0, l_ray], from the grid (the
 * factor sigma_th left out, as in column_from_point). */
static double grid_column(const oracle_grid* g, const double* px, const double* py, const double* pz,
                          const double* h, const double* mass_H, const double* x, double unit_cm,
                          const double* o, const double* dir, double l_ray, int kernel)
{
    int64_t cur[3], step[3], prev[3] = {0, 0, 0};
    double tmax[3], tdelta[3];
    for (int a = 0; a < 3; ++a) {
        cur[a] = (int64_t)floor((o[a] - g->lo[a]) / g->c);
        if (dir[a] > 0.0) {
            step[a] = 1;
            tmax[a] = ((double)(cur[a] + 1) * g->c + g->lo[a] - o[a]) / dir[a];
            tdelta[a] = g->c / dir[a];
        } else if (dir[a] < 0.0) {
            step[a] = -1;
            tmax[a] = ((double)cur[a] * g->c + g->lo[a] - o[a]) / dir[a];
            tdelta[a] = -g->c / dir[a];
        } else {
            step[a] = 0;
            tmax[a] = INFINITY;
            tdelta[a] = INFINITY;
        }
    }
    int have_prev = 0;
    double sum = 0.0;
    for (;;) {
        int inside = 1;
        int64_t s[3];
        for (int a = 0; a < 3; ++a) {
            if (g->periodic) s[a] = pos_mod(cur[a], g->G[a]);
            else {
                s[a] = cur[a];
                if (cur[a] < 0 || cur[a] >= g->G[a]) inside = 0;
            }
        }
        if (inside) {
            const int64_t q = (s[0] * g->G[1] + s[1]) * g->G[2] + s[2];
            for (int64_t e = g->start[q]; e < g->start[q + 1]; ++e) {
                const int64_t j = g->idx[e];
                int64_t img[3];
                int prev_in = have_prev;
                for (int a = 0; a < 3; ++a) {
                    const int64_t l = g->rlo[3 * j + a], u = g->rhi[3 * j + a];
                    /* the image whose unwrapped range holds the current cell */
                    img[a] = g->periodic ? floor_div(cur[a] - (l + pos_mod(s[a] - l, g->G[a])), g->G[a]) : 0;
                    const int64_t lo = l + img[a] * g->G[a], hi = u + img[a] * g->G[a];
                    if (prev[a] < lo || prev[a] > hi) prev_in = 0;
                }
                if (prev_in) continue;       /* met in an earlier cell of this walk */
                sum += pair_term(px[j], py[j], pz[j], h[j], mass_H[j] * x[j], g->periodic ? img[0] * g->L : 0.0,
                                 g->periodic ? img[1] * g->L : 0.0, g->periodic ? img[2] * g->L : 0.0, unit_cm, o,
                                 dir, l_ray, kernel);
            }
        }
        int ax = 0;
        if (tmax[1] < tmax[ax]) ax = 1;
        if (tmax[2] < tmax[ax]) ax = 2;
        if (!(tmax[ax] <= l_ray)) break;
        for (int a = 0; a < 3; ++a) prev[a] = cur[a];
        have_prev = 1;
        cur[ax] += step[ax];
        tmax[ax] += tdelta[ax];
    }
    return sum;
}

/* Columns of rays from particle centres (origins as in oracle_columns) by
 * the grid query: tau_out[o*R + k], the same values as oracle_columns up
 * to the order of the sum. */
void oracle_grid_columns(const oracle_grid* g, const double* px, const double* py, const double* pz,
                         const double* h, const double* mass_H, const double* x, double unit_cm,
                         const int64_t* origins, int64_t n_orig, const double* dirs, int R, double l_ray,
                         int kernel, double* tau_out)
{
    const double sth = oracle_sigma_th();
    const int64_t total = n_orig * (int64_t)R;
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t r = 0; r < total; ++r) {
        const int64_t o = r / R;
        const int k = (int)(r % R);
        const int64_t i = origins ? origins[o] : o;
        const double pt[3] = {px[i], py[i], pz[i]};
        tau_out[r] = sth * grid_column(g, px, py, pz, h, mass_H, x, unit_cm, pt, dirs + 3 * k, l_ray, kernel);
    }
}

/* Near/far split of Sec. 3.3.3 (self-contribution to self-shielding in
 * SPH): on the ray from particle i, a crossed particle j (periodic image
 * r_j + a L) is near when r_i lies inside its smoothing sphere,
 * |r_j + a L - r_i| < h_j, i.e. j contributes to the density at r_i in
 * Eq. nhi (the particle itself included); every other crossed particle is
 * far.  For origins[o] (NULL = all particles) and direction k:
 *   tau_far[o*R+k]  = sigma_th sum_far  (m_j x_j / m_p) int_0^l W dl
 *   tau_near[o*R+k] = sigma_th sum_near (m_j / m_p) int_0^l W dl   (neutral
 *                     fractions set to one: the slab thickness tau_H^near). */
void oracle_columns_nearfar(int64_t n, const double* px, const double* py, const double* pz,
                            const double* h, const double* mass_H, const double* x,
                            int periodic, double L, double unit_cm,
                            const int64_t* origins, int64_t n_orig,
                            const double* dirs, int R, double l_ray, int kernel,
                            double* tau_far, double* tau_near)
{
    int nimg = image_range(periodic, L, n, h, l_ray);
    int64_t total = n_orig * (int64_t)R;
    double sth = oracle_sigma_th();
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t r = 0; r < total; ++r) {
        int64_t o = r / R;
        int k = (int)(r % R);
        int64_t i = origins ? origins[o] : o;
        const double* dir = dirs + 3 * k;
        double far = 0.0, near = 0.0;
        for (int64_t j = 0; j < n; ++j) {
            double hj = h[j];
            for (int a = -nimg; a <= nimg; ++a)
            for (int bb = -nimg; bb <= nimg; ++bb)
            for (int c = -nimg; c <= nimg; ++c) {
                double dx = px[j] + (periodic ? a * L : 0.0) - px[i];
                double dy = py[j] + (periodic ? bb * L : 0.0) - py[i];
                double dz = pz[j] + (periodic ? c * L : 0.0) - pz[i];
                double tc = dx * dir[0] + dy * dir[1] + dz * dir[2];
                double cx = dy * dir[2] - dz * dir[1];
                double cy = dz * dir[0] - dx * dir[2];
                double cz = dx * dir[1] - dy * dir[0];
                double b2 = cx * cx + cy * cy + cz * cz;
                if (b2 >= hj * hj) continue;
                double half = sqrt(hj * hj - b2);
                double t1 = fmax(0.0, tc - half), t2 = fmin(l_ray, tc + half);
                if (t2 <= t1) continue;
                double F = oracle_chord(kernel, sqrt(b2) / hj, (t1 - tc) / hj, (t2 - tc) / hj);
                double hcm = hj * unit_cm;
                double col = mass_H[j] * (8.0 / OR_PI) / (hcm * hcm) * F;
                if (dx * dx + dy * dy + dz * dz < hj * hj) near += col;
                else far += col * x[j];
            }
        }
        tau_far[r] = sth * far;
        tau_near[r] = sth * near;
    }
}

/* ------------------------------------------------------------------------ */
/* HEALPix ray directions (Sec. 3.2; Gorski et al. 2005 ring scheme).       */
/* ------------------------------------------------------------------------ */

/* Pixel centres of the ring scheme, pixel p -> (z, phi):
 * north cap rings i < N_side hold 4i pixels at z = 1 - i^2/(3 N_side^2),
 * phi = pi/(2i) (j - 1/2); equatorial rings N_side <= i <= 3 N_side hold
 * 4 N_side pixels at z = 4/3 - 2i/(3 N_side), phi = pi/(2 N_side) (j - s/2)
 * with s = (i - N_side + 1) mod 2; the south cap mirrors the north. */
void oracle_healpix(int nside, double* dirs)
{
    int64_t npix = 12LL * nside * nside;
    int64_t ncap = 2LL * nside * (nside - 1);
    for (int64_t p = 0; p < npix; ++p) {
        double z, phi;
        if (p < ncap) {
            double ph = 0.5 * (double)(p + 1);
            int64_t i = (int64_t)floor(sqrt(ph - sqrt(floor(ph)))) + 1;
            int64_t j = p + 1 - 2 * i * (i - 1);
            z = 1.0 - (double)(i * i) / (3.0 * nside * nside);
            phi = OR_PI / (2.0 * i) * ((double)j - 0.5);
        } else if (p < npix - ncap) {
            int64_t pp = p - ncap;
            int64_t i = pp / (4 * nside) + nside;
            int64_t j = pp % (4 * nside) + 1;
            int64_t s = (i - nside + 1) % 2;
            z = 4.0 / 3.0 - 2.0 * (double)i / (3.0 * nside);
            phi = OR_PI / (2.0 * nside) * ((double)j - 0.5 * (double)s);
        } else {
            int64_t pp = npix - p;
            double ph = 0.5 * (double)pp;
            int64_t i = (int64_t)floor(sqrt(ph - sqrt(floor(ph)))) + 1;
            int64_t j = 4 * i + 1 - (pp - 2 * i * (i - 1));
            z = -1.0 + (double)(i * i) / (3.0 * nside * nside);
            phi = OR_PI / (2.0 * i) * ((double)j - 0.5);
        }
        double st = sqrt(fmax(0.0, 1.0 - z * z));
        dirs[3 * p] = st * cos(phi);
        dirs[3 * p + 1] = st * sin(phi);
        dirs[3 * p + 2] = z;
    }
}

/* ------------------------------------------------------------------------ */
/* Shielded photoionisation rate, Eq. gamma_shld.                           */
/* ------------------------------------------------------------------------ */

/* Gamma_i = (1/N_ray) sum_k sum_j w_j exp(-s_j tau_ik), the 4 pi of
 * Eq. gamma_shld being absorbed in w (sum_j w_j = Gamma_thin), and
 * tau_eff = -ln(Gamma_i / Gamma_thin). */
void oracle_gamma(const double* tau, int64_t n_orig, int R, int F,
                  const double* s, const double* w, double* gamma_out, double* tau_eff_out)
{
    double gthin = 0.0;
    for (int j = 0; j < F; ++j) gthin += w[j];
#pragma omp parallel for schedule(static)
    for (int64_t o = 0; o < n_orig; ++o) {
        double g = 0.0;
        for (int k = 0; k < R; ++k)
            for (int j = 0; j < F; ++j)
                g += w[j] * exp(-s[j] * tau[o * R + k]);
        g /= (double)R;
        gamma_out[o] = g;
        if (tau_eff_out) tau_eff_out[o] = -log(g / gthin);
    }
}

/* Hydrogen photoionisation rate behind columns of H I, He I and He II (the
 * paper treats hydrogen only; helium columns attenuate the same spectrum):
 * tau, tau1, tau2 are the three columns in units of the H I threshold cross
 * section (N sigma_th) and s, s1, s2 the cross sections of each species in
 * the bins in the same units (zero below a species' threshold):
 *   Gamma_o = (1/R) sum_k sum_j w_j exp(-(s_j tau_ok + s1_j tau1_ok + s2_j tau2_ok)). */
void oracle_gamma_he(const double* tau, const double* tau1, const double* tau2, int64_t n_orig, int R, int F,
                     const double* s, const double* s1, const double* s2, const double* w,
                     double* gamma_out, double* tau_eff_out)
{
    double gthin = 0.0;
    for (int j = 0; j < F; ++j) gthin += w[j];
#pragma omp parallel for schedule(static)
    for (int64_t o = 0; o < n_orig; ++o) {
        double g = 0.0;
        for (int k = 0; k < R; ++k) {
            int64_t r = o * R + k;
            for (int j = 0; j < F; ++j) g += w[j] * exp(-(s[j] * tau[r] + s1[j] * tau1[r] + s2[j] * tau2[r]));
        }
        g /= (double)R;
        gamma_out[o] = g;
        if (tau_eff_out) tau_eff_out[o] = -log(g / gthin);
    }
}

/* ------------------------------------------------------------------------ */
/* Rate coefficients (App. C3 refers to published fits; Hui & Gnedin 1997). */
/* ------------------------------------------------------------------------ */

/* lambda = 2 T_HI / T with T_HI = 157807 K.
 *   alpha_A = 1.269e-13 lambda^1.503 / [1 + (lambda/0.522)^0.470]^1.923
 *   alpha_B = 2.753e-14 lambda^1.500 / [1 + (lambda/2.740)^0.407]^2.242
 *   gamma   = 21.11 T^-1.5 exp(-lambda/2) lambda^-1.089
 *             / [1 + (lambda/0.354)^0.874]^1.101          (cm^3 s^-1) */
void oracle_rates(double T, double* alphaA, double* alphaB, double* gamma_c)
{
    double lam = 2.0 * 157807.0 / T;
    if (alphaA) *alphaA = 1.269e-13 * pow(lam, 1.503) / pow(1.0 + pow(lam / 0.522, 0.470), 1.923);
    if (alphaB) *alphaB = 2.753e-14 * pow(lam, 1.500) / pow(1.0 + pow(lam / 2.740, 0.407), 2.242);
    if (gamma_c) *gamma_c = 21.11 * pow(T, -1.5) * exp(-0.5 * lam) * pow(lam, -1.089)
                            / pow(1.0 + pow(lam / 0.354, 0.874), 1.101);
}

/* ------------------------------------------------------------------------ */
/* Ionisation equilibrium, App. C3 (Eqs. dxdt, xroots, xphys).              */
/* ------------------------------------------------------------------------ */

/* Physical root x_- of R x^2 + Q x + P = 0 with
 *   R = (gamma + alpha) n_H,  Q = -[Gamma + alpha n_H + R (1 + y)],
 *   P = alpha n_H (1 + y),
 * written 2P / (-Q + sqrt(Q^2 - 4PR)) (equal to x_- by Vieta).  The
 * discriminant is evaluated through the identity
 *   Q^2 - 4PR = (Gamma + R(1+y) - alpha n_H)^2 + 4 Gamma alpha n_H,
 *   R(1+y) - alpha n_H = alpha n_H y + gamma n_H (1+y),
 * whose terms are all non-negative, so it does not cancel when
 * gamma << alpha (near-neutral gas). */
double oracle_xeq(double Gamma, double nH, double T, double y, int caseB)
{
    double aA, aB, gc;
    oracle_rates(T, &aA, &aB, &gc);
    double alpha = caseB ? aB : aA;
    double R = (gc + alpha) * nH;
    double Q = -(Gamma + alpha * nH + R * (1.0 + y));
    double P = alpha * nH * (1.0 + y);
    double excess = alpha * nH * y + gc * nH * (1.0 + y);
    double disc = (Gamma + excess) * (Gamma + excess) + 4.0 * Gamma * alpha * nH;
    return 2.0 * P / (-Q + sqrt(disc));
}

/* d x_- / d Gamma by implicit differentiation of f(x, Gamma) = R x^2 + Q x + P
 * = 0, where only Q depends on Gamma (dQ/dGamma = -1):
 *   dx/dGamma = -(df/dGamma) / (df/dx) = x / (2 R x + Q). */
double oracle_xeq_dgamma(double Gamma, double nH, double T, double y, int caseB)
{
    double aA, aB, gc;
    oracle_rates(T, &aA, &aB, &gc);
    double alpha = caseB ? aB : aA;
    double R = (gc + alpha) * nH;
    double Q = -(Gamma + alpha * nH + R * (1.0 + y));
    double x = oracle_xeq(Gamma, nH, T, y, caseB);
    return x / (2.0 * R * x + Q);
}

/* Photoionisation rate at the far side of a uniform hydrogen slab (App.
 * "Neutral fraction in a plane parallel slab", y = 0): monochromatic
 * radiation at the threshold with rate Gamma0 at the surface, density nH,
 * temperature T, recombination case caseB, slab thickness
 * tau_near = N_H sigma_th (all hydrogen, neutral or not).  In equilibrium
 * Gamma(z) x = nH X(x), X = alpha (1-x)^2 - gamma (1-x) x, and the depth at
 * which the neutral fraction is x obeys
 *   z nH sigma = (1/x0 - 1/x) + ln[x (1-x0) / (x0 (1-x))]
 *                + (1/x_ce) ln[x (x_ce - x0) / (x0 (x_ce - x))],
 * with x0 = x(0) (equilibrium with Gamma0) and x_ce = alpha/(alpha+gamma).
 * Solved for the bottom value x_b at z nH sigma = tau_near by bisection in
 * y = ln[x / (x_ce - x)], which resolves both a strongly ionised bottom
 * (x << x_ce) and a neutral one (x_ce - x below double resolution); then
 * Gamma_b = nH X(x_b) / x_b = nH (1-x_b) (alpha+gamma) (x_ce - x_b) / x_b.
 * Every 1 - x is formed as c + (x_ce - x), c = 1 - x_ce = gamma/(alpha+gamma),
 * and x_ce - x0 from the surface equilibrium D (c + D) = Gamma0 x0 /
 * (nH (alpha+gamma)) (exact rewrites that do not cancel in cold, nearly
 * neutral gas where x_ce rounds to 1).  Returns ln Gamma_b (-inf for
 * Gamma0 = 0). */
static double log1pexp(double y) { return y > 0.0 ? y + log1p(exp(-y)) : log1p(exp(y)); }

double oracle_slab_lngamma(double Gamma0, double nH, double T, int caseB, double tau_near)
{
    if (!(Gamma0 > 0.0)) return -INFINITY;
    if (tau_near <= 0.0) return log(Gamma0);
    double aA, aB, gc;
    oracle_rates(T, &aA, &aB, &gc);
    double alpha = caseB ? aB : aA;
    double ag = alpha + gc;
    double xce = alpha / ag;
    double c = gc / ag;                            /* 1 - x_ce */
    double x0 = oracle_xeq(Gamma0, nH, T, 0.0, caseB);
    double K = Gamma0 * x0 / (nH * ag);
    double d0 = 2.0 * K / (c + sqrt(c * c + 4.0 * K));   /* x_ce - x0 */
    double ylo = log(x0) - log(d0);                /* depth 0 */
    double yhi = log(xce) - log(d0) + xce * tau_near + 50.0;   /* deeper than the slab */
    for (int it = 0; it < 400; ++it) {
        double y = 0.5 * (ylo + yhi);
        double lx = log(xce) - log1pexp(-y), le = log(xce) - log1pexp(y);
        double x = exp(lx), e = exp(le);
        double depth = (1.0 / x0 - 1.0 / x) + (lx - log(x0)) + log(c + d0) - log(c + e)
                       + (1.0 / xce) * (lx - log(x0) + log(d0) - le);
        if (depth > tau_near) yhi = y;
        else ylo = y;
    }
    double y = 0.5 * (ylo + yhi);
    double lx = log(xce) - log1pexp(-y), le = log(xce) - log1pexp(y);
    return log(nH) + log(c + exp(le)) + log(ag) + le - lx;
}

/* ln sum_b w_b exp(-s_b tau), factored so that it does not underflow. */
static double ln_spec_rate(int F, const double* s, const double* w, double tau)
{
    double smin = s[0];
    for (int b = 1; b < F; ++b) smin = fmin(smin, s[b]);
    double acc = 0.0;
    for (int b = 0; b < F; ++b) acc += w[b] * exp(-(s[b] - smin) * tau);
    return -smin * tau + log(acc);
}

/* The same slab for a polychromatic spectrum (the numerical slab solution
 * the paper tabulates for Eq. gammashldk; y = 0): the slab of thickness
 * tau_near = N_H sigma_th, density nH and temperature T is lit by the
 * spectrum (s_b = sigma_b / sigma_th, w_b) already attenuated by the far
 * column tau_far (at threshold).  With t = sigma_th nH z and tau_HI(t) the
 * neutral column inside the slab (at threshold),
 *   dtau_HI/dt = x(t),  x(t) = x_eq(Gamma(t)),
 *   Gamma(t) = sum_b w_b exp(-s_b (tau_far + tau_HI(t))),
 * integrated over t in [0, tau_near] with the Dormand-Prince 5(4) pair
 * (adaptive steps, relative tolerance 1e-11).  Returns
 * ln Gamma(tau_near) = ln sum_b w_b exp(-s_b (tau_far + tau_HI(tau_near))). */
static double slab_rhs(int F, const double* s, const double* w, double tau_far, double nH, double T, int caseB,
                       double u)
{
    double lg = ln_spec_rate(F, s, w, tau_far + u);
    return oracle_xeq(exp(lg), nH, T, 0.0, caseB);
}

double oracle_slab_poly_lngamma(int F, const double* s, const double* w, double tau_far, double nH, double T,
                                int caseB, double tau_near)
{
    static const double a21 = 1.0 / 5, a31 = 3.0 / 40, a32 = 9.0 / 40, a41 = 44.0 / 45, a42 = -56.0 / 15,
                        a43 = 32.0 / 9, a51 = 19372.0 / 6561, a52 = -25360.0 / 2187, a53 = 64448.0 / 6561,
                        a54 = -212.0 / 729, a61 = 9017.0 / 3168, a62 = -355.0 / 33, a63 = 46732.0 / 5247,
                        a64 = 49.0 / 176, a65 = -5103.0 / 18656, b1 = 35.0 / 384, b3 = 500.0 / 1113,
                        b4 = 125.0 / 192, b5 = -2187.0 / 6784, b6 = 11.0 / 84, e1 = 71.0 / 57600,
                        e3 = -71.0 / 16695, e4 = 71.0 / 1920, e5 = -17253.0 / 339200, e6 = 22.0 / 525,
                        e7 = -1.0 / 40;
    double t = 0.0, u = 0.0;
    double h = fmin(tau_near, 1e-3);
    double k1 = slab_rhs(F, s, w, tau_far, nH, T, caseB, u);
    int guard = 0;
    while (t < tau_near && guard++ < 10000000) {
        if (t + h > tau_near) h = tau_near - t;
        double k2 = slab_rhs(F, s, w, tau_far, nH, T, caseB, u + h * a21 * k1);
        double k3 = slab_rhs(F, s, w, tau_far, nH, T, caseB, u + h * (a31 * k1 + a32 * k2));
        double k4 = slab_rhs(F, s, w, tau_far, nH, T, caseB, u + h * (a41 * k1 + a42 * k2 + a43 * k3));
        double k5 = slab_rhs(F, s, w, tau_far, nH, T, caseB, u + h * (a51 * k1 + a52 * k2 + a53 * k3 + a54 * k4));
        double k6 = slab_rhs(F, s, w, tau_far, nH, T, caseB,
                             u + h * (a61 * k1 + a62 * k2 + a63 * k3 + a64 * k4 + a65 * k5));
        double un = u + h * (b1 * k1 + b3 * k3 + b4 * k4 + b5 * k5 + b6 * k6);
        double k7 = slab_rhs(F, s, w, tau_far, nH, T, caseB, un);
        double err = h * fabs(e1 * k1 + e3 * k3 + e4 * k4 + e5 * k5 + e6 * k6 + e7 * k7);
        double tol = 1e-11 * fmax(fabs(un), 1e-3 * h) + 1e-300;
        if (err <= tol) {
            t += h;
            u = un;
            k1 = k7;
        }
        double fac = err > 0.0 ? 0.9 * pow(tol / err, 0.2) : 5.0;
        h *= fmin(5.0, fmax(0.2, fac));
    }
    return ln_spec_rate(F, s, w, tau_far + u);
}

/* The numerical slab solver of Test 1 (NS): plane-parallel radiation with
 * the binned spectrum (s_b, w_b = its rate contributions at the surface)
 * onto a uniform hydrogen slab of total thickness tau_total = N_H sigma_th,
 * density nH, temperature T, recombination case caseB, y = 0.  The slab is
 * cut into n_slices equal slices; going down from the surface, each slice
 * takes the neutral column above it, tau = sum over the slices above of
 * x dtau_H, the rate Gamma = sum_b w_b exp(-s_b tau), and x = x_eq(Gamma)
 * (Eq. xroots).  Writes x of every slice (x_out, may be NULL) and returns
 * the neutral column through the slab, N_HI sigma_th = sum x dtau_H. */
double oracle_ns_slab(int F, const double* s, const double* w, double nH, double T, int caseB, double tau_total,
                      int64_t n_slices, double* x_out)
{
    double dt = tau_total / (double)n_slices;
    double tau = 0.0;
    for (int64_t i = 0; i < n_slices; ++i) {
        double g = exp(ln_spec_rate(F, s, w, tau));
        double x = oracle_xeq(g, nH, T, 0.0, caseB);
        if (x_out) x_out[i] = x;
        tau += x * dt;
    }
    return tau;
}

/* NS for Test 3: the same slab lit from both sides, each side with half of
 * the rate (w_b / 2 per side, so that thin gas keeps sum_b w_b).  Starting
 * from the optically thin x, every slice takes the neutral columns above
 * and below it from the previous pass, Gamma = (1/2) sum_b w_b
 * [exp(-s_b tau_above) + exp(-s_b tau_below)], x = x_eq(Gamma); passes
 * repeat until no slice changes by more than tol (relative) or max_pass.
 * Writes x per slice and returns the total N_HI sigma_th. */
double oracle_ns_slab2(int F, const double* s, const double* w, double nH, double T, int caseB, double tau_total,
                       int64_t n_slices, double tol, int max_pass, double* x_out)
{
    double dt = tau_total / (double)n_slices;
    double* x = (double*)malloc(sizeof(double) * (size_t)n_slices);
    double* xn = (double*)malloc(sizeof(double) * (size_t)n_slices);
    double* above = (double*)malloc(sizeof(double) * (size_t)n_slices);
    double g0 = 0.0;
    for (int b = 0; b < F; ++b) g0 += w[b];
    for (int64_t i = 0; i < n_slices; ++i) x[i] = oracle_xeq(g0, nH, T, 0.0, caseB);
    for (int pass = 0; pass < max_pass; ++pass) {
        double acc = 0.0, total = 0.0;
        for (int64_t i = 0; i < n_slices; ++i) total += x[i] * dt;
        double maxrel = 0.0;
        for (int64_t i = 0; i < n_slices; ++i) {
            above[i] = acc;
            acc += x[i] * dt;
        }
        for (int64_t i = 0; i < n_slices; ++i) {
            double below = total - above[i] - x[i] * dt;
            double g = 0.5 * (exp(ln_spec_rate(F, s, w, above[i])) + exp(ln_spec_rate(F, s, w, below)));
            xn[i] = oracle_xeq(g, nH, T, 0.0, caseB);
            double rel = fabs(xn[i] - x[i]) / x[i];
            if (rel > maxrel) maxrel = rel;
        }
        memcpy(x, xn, sizeof(double) * (size_t)n_slices);
        if (maxrel < tol) break;
    }
    double tot = 0.0;
    for (int64_t i = 0; i < n_slices; ++i) {
        tot += x[i] * dt;
        if (x_out) x_out[i] = x[i];
    }
    free(x); free(xn); free(above);
    return tot;
}

/* Shielded rate with the near/far split (Sec. 3.3.3, Eqs. gammafar,
 * gammashldk, gammashld).  Ray k carries the share 4 pi / N_ray of the
 * radiation, here (1/R) of the spectrum weights w (sum_j w_j = Gamma_thin);
 * its slab of near particles is lit by that share attenuated by the far
 * column, Gamma_far,k = (1/R) sum_j w_j exp(-s_j tau_far,k), and the
 * particle's rate is the sum of the slabs' bottom rates,
 * Gamma = sum_k G(Gamma_far,k, nH, T, tau_near,k).  Reading: a slab lit by
 * its ray's share reproduces the one-sided slab test exactly (one ray) and
 * makes each slab miss the other directions' radiation, the shortcoming the
 * paper gives for its two-sided slab test.
 * caseB[o] is the recombination case used inside the slab; poly = 0 takes
 * the analytic slab (radiation at the threshold with the far rate), poly = 1
 * the polychromatic slab (oracle_slab_poly_lngamma).  Writes
 * ln(Gamma / Gamma_thin) per origin (log-sum-exp over rays, finite where
 * Gamma underflows) and Gamma. */
void oracle_gamma_nearfar(const double* tau_far, const double* tau_near, int64_t n_orig, int R, int F,
                          const double* s, const double* w, const double* nH, const double* T,
                          const int* caseB, int poly, double* lnratio_out, double* gamma_out)
{
    double gthin = 0.0;
    for (int j = 0; j < F; ++j) gthin += w[j];
    double* wsh = (double*)malloc(sizeof(double) * (size_t)F);   /* one ray's share */
    for (int j = 0; j < F; ++j) wsh[j] = w[j] / (double)R;
#pragma omp parallel for schedule(static)
    for (int64_t o = 0; o < n_orig; ++o) {
        double lk[512];
        double m = -INFINITY;
        for (int k = 0; k < R; ++k) {
            if (poly) {
                lk[k] = oracle_slab_poly_lngamma(F, s, wsh, tau_far[o * R + k], nH[o], T[o], caseB[o],
                                                 tau_near[o * R + k]) - log(gthin);
            } else {
                double gf = 0.0;
                for (int j = 0; j < F; ++j) gf += wsh[j] * exp(-s[j] * tau_far[o * R + k]);
                lk[k] = oracle_slab_lngamma(gf, nH[o], T[o], caseB[o], tau_near[o * R + k]) - log(gthin);
            }
            if (lk[k] > m) m = lk[k];
        }
        if (m == -INFINITY) {
            /* no ray's radiation reaches the origin: the rate is the empty sum */
            lnratio_out[o] = -INFINITY;
            gamma_out[o] = 0.0;
            continue;
        }
        double acc = 0.0;
        for (int k = 0; k < R; ++k) acc += exp(lk[k] - m);
        double lr = m + log(acc);
        lnratio_out[o] = lr;
        gamma_out[o] = gthin * exp(lr);
    }
    free(wsh);
}

/* Case choice (Sec. 3.3.3 / Sec. 4): 0 = always A, 1 = always B,
 * 2 = B when tau_eff >= 1.  In the iteration driver rule 2 is latched: a
 * particle that has once had tau_eff >= 1 keeps case B (see oracle_solve). */
static int use_caseB(int case_rule, double tau_eff)
{
    if (case_rule == 0) return 0;
    if (case_rule == 1) return 1;
    return tau_eff >= 1.0;
}

/* ------------------------------------------------------------------------ */
/* Iteration driver, Sec. 4 (initial x_thin, tau_skip freeze, dx_tol).      */
/* ------------------------------------------------------------------------ */

/* Runs the Jacobi iteration:
 *   x <- x_thin (Gamma = Gamma_thin, tau_eff = 0);
 *   sweep 0 traces every particle, freezes those with tau_eff < tau_skip at
 *   x_thin for good and updates the others;
 *   later sweeps trace the non-frozen particles only, computing every Gamma
 *   from the previous sweep's x before any x changes;
 *   stop when max over non-frozen particles of |x_new - x| / x < tol, or
 *   after max_iter sweeps.
 * The case rule "B when tau_eff >= 1" is applied as a latch: once a
 * particle has reached tau_eff >= 1 in some sweep it keeps case B.  Read
 * literally, the rule has no self-consistent state for particles whose
 * case-A equilibrium is thick and case-B equilibrium thin, and the Jacobi
 * iteration then alternates between the two forever; the latch settles
 * them in case B.
 * If max_iter < 0 the run does exactly -max_iter sweeps (step-matched mode).
 * blocks > 1 selects the update order of Sec. 4 instead of Jacobi: after
 * sweep 0 the non-frozen particles are ordered from high to low density
 * (n_H rounded to float, ties by particle index), cut into `blocks`
 * contiguous blocks of sizes floor((b+1) m / blocks) - floor(b m / blocks),
 * and each sweep updates block after block, every block's columns using the
 * x of the blocks already updated in that sweep.
 * near_far = 1 (analytic slab) or 2 (polychromatic slab) replaces the
 * columns and Gamma by the near/far split of Sec. 3.3.3
 * (oracle_columns_nearfar, oracle_gamma_nearfar): the slab of
 * near particles uses each particle's case before the sweep (its latch, or
 * the forced case), then tau_eff = -ln(Gamma/Gamma_thin) decides the case
 * of the update as above.  It needs blocks <= 1 (returns 2 otherwise).
 * he_tau1 / he_tau2 (optional, [n*R] per particle and ray, fixed) are He I
 * and He II columns that attenuate the spectrum with the bin cross sections
 * he_s1 / he_s2 (oracle_gamma_he); they need near_far = 0 and blocks <= 1.
 * x_out[n] receives the final x, frozen_out[n] (optional) 1 for frozen
 * particles, caseB_out[n] (optional) 1 where the final update used case B,
 * stats[0] = sweeps done, stats[1] = last max |dx|/x,
 * stats[2] = rays traced.  x_start (optional) replaces x_thin as the start
 * (sweep 0 still applies the freeze rule).  grid_cell > 0 takes the columns
 * from the uniform-grid query with cells of about that size (not with the
 * near/far split).  Returns 0 when converged, 1 when the sweep limit ended
 * the run, 3 when the grid cannot be built (a sphere spanning the box). */
static const double* g_sort_nH;
static int by_density(const void* a, const void* b)
{
    int64_t i = *(const int64_t*)a, j = *(const int64_t*)b;
    float fi = (float)g_sort_nH[i], fj = (float)g_sort_nH[j];
    if (fi > fj) return -1;
    if (fi < fj) return 1;
    return (i > j) - (i < j);
}

/* Columns for the driver: brute force, or the grid query when a grid is given. */
static void solve_columns(const oracle_grid* grid, int64_t n, const double* px, const double* py,
                          const double* pz, const double* h, const double* mass_H, const double* x, int periodic,
                          double L, double unit_cm, const int64_t* origins, int64_t n_orig, const double* dirs,
                          int R, double l_ray, int kernel, double* tau)
{
    if (grid)
        oracle_grid_columns(grid, px, py, pz, h, mass_H, x, unit_cm, origins, n_orig, dirs, R, l_ray, kernel, tau);
    else
        oracle_columns(n, px, py, pz, h, mass_H, x, periodic, L, unit_cm, origins, n_orig, dirs, R, l_ray, kernel,
                       tau);
}

int oracle_solve(int64_t n, const double* px, const double* py, const double* pz,
                 const double* h, const double* mass_H, const double* nH, const double* T,
                 double y, int periodic, double L, double unit_cm,
                 const double* dirs, int R, double l_ray, int kernel,
                 int F, const double* s, const double* w,
                 double tol, double tau_skip, int max_iter, int case_rule, int blocks, int near_far,
                 const double* he_tau1, const double* he_tau2, const double* he_s1, const double* he_s2,
                 const double* x_start, double* x_out, int* frozen_out, int* caseB_out, double* stats,
                 double grid_cell)
{
    if (he_tau1 && (near_far || blocks > 1)) return 2;
    if (near_far && blocks > 1) return 2;
    /* grid_cell > 0: columns by the uniform-grid query (oracle_grid_columns)
     * instead of brute force; the grid holds positions only, so one build
     * serves every sweep */
    oracle_grid* grid = NULL;
    if (grid_cell > 0.0 && !near_far) {
        grid = oracle_grid_build(n, px, py, pz, h, periodic, L, grid_cell);
        if (!grid) return 3;
    }
    double gthin = 0.0;
    for (int j = 0; j < F; ++j) gthin += w[j];
    double* x = x_out;
    int* frozen = (int*)calloc((size_t)n, sizeof(int));
    int* latchB = (int*)calloc((size_t)n, sizeof(int));
    double* tau = (double*)malloc(sizeof(double) * (size_t)n * R);
    double* tau_nr = near_far ? (double*)malloc(sizeof(double) * (size_t)n * R) : NULL;
    double* nH_o = near_far ? (double*)malloc(sizeof(double) * (size_t)n) : NULL;
    double* T_o = near_far ? (double*)malloc(sizeof(double) * (size_t)n) : NULL;
    int* cb_o = near_far ? (int*)malloc(sizeof(int) * (size_t)n) : NULL;
    double* he1_o = he_tau1 ? (double*)malloc(sizeof(double) * (size_t)n * R) : NULL;
    double* he2_o = he_tau1 ? (double*)malloc(sizeof(double) * (size_t)n * R) : NULL;
    double* G = (double*)malloc(sizeof(double) * (size_t)n);
    double* te = (double*)malloc(sizeof(double) * (size_t)n);
    double* xn = (double*)malloc(sizeof(double) * (size_t)n);
    int64_t* act = (int64_t*)malloc(sizeof(int64_t) * (size_t)n);
    for (int64_t i = 0; i < n; ++i)
        x[i] = x_start ? x_start[i] : oracle_xeq(gthin, nH[i], T[i], y, use_caseB(case_rule, 0.0));
    int fixed = max_iter < 0;
    int limit = fixed ? -max_iter : max_iter;
    int sweeps = 0, converged = 0;
    double maxrel = 0.0, rays = 0.0;
    int64_t nact = n;
    for (int64_t i = 0; i < n; ++i) act[i] = i;
    while (sweeps < limit) {
        if (sweeps == 0 || blocks <= 1) {
            if (near_far) {
                oracle_columns_nearfar(n, px, py, pz, h, mass_H, x, periodic, L, unit_cm,
                                       act, nact, dirs, R, l_ray, kernel, tau, tau_nr);
                for (int64_t o = 0; o < nact; ++o) {
                    int64_t i = act[o];
                    nH_o[o] = nH[i];
                    T_o[o] = T[i];
                    cb_o[o] = use_caseB(case_rule, 0.0) || (case_rule == 2 && latchB[i]);
                }
                oracle_gamma_nearfar(tau, tau_nr, nact, R, F, s, w, nH_o, T_o, cb_o, near_far == 2, te, G);
                for (int64_t o = 0; o < nact; ++o) te[o] = -te[o];
            } else if (he_tau1) {
                solve_columns(grid, n, px, py, pz, h, mass_H, x, periodic, L, unit_cm,
                              act, nact, dirs, R, l_ray, kernel, tau);
                for (int64_t o = 0; o < nact; ++o)
                    for (int k = 0; k < R; ++k) {
                        he1_o[o * R + k] = he_tau1[act[o] * R + k];
                        he2_o[o * R + k] = he_tau2[act[o] * R + k];
                    }
                oracle_gamma_he(tau, he1_o, he2_o, nact, R, F, s, he_s1, he_s2, w, G, te);
            } else {
                solve_columns(grid, n, px, py, pz, h, mass_H, x, periodic, L, unit_cm,
                              act, nact, dirs, R, l_ray, kernel, tau);
                oracle_gamma(tau, nact, R, F, s, w, G, te);
            }
            rays += (double)nact * R;
            if (sweeps == 0) {
                int64_t m = 0;
                for (int64_t o = 0; o < nact; ++o) {
                    int64_t i = act[o];
                    if (te[o] < tau_skip) { frozen[i] = 1; continue; }
                    act[m] = i; G[m] = G[o]; te[m] = te[o]; ++m;
                }
                nact = m;
            }
            maxrel = 0.0;
            for (int64_t o = 0; o < nact; ++o) {
                int64_t i = act[o];
                int cb = use_caseB(case_rule, te[o]) || (case_rule == 2 && latchB[i]);
                latchB[i] = cb;
                xn[o] = oracle_xeq(G[o], nH[i], T[i], y, cb);
                double rel = fabs(xn[o] - x[i]) / x[i];
                if (rel > maxrel) maxrel = rel;
            }
            for (int64_t o = 0; o < nact; ++o) x[act[o]] = xn[o];
            if (sweeps == 0 && blocks > 1) {
                g_sort_nH = nH;
                qsort(act, (size_t)nact, sizeof(int64_t), by_density);
            }
        } else {
            maxrel = 0.0;
            for (int b = 0; b < blocks; ++b) {
                int64_t lo = (b * nact) / blocks;
                int64_t hi = ((b + 1) * nact) / blocks;
                int64_t m = hi - lo;
                if (m <= 0) continue;
                solve_columns(grid, n, px, py, pz, h, mass_H, x, periodic, L, unit_cm,
                              act + lo, m, dirs, R, l_ray, kernel, tau);
                oracle_gamma(tau, m, R, F, s, w, G, te);
                rays += (double)m * R;
                for (int64_t o = 0; o < m; ++o) {
                    int64_t i = act[lo + o];
                    int cb = use_caseB(case_rule, te[o]) || (case_rule == 2 && latchB[i]);
                    latchB[i] = cb;
                    double xv = oracle_xeq(G[o], nH[i], T[i], y, cb);
                    double rel = fabs(xv - x[i]) / x[i];
                    if (rel > maxrel) maxrel = rel;
                    xn[o] = xv;
                }
                for (int64_t o = 0; o < m; ++o) x[act[lo + o]] = xn[o];
            }
        }
        ++sweeps;
        if (!fixed && maxrel < tol) { converged = 1; break; }
    }
    if (frozen_out) for (int64_t i = 0; i < n; ++i) frozen_out[i] = frozen[i];
    if (caseB_out) for (int64_t i = 0; i < n; ++i) caseB_out[i] = frozen[i] ? use_caseB(case_rule, 0.0) : latchB[i];
    if (stats) { stats[0] = sweeps; stats[1] = maxrel; stats[2] = rays; }
    free(frozen); free(latchB); free(tau); free(G); free(te); free(xn); free(act);
    free(tau_nr); free(nH_o); free(T_o); free(cb_o); free(he1_o); free(he2_o);
    oracle_grid_free(grid);
    return (fixed || converged) ? 0 : 1;
}

/* Columns are linear in x (Eq. colden): tau = M x with
 *   M[(o R + k) n + j] = sigma_th (m_j / m_p) int_0^{l_ray} W(|r_o + t n_k - r_j| / h_j) dt,
 * summed over the periodic images of j.  Brute force, like oracle_columns. */
void oracle_column_matrix(int64_t n, const double* px, const double* py, const double* pz,
                          const double* h, const double* mass_H,
                          int periodic, double L, double unit_cm,
                          const int64_t* origins, int64_t n_orig,
                          const double* dirs, int R, double l_ray, int kernel, double* M)
{
    int nimg = image_range(periodic, L, n, h, l_ray);
    int64_t total = n_orig * (int64_t)R;
    double sth = oracle_sigma_th();
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t r = 0; r < total; ++r) {
        int64_t o = r / R;
        int k = (int)(r % R);
        int64_t i = origins ? origins[o] : o;
        const double* dir = dirs + 3 * k;
        double* row = M + r * n;
        for (int64_t j = 0; j < n; ++j) {
            double hj = h[j], acc = 0.0;
            for (int a = -nimg; a <= nimg; ++a)
            for (int bb = -nimg; bb <= nimg; ++bb)
            for (int c = -nimg; c <= nimg; ++c) {
                double dx = px[j] + (periodic ? a * L : 0.0) - px[i];
                double dy = py[j] + (periodic ? bb * L : 0.0) - py[i];
                double dz = pz[j] + (periodic ? c * L : 0.0) - pz[i];
                double tc = dx * dir[0] + dy * dir[1] + dz * dir[2];
                double cx = dy * dir[2] - dz * dir[1];
                double cy = dz * dir[0] - dx * dir[2];
                double cz = dx * dir[1] - dy * dir[0];
                double b2 = cx * cx + cy * cy + cz * cz;
                if (b2 >= hj * hj) continue;
                double half = sqrt(hj * hj - b2);
                double t1 = fmax(0.0, tc - half), t2 = fmin(l_ray, tc + half);
                if (t2 <= t1) continue;
                acc += oracle_chord(kernel, sqrt(b2) / hj, (t1 - tc) / hj, (t2 - tc) / hj);
            }
            double hcm = hj * unit_cm;
            row[j] = sth * mass_H[j] * (8.0 / OR_PI) / (hcm * hcm) * acc;
        }
    }
}

/* Directional derivative of the sweep map along v (for checking tangents):
 * dtau = sigma_th sum_j (m_j v_j / m_p) int W dl is the column of Eq. colden
 * with x replaced by v (columns are linear in x). */
void oracle_columns_linear(int64_t n, const double* px, const double* py, const double* pz,
                           const double* h, const double* mass_H, const double* v,
                           int periodic, double L, double unit_cm,
                           const int64_t* origins, int64_t n_orig,
                           const double* dirs, int R, double l_ray, int kernel, double* out)
{
    oracle_columns(n, px, py, pz, h, mass_H, v, periodic, L, unit_cm,
                   origins, n_orig, dirs, R, l_ray, kernel, out);
}

int oracle_num_threads(void)
{
#ifdef _OPENMP
    extern int omp_get_max_threads(void);
    return omp_get_max_threads();
#else
    return 1;
#endif
}
