/*
 * soap_oracle.c -- plain FP64 CPU oracle for the stellar-disk integration of SOAP-GPU
 * (Zhao & Dumusque, arXiv 2301.04259).
 *
 * TEST INFRASTRUCTURE.  Only the tests, the package smoke check and the CPU-baseline leg of
 * the benchmark may load this code.  It shares no code, header or constant table with the
 * CUDA library; it is deliberately slow and follows the paper's definitions step by step:
 *
 *   - Alg. 1 / Alg. 4 (quiet integration): for every disk cell, Doppler-shift the local
 *     spectrum (Eq. 6), project it back on the common grid by linear interpolation
 *     (Eqs. 9-11), weight it by the limb-darkening intensity and add it to the sum.
 *   - Alg. 5 (active regions): per time step, build the InfoMap (later regions in list
 *     order overwrite earlier ones), evaluate Eqs. 1-3 per active cell, sum them and apply
 *     Eq. 4.
 *   - Sect. 4.3.1: wavelength-dependent contrast = ratio of two Planck functions.
 *   - Sect. 4.1: CCF of the spectrum with a line mask (the RV is then the centre of a
 *     Gaussian fitted to it; the fit is done in oracle.py).
 *
 * Readings where the paper is silent:
 *   - the grid is log-uniform, lambda_n = lambda_s exp(n Delta), both ends included;
 *   - interpolation is a gather: output pixel m takes the shifted interval
 *     lambda'_n <= lambda_m < lambda'_{n+1} (Eqs. 9-10 read as a bracketing); outside the
 *     shifted grid the end values are repeated;
 *   - the Eq. 11 weight (lambda_m - lambda'_n)/(lambda'_{n+1} - lambda'_n) is evaluated in
 *     the algebraically identical, well-conditioned form
 *     expm1((m-n) Delta - atanh(beta)) / expm1(Delta), since ln D = atanh(beta);
 *   - cell (i,j) of an N x N grid has centre x = (2i+1-N)/N, y = (2j+1-N)/N, area (2/N)^2,
 *     is visible iff x^2+y^2 < 1 and has mu = sqrt(1-x^2-y^2); observer on +z, rotation
 *     axis (0, sin i, cos i), x > 0 recedes; v = vsini x (1 + alpha sin^2(latitude));
 *   - each cell uses the local spectrum of the nearest tabulated mu (ties: lower index);
 *   - a region is the spherical cap of angular radius asin(r) around its centre; at
 *     rotational phase p its longitude is lon + 360 p (1 + alpha sin^2 lat) degrees;
 *   - contrast is applied on the common grid, after the shift (Eqs. 1-3 multiply the
 *     shifted spectra by I_ratio(lambda)).
 *
 * Decisions that produce integers (visibility, mu bin, region membership) are written as
 * explicit FP64 operation sequences without contraction (-ffp-contract=off), so that the
 * CUDA path, which takes the same decisions in FP64, can reproduce them exactly.
 *
 * Sums over cells use Neumaier compensated summation in cell-index order.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_C_KMS 299792.458
#define OR_PI 3.14159265358979323846
/* Planck: h c / k_B in Angstrom Kelvin, from the exact SI values of h, c, k_B. */
#define OR_H 6.62607015e-34
#define OR_C_SI 299792458.0
#define OR_KB 1.380649e-23

/* ---------------------------------------------------------------------------------- */
/* compensated sum                                                                     */
/* ---------------------------------------------------------------------------------- */
typedef struct { double s, c; } or_sum;

static void or_add(or_sum* a, double x) {
    double t = a->s + x;
    if (fabs(a->s) >= fabs(x)) a->c += (a->s - t) + x;
    else a->c += (x - t) + a->s;
    a->s = t;
}
static double or_val(const or_sum* a) { return a->s + a->c; }

/* ---------------------------------------------------------------------------------- */
/* grid (Eq. 5 replaced by its log-uniform counterpart)                                */
/* ---------------------------------------------------------------------------------- */
/* Delta = ln(lambda_end / lambda_start) / (n_px - 1), evaluated as log1p of the exactly
 * representable difference: a plain log of a ratio close to 1 loses ~1e-13 relative. */
double or_delta(double lambda_start, double lambda_end, int64_t n_px) {
    return log1p((lambda_end - lambda_start) / lambda_start) / (double)(n_px - 1);
}

void or_grid(double lambda_start, double lambda_end, int64_t n_px, double* lam) {
    double d = or_delta(lambda_start, lambda_end, n_px);
    for (int64_t n = 0; n < n_px; n++) lam[n] = lambda_start * exp((double)n * d);
}

/* ---------------------------------------------------------------------------------- */
/* disk cells (Sect. 2.1, Fig. 0; differential rotation Sect. 3.4)                     */
/* ---------------------------------------------------------------------------------- */
typedef struct {
    int visible;
    double x, y, mu, I, v;
    int bin;
} or_cellgeo;

static int or_nearest_mu(double mu, int n_mu, const double* mu_values) {
    int best = 0;
    double bd = fabs(mu - mu_values[0]);
    for (int b = 1; b < n_mu; b++) {
        double d = fabs(mu - mu_values[b]);
        if (d < bd) { bd = d; best = b; }
    }
    return best;
}

static or_cellgeo or_cell(int N, int i, int j, double vsini, double incl_deg, double u1, double u2,
                          double alpha, int n_mu, const double* mu_values) {
    or_cellgeo g;
    g.x = (double)(2 * i + 1 - N) / (double)N;
    g.y = (double)(2 * j + 1 - N) / (double)N;
    double r2 = g.x * g.x + g.y * g.y;
    g.visible = r2 < 1.0;
    g.mu = 0.0; g.I = 0.0; g.v = 0.0; g.bin = -1;
    if (!g.visible) return g;
    g.mu = sqrt(1.0 - r2);
    double area = (2.0 / (double)N) * (2.0 / (double)N);
    double om = 1.0 - g.mu;
    /* quadratic limb darkening */
    g.I = area * (1.0 - u1 * om - u2 * om * om);
    double incl = incl_deg * (OR_PI / 180.0);
    /* sin(latitude) of the cell: projection on the rotation axis (0, sin i, cos i) */
    double slat = g.y * sin(incl) + g.mu * cos(incl);
    g.v = vsini * g.x * (1.0 + alpha * slat * slat);
    g.bin = or_nearest_mu(g.mu, n_mu, mu_values);
    return g;
}

/* Per-cell geometry for the whole grid, index j*N + i (i along x).  Invisible cells get
 * I = 0, v = 0, mu = 0, bin = -1. */
void or_cell_geometry(int N, double vsini, double incl_deg, double u1, double u2, double alpha,
                      int n_mu, const double* mu_values, double* I, double* v, double* mu,
                      int32_t* bin) {
    for (int j = 0; j < N; j++)
        for (int i = 0; i < N; i++) {
            or_cellgeo g = or_cell(N, i, j, vsini, incl_deg, u1, u2, alpha, n_mu, mu_values);
            int64_t k = (int64_t)j * N + i;
            I[k] = g.I; v[k] = g.v; mu[k] = g.mu; bin[k] = g.bin;
        }
}

/* ---------------------------------------------------------------------------------- */
/* Doppler shift + linear interpolation of one spectrum at one output pixel            */
/* (Eq. 6, Eqs. 9-11, gather form)                                                     */
/* ---------------------------------------------------------------------------------- */
double or_shift_interp(const double* lam, const double* S, int64_t n_px, double delta,
                       double beta, int64_t m) {
    /* Eq. 6: lambda'_n = lambda_n (1 + f(beta)), 1 + f = sqrt((1+beta)/(1-beta)) */
    double D = sqrt((1.0 + beta) / (1.0 - beta));
    double target = lam[m];
    if (target < lam[0] * D) return S[0];
    if (target >= lam[n_px - 1] * D) return S[n_px - 1];
    /* bracket lambda'_n <= lambda_m < lambda'_{n+1} by bisection on the shifted grid */
    int64_t lo = 0, hi = n_px - 1;           /* invariant: lam'[lo] <= target < lam'[hi] */
    while (hi - lo > 1) {
        int64_t mid = lo + (hi - lo) / 2;
        if (lam[mid] * D <= target) lo = mid; else hi = mid;
    }
    int64_t n = lo;
    /* Eq. 11: S'_m = (S_{n+1}-S_n) / (lambda'_{n+1}-lambda'_n) * (lambda_m - lambda'_n) + S_n,
     * with the ratio written as expm1((m-n) Delta - ln D) / expm1(Delta). */
    double w = expm1((double)(m - n) * delta - atanh(beta)) / expm1(delta);
    return (S[n + 1] - S[n]) * w + S[n];
}

/* ---------------------------------------------------------------------------------- */
/* Alg. 1: quiet spectrum integration                                                  */
/* ---------------------------------------------------------------------------------- */
typedef struct {
    int64_t n;          /* number of visible cells */
    int32_t* idx;       /* cell index j*N+i */
    double* I;
    double* beta;
    int32_t* bin;
    double* x;
    double* y;
    double* mu;
} or_disk;

static void or_disk_build(or_disk* d, int N, double vsini, double incl_deg, double u1, double u2,
                          double alpha, int n_mu, const double* mu_values) {
    int64_t cap = (int64_t)N * N;
    d->idx = (int32_t*)malloc(sizeof(int32_t) * cap);
    d->I = (double*)malloc(sizeof(double) * cap);
    d->beta = (double*)malloc(sizeof(double) * cap);
    d->bin = (int32_t*)malloc(sizeof(int32_t) * cap);
    d->x = (double*)malloc(sizeof(double) * cap);
    d->y = (double*)malloc(sizeof(double) * cap);
    d->mu = (double*)malloc(sizeof(double) * cap);
    d->n = 0;
    for (int j = 0; j < N; j++)
        for (int i = 0; i < N; i++) {
            or_cellgeo g = or_cell(N, i, j, vsini, incl_deg, u1, u2, alpha, n_mu, mu_values);
            if (!g.visible) continue;
            int64_t k = d->n++;
            d->idx[k] = j * N + i;
            d->I[k] = g.I;
            d->beta[k] = g.v / OR_C_KMS;
            d->bin[k] = g.bin;
            d->x[k] = g.x; d->y[k] = g.y; d->mu[k] = g.mu;
        }
}

static void or_disk_free(or_disk* d) {
    free(d->idx); free(d->I); free(d->beta); free(d->bin); free(d->x); free(d->y); free(d->mu);
}

/* pixel list: NULL means all pixels 0..n_px-1 */
static int64_t or_pix(const int64_t* pix, int64_t s) { return pix ? pix[s] : s; }

/* F_quiet at the requested pixels: sum over visible cells of I_XY * S'_quiet (Alg. 1).
 * quiet: [n_mu][n_px] row-major. out: [n_sample]. */
int or_quiet(int N, double vsini, double incl_deg, double u1, double u2, double alpha,
             int n_mu, const double* mu_values, double lambda_start, double lambda_end,
             int64_t n_px, const double* quiet, const int64_t* pix, int64_t n_sample,
             double* out) {
    double* lam = (double*)malloc(sizeof(double) * n_px);
    or_grid(lambda_start, lambda_end, n_px, lam);
    double delta = or_delta(lambda_start, lambda_end, n_px);
    or_disk d;
    or_disk_build(&d, N, vsini, incl_deg, u1, u2, alpha, n_mu, mu_values);
    #pragma omp parallel for schedule(dynamic, 4)
    for (int64_t s = 0; s < n_sample; s++) {
        int64_t m = or_pix(pix, s);
        or_sum acc = {0.0, 0.0};
        for (int64_t c = 0; c < d.n; c++) {
            const double* S = quiet + (int64_t)d.bin[c] * n_px;
            or_add(&acc, d.I[c] * or_shift_interp(lam, S, n_px, delta, d.beta[c], m));
        }
        out[s] = or_val(&acc);
    }
    or_disk_free(&d);
    free(lam);
    return 0;
}

/* ---------------------------------------------------------------------------------- */
/* Sect. 4.3.1: wavelength-dependent contrast, ratio of Planck functions               */
/* ---------------------------------------------------------------------------------- */
double or_planck_ratio(double lambda_A, double t_active, double t_quiet) {
    double hc_k = OR_H * OR_C_SI / OR_KB * 1e10;       /* Angstrom Kelvin */
    /* B(l,Ta)/B(l,Tq) = (exp(hc/lkTq) - 1) / (exp(hc/lkTa) - 1) */
    return expm1(hc_k / (lambda_A * t_quiet)) / expm1(hc_k / (lambda_A * t_active));
}

void or_contrast(const double* lam, int64_t n, double t_active, double t_quiet, double* out) {
    for (int64_t k = 0; k < n; k++) out[k] = or_planck_ratio(lam[k], t_active, t_quiet);
}

/* ---------------------------------------------------------------------------------- */
/* Localize / InfoMap (Sect. 2.1, Alg. 5)                                              */
/* ---------------------------------------------------------------------------------- */
/* Unit vector of a region centre in the observer frame at rotational phase p. */
static void or_region_centre(double lat_deg, double lon_deg, double incl_deg, double alpha,
                             double phase, double* P) {
    double lat = lat_deg * (OR_PI / 180.0);
    double sl = sin(lat);
    double lon_deg_p = lon_deg + 360.0 * phase * (1.0 + alpha * sl * sl);
    double lon = lon_deg_p * (OR_PI / 180.0);
    double incl = incl_deg * (OR_PI / 180.0);
    /* star frame (rotation axis = y'): (cos lat sin lon, sin lat, cos lat cos lon) */
    double px = cos(lat) * sin(lon), py = sl, pz = cos(lat) * cos(lon);
    /* tilt the axis to (0, sin i, cos i) */
    P[0] = px;
    P[1] = py * sin(incl) - pz * cos(incl);
    P[2] = py * cos(incl) + pz * sin(incl);
}

/* InfoMap for one phase: owner[c] = index of the last region (list order) whose cap contains
 * visible cell c, or -1. */
static void or_infomap(const or_disk* d, int n_regions, const double* lat, const double* lon,
                       const double* radius, double incl_deg, double alpha, double phase,
                       int32_t* owner) {
    double P[64][3];
    double cosr[64];
    for (int r = 0; r < n_regions; r++) {
        or_region_centre(lat[r], lon[r], incl_deg, alpha, phase, P[r]);
        cosr[r] = sqrt(1.0 - radius[r] * radius[r]);
    }
    for (int64_t c = 0; c < d->n; c++) {
        int32_t o = -1;
        for (int r = 0; r < n_regions; r++) {
            double dot = d->x[c] * P[r][0] + d->y[c] * P[r][1] + d->mu[c] * P[r][2];
            if (dot >= cosr[r]) o = r;
        }
        owner[c] = o;
    }
}

/* InfoMap on the full N x N grid (index j*N+i): region index or -1; invisible cells -2. */
int or_infomap_grid(int N, double incl_deg, double alpha, int n_regions, const double* lat,
                    const double* lon, const double* radius, double phase, int32_t* out) {
    if (n_regions > 64) return -1;
    or_disk d;
    double mu1[1] = {1.0};
    or_disk_build(&d, N, 0.0, incl_deg, 0.0, 0.0, alpha, 1, mu1);
    int32_t* own = (int32_t*)malloc(sizeof(int32_t) * (d.n ? d.n : 1));
    or_infomap(&d, n_regions, lat, lon, radius, incl_deg, alpha, phase, own);
    for (int64_t k = 0; k < (int64_t)N * N; k++) out[k] = -2;
    for (int64_t c = 0; c < d.n; c++) out[d.idx[c]] = own[c];
    free(own);
    or_disk_free(&d);
    return 0;
}

/* ---------------------------------------------------------------------------------- */
/* Alg. 5 with Eqs. 1-4: spectra of the active star per phase                          */
/* ---------------------------------------------------------------------------------- */
/* effects bit mask: 1 = total (Eq. 3), 2 = flux (Eq. 1), 4 = convective blueshift (Eq. 2).
 * active: [2][n_mu][n_px], row 0 = spot spectra, row 1 = facula spectra.
 * region arrays: type (1 spot, 2 facula), lat, lon (deg), radius (R*), temperature (K).
 * out_F  : [n_eff][n_phases][n_sample]  S_final = S_quiet - Delta S   (Eq. 4)
 * out_dF : [n_eff][n_phases][n_sample]  Delta S (may be NULL)
 * effects appear in the output in the order total, flux, bconv (those requested). */
int or_active(int N, double vsini, double incl_deg, double u1, double u2, double alpha,
              int n_mu, const double* mu_values, double lambda_start, double lambda_end,
              int64_t n_px, double t_quiet, const double* quiet, const double* active,
              int n_regions, const int32_t* rtype, const double* lat, const double* lon,
              const double* radius, const double* temp, int n_phases, const double* phases,
              uint32_t effects, const int64_t* pix, int64_t n_sample, double* out_F,
              double* out_dF, int facula_mu) {
    if (n_regions > 64 || n_regions < 0 || n_mu > 64) return -1;
    double* lam = (double*)malloc(sizeof(double) * n_px);
    or_grid(lambda_start, lambda_end, n_px, lam);
    double delta = or_delta(lambda_start, lambda_end, n_px);
    or_disk d;
    or_disk_build(&d, N, vsini, incl_deg, u1, u2, alpha, n_mu, mu_values);
    int32_t* owner = (int32_t*)malloc(sizeof(int32_t) * (size_t)n_phases * (d.n ? d.n : 1));
    #pragma omp parallel for schedule(dynamic, 1)
    for (int p = 0; p < n_phases; p++)
        or_infomap(&d, n_regions, lat, lon, radius, incl_deg, alpha, phases[p], owner + (int64_t)p * d.n);
    int eff_list[3], n_eff = 0;
    if (effects & 1u) eff_list[n_eff++] = 1;
    if (effects & 2u) eff_list[n_eff++] = 2;
    if (effects & 4u) eff_list[n_eff++] = 4;

    #pragma omp parallel for schedule(dynamic, 1)
    for (int64_t s = 0; s < n_sample; s++) {
        int64_t m = or_pix(pix, s);
        /* quiet integral at this pixel (Alg. 1) */
        or_sum fq = {0.0, 0.0};
        for (int64_t c = 0; c < d.n; c++) {
            const double* S = quiet + (int64_t)d.bin[c] * n_px;
            or_add(&fq, d.I[c] * or_shift_interp(lam, S, n_px, delta, d.beta[c], m));
        }
        double Fq = or_val(&fq);
        double C[64];
        for (int r = 0; r < n_regions; r++) C[r] = or_planck_ratio(lam[m], temp[r], t_quiet);
        /* facula limb brightening (Sect. 4.3.1, SOAP 2.0's model): a facula cell of mu bin b has
         * the temperature T_quiet + dT_f(mu_b), dT_f(mu) = 250.9 - 407.7 mu + 190.9 mu^2 */
        double Cf[64];
        if (facula_mu)
            for (int b = 0; b < n_mu; b++) {
                double mu = mu_values[b];
                Cf[b] = or_planck_ratio(lam[m], t_quiet + (250.9 - 407.7 * mu + 190.9 * mu * mu), t_quiet);
            }
        for (int p = 0; p < n_phases; p++) {
            const int32_t* own = owner + (int64_t)p * d.n;
            or_sum dtot = {0, 0}, dflux = {0, 0}, dbconv = {0, 0};
            for (int64_t c = 0; c < d.n; c++) {
                int32_t r = own[c];
                if (r < 0) continue;
                const double* Sq = quiet + (int64_t)d.bin[c] * n_px;
                const double* Sa = active + ((int64_t)(rtype[r] == 2 ? 1 : 0) * n_mu + d.bin[c]) * n_px;
                double sq = or_shift_interp(lam, Sq, n_px, delta, d.beta[c], m);
                double sa = or_shift_interp(lam, Sa, n_px, delta, d.beta[c], m);
                double I = d.I[c];
                double Cc = (facula_mu && rtype[r] == 2) ? Cf[d.bin[c]] : C[r];
                or_add(&dflux, I * (sq - Cc * sq));        /* Eq. 1 */
                or_add(&dbconv, I * (sq - sa));            /* Eq. 2 */
                or_add(&dtot, I * (sq - Cc * sa));         /* Eq. 3 */
            }
            for (int e = 0; e < n_eff; e++) {
                double dF = eff_list[e] == 1 ? or_val(&dtot) : eff_list[e] == 2 ? or_val(&dflux) : or_val(&dbconv);
                int64_t o = ((int64_t)e * n_phases + p) * n_sample + s;
                out_F[o] = Fq - dF;                        /* Eq. 4 */
                if (out_dF) out_dF[o] = dF;
            }
        }
    }
    free(owner);
    or_disk_free(&d);
    free(lam);
    return 0;
}

/* ---------------------------------------------------------------------------------- */
/* CCF with a line mask (Sect. 4.1)                                                     */
/* ---------------------------------------------------------------------------------- */
/* Pixel n covers [n-1/2, n+1/2] in pixel coordinates u = ln(lambda/lambda_s)/Delta (edges at
 * geometric midpoints).  Mask line l at velocity v is a box of full width W (km/s) centred
 * at u_l(v) = (ln(lambda_l/lambda_s) + atanh(v/c)) / Delta, half width W/(2 c Delta).
 * CCF(v) = sum_l w_l sum_n F_n |[n-1/2, n+1/2] intersect box_l(v)|.
 * Lines whose box leaves [-1/2, n_px-1/2] anywhere on the velocity grid are skipped.
 * F: [n_spec][n_px]; out: [n_spec][n_v]. */
int or_ccf(const double* F, int n_spec, int64_t n_px, double lambda_start, double lambda_end,
           const double* mask_lambda, const double* mask_w, int n_lines, double width_kms,
           double v_lo, double v_step, int n_v, double* out) {
    double delta = or_delta(lambda_start, lambda_end, n_px);
    double h = width_kms / (2.0 * OR_C_KMS * delta);
    double v_hi = v_lo + (double)(n_v - 1) * v_step;
    #pragma omp parallel for collapse(2) schedule(static)
    for (int sp = 0; sp < n_spec; sp++)
        for (int k = 0; k < n_v; k++) {
            const double* f = F + (int64_t)sp * n_px;
            double v = v_lo + (double)k * v_step;
            or_sum acc = {0.0, 0.0};
            for (int l = 0; l < n_lines; l++) {
                double u0 = log(mask_lambda[l] / lambda_start);
                double ulo = (u0 + atanh(v_lo / OR_C_KMS)) / delta - h;
                double uhi = (u0 + atanh(v_hi / OR_C_KMS)) / delta + h;
                if (ulo < -0.5 || uhi > (double)n_px - 0.5) continue;
                double uc = (u0 + atanh(v / OR_C_KMS)) / delta;
                /* box edges relative to the pixel below the centre, so that the box keeps its
                 * width W exactly (edges rounded at the magnitude of uc would not) */
                double nc = floor(uc);
                double frac = uc - nc;
                double a = frac - h, b = frac + h;
                int64_t i0 = (int64_t)floor(a + 0.5), i1 = (int64_t)floor(b + 0.5);
                for (int64_t i = i0; i <= i1; i++) {
                    int64_t n = (int64_t)nc + i;
                    if (n < 0 || n >= n_px) continue;
                    double lo = fmax(a, (double)i - 0.5), hi = fmin(b, (double)i + 0.5);
                    if (hi > lo) or_add(&acc, mask_w[l] * f[n] * (hi - lo));
                }
            }
            out[(int64_t)sp * n_v + k] = or_val(&acc);
        }
    return 0;
}

int or_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
