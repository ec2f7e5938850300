/*
 * soap.h -- C-ABI of the GB300 (sm_103a) stellar-disk integration library (libsoap.so).
 *
 * Computes the hot path of SOAP-GPU (Zhao & Dumusque, arXiv 2301.04259): every cell of an
 * N x N stellar-disk grid takes the local spectrum of its centre-to-limb angle mu, Doppler
 * shifts it by the cell's projected rotational velocity (Eq. 6), interpolates it back onto
 * the common wavelength grid (Eqs. 9-11), weights it by limb darkening and sums it over the
 * disk (Alg. 1 / Alg. 4).  Per rotational phase, the cells covered by spots and faculae
 * (InfoMap, Alg. 5) contribute the differences of Eqs. 1-3, and Eq. 4 gives the spectrum of
 * the active star.  Radial velocities come from a line-mask CCF and a Gaussian fit
 * (Sect. 4.1).
 *
 * Conventions shared by every entry point
 *  - Status: every call returns a soap_status.  On anything but SOAP_OK the outputs are
 *    unspecified and soap_last_error() (per thread) describes the failure.  No C++
 *    exception crosses this boundary.
 *  - Ownership: the caller owns every pointer it passes.  The library copies what it keeps
 *    (star parameters, local spectra) into memory owned by the context, never frees caller
 *    memory and never retains caller pointers after a call returns.  The context owns all
 *    device memory it allocates; soap_free() releases it.
 *  - Memory space: pointer arguments documented "host or device" come with an `*_on_device`
 *    flag: 0 = host memory (pageable or pinned), 1 = device memory of the context's GPU.
 *    Everything else is host memory.
 *  - Streams: all GPU work of a context is enqueued on its stream (soap_init_star's
 *    `cuda_stream`, or soap_set_stream(); NULL = the legacy default stream).  Calls whose
 *    outputs are in device memory return without synchronising: the caller orders later
 *    work on the same stream or synchronises.  Calls with host outputs synchronise the
 *    stream before returning, unless the host-transfer pipeline is on
 *    (soap_set_host_async): then copies from and to host memory run on two streams of the
 *    context's own, ordered against the compute stream by events, and results reach the host
 *    only by the next soap_synchronize().
 *  - Threads: a context must not be used by two threads at once.  Different contexts are
 *    independent.
 *  - Layout: arrays are C row-major; spectra are float64 unless stated otherwise.
 *
 * Wavelength grid.  The grid is log-uniform with both ends included:
 *   lambda_n = lambda_start * exp(n * Delta), n = 0 .. n_px-1,
 *   Delta = log1p((lambda_end - lambda_start) / lambda_start) / (n_px - 1).
 * (The paper's Eq. 5 grid is linear; on a log grid a Doppler shift is a uniform translation
 * in pixel space, which makes the interpolation weight the same for every pixel of a cell.)
 */
#ifndef SOAP_H
#define SOAP_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    SOAP_OK = 0,
    SOAP_EINVAL = 1,     /* invalid argument (NULL pointer, size, range, non-finite value) */
    SOAP_ENOMEM = 2,     /* device or host allocation failed */
    SOAP_ECUDA = 3,      /* a CUDA runtime call or kernel launch failed */
    SOAP_ERANGE = 4,     /* a size exceeds a documented limit */
    SOAP_ETIMEOUT = 5,   /* a bounded device-side wait gave up */
    SOAP_ESTATE = 6      /* call not valid in the context's state (e.g. no active spectrum) */
} soap_status;

/* Arithmetic of the disk sum.  SOAP_FP64: FP64 everywhere (outputs float64).
 * SOAP_FP32: FP64 cell velocities, shifts and weights; FP32 contraction with FP32
 * accumulation (outputs float32).
 * SOAP_BF16X3 (active-phase calls only: soap_active_phases(_radii), soap_active_rv): as
 * SOAP_FP32, but the contraction of Eqs. 1-4 runs on the tensor cores as a GEMM (pixels x
 * phases x (class, mu bin, tap)) with both operands split into BF16 high and low parts and three
 * products accumulated in FP32 (outputs float32); in soap_active_rv the CCF runs the same way
 * (as soap_rv_ccf with spectra_f32 = 2). */
typedef enum {
    SOAP_FP64 = 0,
    SOAP_FP32 = 1,
    SOAP_BF16X3 = 2
} soap_precision;

/* Form of the sum over cells (soap_quiet_spectrum). */
typedef enum {
    SOAP_FORM_TOEPLITZ = 0,   /* per-mu integer-offset velocity kernels, banded contraction */
    SOAP_FORM_DIRECT = 1      /* per-cell gather-interpolate-reduce */
} soap_form;

/* Effects (Eqs. 1-3), OR-able.  Outputs list the requested effects in this order. */
enum {
    SOAP_EFFECT_TOT = 1,      /* Eq. 3: S'_quiet - I_ratio S'_active */
    SOAP_EFFECT_FLUX = 2,     /* Eq. 1: S'_quiet - I_ratio S'_quiet */
    SOAP_EFFECT_BCONV = 4     /* Eq. 2: S'_quiet - S'_active */
};

/* Region types (InfoMap values, Sect. 3.3). */
enum { SOAP_SPOT = 1, SOAP_FACULA = 2 };

/* Limits. */
#define SOAP_MAX_REGIONS 64         /* regions per soap_active_phases call */
#define SOAP_MAX_CLASSES 8          /* distinct (type, temperature) pairs per call */
#define SOAP_MAX_MU 64              /* tabulated mu values */
#define SOAP_MAX_TAPS 256           /* velocity-kernel taps, 2 ceil(s_max) + 2 */

/* Star (Sect. 2.1, Fig. 0; differential rotation Sect. 3.4).
 *  grid_n        N of the N x N disk grid, 1 .. 8192.  Cell (i, j) has centre
 *                x = (2i+1-N)/N, y = (2j+1-N)/N, area (2/N)^2, is visible iff x^2+y^2 < 1,
 *                mu = sqrt(1 - x^2 - y^2).
 *  n_mu          number of tabulated mu values (local spectra), 1 .. SOAP_MAX_MU.
 *  n_px          pixels of the wavelength grid, 2 .. 2^28.
 *  vsini_kms     projected equatorial velocity, |vsini| < c.  Observer on +z, rotation axis
 *                (0, sin i, cos i); cells with x > 0 recede (positive velocity = redshift).
 *  incl_deg      inclination of the rotation axis to the line of sight (0 .. 180).
 *  u1, u2        quadratic limb darkening I(mu) = 1 - u1 (1-mu) - u2 (1-mu)^2; cell weight
 *                I = area * I(mu).
 *  diff_rot_alpha  omega(lat) = omega0 (1 + alpha sin^2 lat) (alpha = omega1/omega0, the
 *                paper's DIFF_ROT); projected velocity vsini x (1 + alpha sin^2 lat).
 *  lambda_start_A, lambda_end_A  grid ends (vacuum Angstrom), 0 < start < end.
 *  t_quiet_K     effective temperature of the quiet photosphere (contrast, Sect. 4.3.1).
 *  mu_values     host array [n_mu] in (0, 1]; each cell uses the nearest value (ties: lower
 *                index). */
typedef struct {
    int32_t grid_n;
    int32_t n_mu;
    int64_t n_px;
    double vsini_kms;
    double incl_deg;
    double u1;
    double u2;
    double diff_rot_alpha;
    double lambda_start_A;
    double lambda_end_A;
    double t_quiet_K;
    const double* mu_values;
} soap_star_desc;

/* One active region (Sect. 2.1 Localize; Alg. 5): a spherical cap of angular radius
 * asin(radius_rstar) centred at (lat_deg, lon_deg).  At rotational phase p its longitude is
 * lon_deg + 360 p (1 + alpha sin^2 lat); longitude 0 at phase 0 faces the observer.  Regions
 * later in the list overwrite earlier ones in the InfoMap (a spot listed after a facula
 * inside it keeps its own type).  The contrast is the Planck ratio
 * B(lambda, temp_K) / B(lambda, t_quiet_K) (Sect. 4.3.1).  radius_rstar in [0, 1]. */
typedef struct {
    int32_t type;          /* SOAP_SPOT or SOAP_FACULA */
    int32_t reserved;      /* must be 0 */
    double lat_deg;
    double lon_deg;
    double radius_rstar;
    double temp_K;
} soap_region;

/* Kernel timers (soap_set_profiling / soap_get_kernel_time). */
typedef enum {
    SOAP_TIMER_GEOMETRY = 0,     /* per-cell geometry + quiet velocity kernels (batched form: per-column
                                    tables and quiet kernels of every configuration) */
    SOAP_TIMER_PAD_ROWS = 1,     /* local spectra -> replicate-padded rows */
    SOAP_TIMER_CONTRAST = 2,     /* Planck contrast per region class */
    SOAP_TIMER_PHASE_HIST = 3,   /* InfoMap + per-phase velocity kernels */
    SOAP_TIMER_REGIONS = 4,      /* region centres and cell boxes per (phase, region) */
    SOAP_TIMER_CONTRACT = 5,     /* Toeplitz contraction, active phases */
    SOAP_TIMER_CONTRACT_QUIET = 6, /* Toeplitz contraction, quiet star */
    SOAP_TIMER_DIRECT = 7,       /* direct-form disk sum (+ split reduction) */
    SOAP_TIMER_CCF = 8,          /* CCF partial sums (the main CCF kernel) */
    SOAP_TIMER_FIT = 9,          /* Gaussian fits */
    SOAP_TIMER_CCF_AUX = 10,     /* CCF line / velocity tables (when rebuilt) + partial-sum reduction */
    SOAP_TIMER_LSF = 11,         /* instrumental line-spread function */
    SOAP_TIMER_BISECTORS = 12,   /* bisector injection (soap_inject_bisectors, kernel only) */
    SOAP_TIMER_COUNT = 13
} soap_timer;

/* Read-only facts about an initialised star. */
typedef struct {
    int64_t n_visible;      /* visible cells */
    int32_t tap_min;        /* smallest velocity-kernel tap offset (pixels) */
    int32_t n_taps;         /* taps of every velocity kernel */
    double delta;           /* ln-lambda step of the grid */
    double total_intensity; /* sum of the cell weights I */
    int32_t fixed_point_bits; /* kernels are accumulated exactly as integers in units of 2^-bits */
    int32_t reserved;
} soap_star_info;

typedef struct soap_ctx soap_ctx;

/* Create a context for one star and upload its quiet local spectra.
 *  star            star description (host).
 *  quiet_local     [n_mu][n_px] float64 quiet-photosphere local spectra, host or device.
 *  quiet_on_device 0 host, 1 device.
 *  cuda_stream     cudaStream_t to enqueue on (NULL = legacy default stream).
 *  out             receives the new context; NULL on failure.
 * Computes the per-cell geometry on the GPU (Sect. 2.1): mu, I, velocity, nearest-mu bin,
 * pixel shift s = atanh(v/c)/Delta, tap j = ceil(s) and interpolation weight
 * w = expm1((j - s) Delta) / expm1(Delta) (Eq. 11 on a log grid).  Uses the current CUDA
 * device.  Errors: SOAP_EINVAL for an invalid description, SOAP_ERANGE when a limit above is
 * exceeded, SOAP_ENOMEM, SOAP_ECUDA. */
soap_status soap_init_star(const soap_star_desc* star, const double* quiet_local,
                           int quiet_on_device, void* cuda_stream, soap_ctx** out);

/* Recompute the disk geometry of an existing context for new stellar parameters (vsini,
 * inclination, limb darkening, differential rotation, t_quiet, mu values).  grid_n, n_mu, n_px
 * and the wavelength range must equal those of soap_init_star; the new velocity kernels must
 * fit the padding chosen then (SOAP_ERANGE otherwise: create a new context).  Local spectra are
 * kept (their nearest-mu assignment follows the new mu values). */
soap_status soap_update_star(soap_ctx* ctx, const soap_star_desc* star);

/* Replace the quiet local spectra ([n_mu][n_px] float64, host or device). */
soap_status soap_set_quiet_spectrum(soap_ctx* ctx, const double* quiet_local, int on_device);

/* The same from float32 local spectra ([n_mu][n_px] float32, host or device), for callers of
 * the SOAP_FP32 path only: the SOAP_FP32 results are those of float64 spectra rounded to
 * float32 (which that path reads anyway), at half the upload.  Until float64 spectra are set
 * again, SOAP_FP64 calls fail with SOAP_ESTATE. */
soap_status soap_set_quiet_spectrum_f32(soap_ctx* ctx, const float* quiet_local, int on_device);

/* Upload the active-region local spectra of one region type (Sect. 2.1: S_active).
 *  type          SOAP_SPOT or SOAP_FACULA.  Until a facula spectrum is set, faculae use the
 *                spot spectrum (as SOAP 2.0 did).
 *  active_local  [n_mu][n_px] float64, host or device. */
soap_status soap_set_active_spectrum(soap_ctx* ctx, int32_t type, const double* active_local,
                                     int on_device);

/* The same from float32 active local spectra (see soap_set_quiet_spectrum_f32). */
soap_status soap_set_active_spectrum_f32(soap_ctx* ctx, int32_t type, const float* active_local,
                                         int on_device);

/* Replace the context's stream (cudaStream_t or NULL). */
soap_status soap_set_stream(soap_ctx* ctx, void* cuda_stream);

/* Block until all work of the context's streams (its compute stream and, once used, its two
 * host-transfer streams) has finished; then report any condition the kernels flagged
 * (SOAP_ERANGE) since the last check. */
soap_status soap_synchronize(soap_ctx* ctx);

/* Host-transfer pipeline on (enabled = 1) or off (0; the default).  While it is on:
 *  - soap_set_quiet_spectrum / soap_set_active_spectrum with a host source copy it on the
 *    context's upload stream into a stage of their own (quiet, spot, facula) and return; the
 *    compute stream waits for that copy only, and the next upload to the same stage waits until
 *    the compute stream has read the previous one;
 *  - soap_active_rv with host outputs returns once its work is enqueued; its results are on
 *    the host after the next soap_synchronize().
 * So a caller can enqueue step after step and the uploads of one step, the compute of another
 * and the downloads of a third overlap.  The caller keeps host sources unchanged and host
 * outputs unread until soap_synchronize(); overlap needs pinned host memory (pageable copies
 * are correct but block the host).  Turning it off synchronises all streams. */
soap_status soap_set_host_async(soap_ctx* ctx, int enabled);

/* Fill *out with facts about the star. */
soap_status soap_get_star_info(soap_ctx* ctx, soap_star_info* out);

/* Integrated quiet spectrum (Alg. 1 / Alg. 4): F_q[m] = sum_c I_c S'_c[m].
 *  form       SOAP_FORM_TOEPLITZ or SOAP_FORM_DIRECT (same result up to rounding).
 *  precision  SOAP_FP64 (out: float64 [n_px]) or SOAP_FP32 (out: float32 [n_px]).
 *  out        host or device per out_on_device. */
soap_status soap_quiet_spectrum(soap_ctx* ctx, int32_t form, int32_t precision, void* out,
                                int out_on_device);

/* Spectra of the active star at each phase (Alg. 5 with Eqs. 1-4).
 *  regions    host [n_regions], 0 .. SOAP_MAX_REGIONS, order-significant (see soap_region).
 *  phases     host [n_phases] rotational phases (any real value; 1.0 = one rotation).
 *  effects    OR of SOAP_EFFECT_* (at least one).
 *  precision  SOAP_FP64 (float64 output), SOAP_FP32 or SOAP_BF16X3 (float32 output).
 *  out        [n_effects][n_phases][n_px], effects in the order TOT, FLUX, BCONV (those
 *             requested); out[e][p][m] = F_q[m] - Delta F_e[p][m] (Eq. 4).  Host or device.
 * Errors: SOAP_ESTATE if no active spectrum was set; SOAP_ERANGE if more than
 * SOAP_MAX_CLASSES distinct (type, temperature) pairs are given, or (SOAP_BF16X3) if the
 * row windows of a 128-pixel tile (3 row sets x n_mu bins x (127 + n_taps) values), the
 * contrast of the tile and the decode table need more than 227 KB of shared memory;
 * SOAP_ETIMEOUT if a tensor-core barrier wait gave up (bounded, about a second). */
soap_status soap_active_phases(soap_ctx* ctx, const soap_region* regions, int32_t n_regions,
                               const double* phases, int32_t n_phases, uint32_t effects,
                               int32_t precision, void* out, int out_on_device);

/* Spectra of the active star at each phase and their radial velocities in one call: the
 * spectra of one effect as soap_active_phases computes them (Alg. 5 with Eqs. 1-4), then the
 * CCF and Gaussian fit of soap_rv_ccf on those spectra, which stay in device memory between
 * the two steps.
 *  regions, n_regions, phases, n_phases, precision   as for soap_active_phases.
 *  effect       exactly one of SOAP_EFFECT_TOT, SOAP_EFFECT_FLUX, SOAP_EFFECT_BCONV.
 *  mask_lambda, mask_weight, n_lines, mask_width_kms, v_lo, v_step, n_v   as for soap_rv_ccf.
 *  spectra_out  [n_phases][n_px] float64 (SOAP_FP64) or float32 (SOAP_FP32), or NULL for RVs
 *               only.  Host or device per out_on_device.
 *  rv_kms       [n_phases] fitted line centres (km/s; NaN as in soap_rv_ccf).  Host or device
 *               per out_on_device.
 * With host outputs the results are computed into one of two alternating device buffers of
 * the context; the spectra are copied to the host on the download stream while the CCF runs,
 * the RVs after the fit.  Without the host-transfer pipeline the call returns when both copies
 * are done; with it, see soap_set_host_async.
 * Errors: those of soap_active_phases and soap_rv_ccf; SOAP_EINVAL if effect is not a single
 * SOAP_EFFECT_* bit. */
soap_status soap_active_rv(soap_ctx* ctx, const soap_region* regions, int32_t n_regions,
                           const double* phases, int32_t n_phases, uint32_t effect,
                           int32_t precision, const double* mask_lambda, const double* mask_weight,
                           int32_t n_lines, double mask_width_kms, double v_lo, double v_step,
                           int32_t n_v, void* spectra_out, double* rv_kms, int out_on_device);

/* Instrumental resolution (Sect. 3.3, after Eq. 4): the integrated spectra are degraded to
 * an instrument's resolving power R.  The paper does not give the method; the line-spread
 * function here is a Gaussian of FWHM lambda / R, on the log grid a fixed kernel of 1/(R Delta)
 * pixels FWHM, one tap per pixel (the Gaussian's mass over it) for |k| <= ceil(6 sigma) + 1,
 * renormalised to unit sum; out[m] = sum_k g[k] F[clamp(m - k)] (end values repeat).
 *  resolving_power  R > 0 switches it on for soap_quiet_spectrum, soap_active_phases and
 *                   soap_active_rv (the CCF then sees the degraded spectra); 0 switches it off
 *                   (the default).  SOAP_ERANGE if sigma > 800 pixels or the kernel is wider
 *                   than the grid.
 * The batched form (soap_active_batch) does not apply it. */
soap_status soap_set_instrument_resolution(soap_ctx* ctx, double resolving_power);

/* Bisector injection (Sect. 4.3, the paper's Convec.model): normalised local spectra
 * (continuum 1) get their line bisector replaced, every point moved by the velocity of its
 * normalised depth.  The paper fits solar bisectors (not available); here the bisectors are
 * tables: a point of depth d = clip(1 - F, 0, 1) moves by B_row(d) - B_orig(d) km/s, B given at
 * n_depth equally spaced depths 0..1 and linear in between, i.e. by atanh(v/c)/Delta pixels; the
 * moved points are re-sampled at the pixel centres linearly in wavelength (Eq. 11), the end
 * values repeating outside.
 *  in, out      [n_rows][n_px] float64, distinct, both host or both device per on_device
 *               (typically the n_mu rows of a quiet or active local spectrum set).
 *  bis_table    host [n_rows][n_depth] target bisector of each row (km/s).
 *  orig_table   host [n_depth] the input spectra's own bisector (km/s; zeros when they have none).
 * Errors: SOAP_ERANGE if |B| exceeds 1e-3 c or moves points by more than 62 pixels, or if the
 * moved positions of a row are not increasing (checked on the device; the call synchronises). */
soap_status soap_inject_bisectors(soap_ctx* ctx, const double* in, double* out, int32_t n_rows,
                                  const double* bis_table, const double* orig_table, int32_t n_depth,
                                  int on_device);

/* Apply the context's line-spread function to n_spec spectra [n_spec][n_px] (float64, or
 * float32 with spectra_f32 = 1): in -> out, distinct arrays, both host or both device per
 * on_device.  SOAP_ESTATE if no resolution is set. */
soap_status soap_lower_resolution(soap_ctx* ctx, const void* in, void* out, int32_t spectra_f32,
                                  int32_t n_spec, int on_device);

/* Facula limb brightening (Sect. 4.3.1: the SOAP 2.0 model the paper quotes).  When enabled,
 * a facula cell takes the temperature T_quiet + dT_f(mu_b) of its mu bin, dT_f(mu) =
 * 250.9 - 407.7 mu + 190.9 mu^2 (K), instead of its region's temp_K; the contrast then has one
 * row per (class, mu bin) and the Toeplitz contraction folds each bin's sum with its own row
 * (exact: the contrast multiplies on the common grid, Eqs. 1-3).  Off by default.  Applies to
 * soap_active_phases(_radii) and soap_active_rv; the batched form does not use it. */
soap_status soap_set_facula_limb_brightening(soap_ctx* ctx, int enabled);

/* CCF of the FP32 spectra of soap_active_rv (precision SOAP_FP32) on the tensor cores: when
 * enabled, the CCF of Sect. 4.1 runs as soap_rv_ccf with spectra_f32 = 2 (a tcgen05 GEMM of
 * spectra x velocities over pixels against the line-mask matrix, both split into BF16 high and
 * low parts, three products accumulated in FP32: within 1.7e-4 of the largest CCF value, RVs
 * within 0.05 cm/s of the FP32 CCF's on the 205,800-pixel workload); the contraction and the
 * Gaussian fit are unchanged.  Masks not sorted by wavelength and grids of more than 256
 * velocities keep the FP32 CCF.  Off by default (SOAP_BF16X3 always takes this form). */
soap_status soap_set_ccf_tensor_cores(soap_ctx* ctx, int enabled);

/* Active-region size evolution (Sect. 4.2.1).  The paper names three laws and their
 * parameters; the formulas are readings:
 *  SOAP_EVOLVE_NONE            the region keeps its radius_rstar;
 *  SOAP_EVOLVE_LINEAR_GROWTH   A(t) = A0 + rate max(t, 0);
 *  SOAP_EVOLVE_LINEAR_DECAY    A(t) = max(0, A0 - rate max(t, 0));
 *  SOAP_EVOLVE_ASYM_GAUSSIAN   A(t) = A0 exp(-(t - t_peak)^2 / (2 s^2)) (Murakozy et al. 2014),
 *                              s = s_rise before the peak, s_decay after it, s_rise + s_decay =
 *                              fwhm / sqrt(2 ln 2), (s_decay - s_rise) / (s_decay + s_rise) = asymmetry;
 * A in millionths of the solar hemisphere (MSH), t in days; the radius is sqrt(A 1e-6) stellar
 * radii (10000 MSH = 1% of the visible hemisphere = a disk-centre region of radius 0.1), at
 * most 1. */
enum { SOAP_EVOLVE_NONE = 0, SOAP_EVOLVE_LINEAR_GROWTH = 1, SOAP_EVOLVE_LINEAR_DECAY = 2,
       SOAP_EVOLVE_ASYM_GAUSSIAN = 3 };
typedef struct {
    int32_t law;               /* SOAP_EVOLVE_* */
    int32_t reserved;          /* 0 */
    double area0_msh;          /* A0: initial (linear laws) or peak (Gaussian) area, MSH */
    double rate_msh_per_day;   /* linear laws */
    double t_peak_day;         /* Gaussian */
    double fwhm_day;           /* Gaussian, > 0 */
    double asymmetry;          /* Gaussian, |asymmetry| < 1 */
} soap_region_evolution;

/* Radii [n_times][n_regions] (host) of evolving regions at times_day[n_times] (host): evo[q]
 * governs regions[q] (host arrays of n_regions).  Host arithmetic only. */
soap_status soap_evolve_radii(const soap_region_evolution* evo, const soap_region* regions, int32_t n_regions,
                              const double* times_day, int32_t n_times, double* radii);

/* soap_active_phases with per-phase region radii: radii host [n_phases][n_regions], each in
 * [0, 1] (e.g. from soap_evolve_radii at the phases' times); every other argument as there. */
soap_status soap_active_phases_radii(soap_ctx* ctx, const soap_region* regions, int32_t n_regions,
                                     const double* phases, int32_t n_phases, const double* radii,
                                     uint32_t effects, int32_t precision, void* out, int out_on_device);

/* One configuration of a batch (soap_active_batch): a star of the context's type (same grid,
 * mu table, limb darkening, local spectra and wavelength grid) seen with its own projected
 * velocity and inclination, carrying its own regions at its own phases. */
typedef struct {
    double vsini_kms;      /* |vsini_kms| <= the context star's |vsini| (its velocity kernels' range) */
    double incl_deg;       /* 0 .. 180 */
    int32_t first_region;  /* regions[first_region .. first_region + n_regions), list order as in */
    int32_t n_regions;     /*   soap_active_phases; 0 .. SOAP_MAX_REGIONS */
    int32_t first_phase;   /* phases / output rows [first_phase .. first_phase + n_phases) */
    int32_t n_phases;
} soap_batch_item;

/* Output of soap_active_batch. */
enum {
    SOAP_BATCH_SPECTRUM = 0,   /* F = F_q - Delta F (Eq. 4) */
    SOAP_BATCH_RESIDUAL = 1    /* F - F_q = -Delta F: the active regions' change alone */
};

/* Spectra of many independent active-star configurations in one call: for every item and
 * each of its phases, the TOT effect of soap_active_phases (Alg. 5 with Eqs. 3-4) for a star
 * that differs from the context's only in vsini and inclination.  The paper computes one
 * configuration per run; batching them, and the schedule below, have no counterpart there.
 *  items      host [n_items]; every phase index 0 .. n_phases-1 belongs to exactly one item.
 *  regions    host [n_regions], shared pool that items index into.
 *  phases     host [n_phases] rotational phases.
 *  output     SOAP_BATCH_SPECTRUM or SOAP_BATCH_RESIDUAL (skips the quiet spectra).
 *  out        float32 [n_phases][n_px], row p for phase p, host or device per out_on_device.
 * Arithmetic as SOAP_FP32 (FP64 velocities and shift positions, FP32 contraction and
 * accumulation); a cell's interpolation weight is held to 32 fractional bits; the contrast
 * (Sect. 4.3.1) is evaluated per pixel in FP32.  Needs diff_rot_alpha = 0 (a cell's velocity is
 * then vsini x, so one table per item and grid column replaces per-cell geometry) and at most
 * SOAP_MAX_CLASSES distinct (type, temperature) pairs within each item.  Work is cut into
 * phase blocks run by one persistent kernel in decreasing order of estimated cost; the kernel
 * sequence is captured once per batch shape into a CUDA graph owned by the context and
 * replayed on later calls with the same shape (soap_set_profiling(ctx, 1) runs it without the
 * graph).  The variant (phases per block, pixels per thread) is the one soap_batch_set_variant
 * or soap_batch_autotune chose, else 1 or 2 phases per block when no item has more phases, and
 * 4 otherwise.
 *  rv_kms     [n_phases] radial velocity of each phase's spectrum (Sect. 4.1: CCF with the mask
 *             of soap_batch_set_rv and least-squares Gaussian, as soap_rv_ccf on float32 spectra),
 *             or NULL for spectra only.  Host or device per out_on_device.  Needs
 *             soap_batch_set_rv (SOAP_ESTATE otherwise) and output = SOAP_BATCH_SPECTRUM (the
 *             residual rows are not spectra: SOAP_EINVAL).  The CCF, its reduction and the fits
 *             run inside the same captured graph, on the output rows while they are in device
 *             memory.
 * Errors: SOAP_EINVAL (bad item, phase not covered exactly once, alpha != 0), SOAP_ESTATE (no
 * active spectrum for a region type), SOAP_ERANGE (class limit). */
soap_status soap_active_batch(soap_ctx* ctx, const soap_batch_item* items, int32_t n_items,
                              const soap_region* regions, int32_t n_regions, const double* phases,
                              int32_t n_phases, int32_t output, float* out, double* rv_kms,
                              int out_on_device);

/* Mask and velocity grid of the batched radial velocities (soap_active_batch with rv_kms).
 *  mask_lambda, mask_weight, n_lines, mask_width_kms   as for soap_rv_ccf (host, copied).
 *  v_lo, v_step, n_v   one velocity grid v_k = v_lo + k v_step for every configuration (it must
 *                      cover the widest one); the CCF is computed on all of it.
 *  fit_margin_kms      > 0: configuration q fits its CCF only at the grid velocities with
 *                      |v_k| <= |vsini_q| + fit_margin_kms (at least 5 of them, else SOAP_EINVAL
 *                      at the batch call), the window a single star of that vsini would use;
 *                      <= 0: every configuration fits the whole grid.
 *  tensor_cores        0: the FP32 SIMT CCF; 1: the CCF as a tensor-core GEMM (BF16 hi/lo, as
 *                      soap_rv_ccf with spectra_f32 = 2) where that form applies.
 * Lines whose box leaves the wavelength grid anywhere on the velocity grid are skipped (as in
 * soap_rv_ccf).  Errors: SOAP_EINVAL (as soap_rv_ccf's checks), SOAP_ERANGE (box wider than 14
 * pixels). */
soap_status soap_batch_set_rv(soap_ctx* ctx, const double* mask_lambda, const double* mask_weight,
                              int32_t n_lines, double mask_width_kms, double v_lo, double v_step,
                              int32_t n_v, double fit_margin_kms, int32_t tensor_cores);

/* Number of variants of the batched form (valid variants are 0 .. *n - 1). */
soap_status soap_batch_num_variants(int32_t* n);

/* Phases per block and pixels per thread of a variant; SOAP_ERANGE outside 0 .. n-1. */
soap_status soap_batch_variant_info(int32_t variant, int32_t* phases_per_block,
                                    int32_t* px_per_thread);

/* Variant soap_active_batch uses on this context (-1: chosen from the items' phase counts). */
soap_status soap_batch_set_variant(soap_ctx* ctx, int32_t variant);
soap_status soap_batch_get_variant(const soap_ctx* ctx, int32_t* variant);

/* Time every variant on the given batch (one untimed run, then `reps` runs timed with CUDA
 * events on the context's stream), set the fastest on the context and return it.
 *  out        device float32 [n_phases][n_px] (scratch; holds the last run's result).
 *  ms         host [n_variants] mean milliseconds per run, or NULL.
 * Synchronises the context's stream. */
soap_status soap_batch_autotune(soap_ctx* ctx, const soap_batch_item* items, int32_t n_items,
                                const soap_region* regions, int32_t n_regions, const double* phases,
                                int32_t n_phases, float* out, int32_t reps, float* ms,
                                int32_t* best_variant);

/* Radial velocities from a line-mask CCF and a Gaussian fit (Sect. 4.1).
 *  spectra        [n_spec][n_px] on the context's grid, float64 (spectra_f32 = 0) or float32
 *                 (spectra_f32 = 1, or 2: float32 with the CCF sum as a tensor-core GEMM over
 *                 pixels, both operands split into BF16 hi + lo, three products, FP32
 *                 accumulation; where that form does not apply -- a mask not sorted by
 *                 wavelength or more than 256 velocities -- 2 computes as 1); host or device
 *                 per spectra_on_device.  Other values: SOAP_EINVAL.
 *  mask_lambda    host [n_lines] rest wavelengths (Angstrom); mask_weight host [n_lines].
 *  mask_width_kms full width W of each mask box in velocity.
 *  v_lo, v_step, n_v  velocity grid v_k = v_lo + k v_step (km/s), n_v >= 5.
 * CCF(v) = sum_l w_l sum_n F_n |[n-1/2, n+1/2] intersect box_l(v)| in pixel coordinates
 * u = ln(lambda/lambda_start)/Delta, box_l(v) centred at (ln(lambda_l/lambda_start) +
 * atanh(v/c))/Delta with half width W/(2 c Delta); lines whose box leaves the grid anywhere on
 * the velocity grid are skipped.  The fit minimises sum_k (A + B exp(-(v_k-mu)^2/(2 s^2)) -
 * CCF_k)^2 (in variables scaled by max CCF and by the starting width) from A = max CCF,
 * B = min - max, mu = velocity of the (first) CCF minimum and s = dip area / (|B| sqrt(2 pi)),
 * at least one velocity step: Levenberg-Marquardt in FP32 until its step is below 1e-4, then
 * Newton steps on the exact Hessian.  Float64 spectra: the Newton steps take FP64 residuals and
 * gradient, so that the result is the least-squares minimum to FP64 rounding.  Float32 spectra
 * (whose CCF carries FP32 rounding already): FP32 throughout, a block of four warps per spectrum
 * for at most 304 spectra and one warp per spectrum beyond, which places the centre within ~1e-8
 * of the Gaussian's width of that minimum.
 *  rv_kms         [n_spec] fitted mu (km/s); NaN when the fit leaves the velocity grid (mu
 *                 outside it or a width larger than it: no dip to fit).
 *  fit_params     [n_spec][4] (A, B, mu, s), or NULL.
 *  ccf_out        [n_spec][n_v] float64 CCF, or NULL.
 *  Outputs are host or device per out_on_device.
 * Errors: SOAP_EINVAL (arguments), SOAP_ETIMEOUT if a tensor-core barrier wait gave up (the CCF
 * is then incomplete): with host outputs this call reports it, with device outputs the next
 * soap_synchronize() does. */
soap_status soap_rv_ccf(soap_ctx* ctx, const void* spectra, int32_t spectra_f32, int32_t n_spec,
                        int spectra_on_device, const double* mask_lambda,
                        const double* mask_weight, int32_t n_lines, double mask_width_kms,
                        double v_lo, double v_step, int32_t n_v, double* rv_kms,
                        double* fit_params, double* ccf_out, int out_on_device);

/* Enable (1) or disable (0) per-kernel timing: while enabled, the main kernels of every call
 * are bracketed by CUDA events on the context's stream. */
soap_status soap_set_profiling(soap_ctx* ctx, int enabled);

/* Total device time (ms) and number of timed launches of one timer since the last reset.
 * Synchronises the context's stream.  timer: a soap_timer value. */
soap_status soap_get_kernel_time(soap_ctx* ctx, int32_t timer, double* total_ms, uint64_t* launches);

/* Zero all timers. */
soap_status soap_reset_kernel_times(soap_ctx* ctx);

/* Allocation-free CCF + RV fit, without a context.  The paper has no counterpart: this entry
 * point exists for callers that may not allocate device memory once running (an application
 * that gives the whole GPU to its own memory pool at start-up, a real-time pipeline where an
 * allocation -- which can synchronise the device -- is not allowed after initialisation, or a
 * plug-in that only receives buffers from its host).  It computes what soap_rv_ccf computes
 * (same CCF definition, same fit) on caller buffers only and calls no cudaMalloc, cudaFree or
 * other allocating routine.
 *  Grid: lambda_start_A, lambda_end_A, n_px as in soap_star_desc.
 *  spectra      DEVICE [n_spec][n_px], float64 (spectra_f32 = 0) or float32 (1).
 *  mask_lambda, mask_weight  DEVICE [n_lines] (any order).
 *  rv_kms       DEVICE [n_spec]; fit_params DEVICE [n_spec][4] or NULL; ccf_out DEVICE
 *               [n_spec][n_v] or NULL.
 *  cuda_stream  stream to enqueue on (NULL = legacy default stream); returns without
 *               synchronising.
 * Scratch: one fixed 16 MiB device array inside the library, which every GPU that loads the
 * library keeps until the process exits.  A call needs
 *   24 n_lines + 16 n_v + 8 n_spec n_v (ceil(n_lines / 128) + 2) bytes (plus alignment);
 * larger requests are rejected with SOAP_ERANGE and a message giving both sizes.  The first
 * call on each device looks up the array's device address (cudaGetSymbolAddress); make that
 * first call before any stream capture.  All calls share the one array and it keeps the last
 * call's contents (every element a call reads is written earlier in that call): calls whose
 * GPU work can overlap -- on different streams, or from different threads -- race on it and
 * must be serialised by the caller. */
soap_status soap_rv_ccf_static(double lambda_start_A, double lambda_end_A, int64_t n_px,
                               const void* spectra, int32_t spectra_f32, int32_t n_spec,
                               const double* mask_lambda, const double* mask_weight,
                               int32_t n_lines, double mask_width_kms, double v_lo, double v_step,
                               int32_t n_v, double* rv_kms, double* fit_params, double* ccf_out,
                               void* cuda_stream);

/* Dense BF16 GEMM on the tensor cores (tcgen05, FP32 accumulation), the building block of the
 * surrogate network: C[m][n] = act(sum_k A[m][k] B[n][k] + bias[n]).  No counterpart in the
 * paper.
 *  A          device BF16 [M][lda], B device BF16 [N][ldb] (K contiguous in both); bases 16-byte
 *             aligned, lda and ldb multiples of 8 elements, >= K.
 *  bias       device float [N] or NULL.  activation: 0 none, 1 GELU (exact, erf form).
 *  C          device float [M][ldc], ldc >= N.
 * Synchronises the stream; SOAP_ETIMEOUT if a bounded device-side wait gave up. */
soap_status soap_gemm_bf16_tn(int32_t M, int32_t N, int32_t K, const void* A, int64_t lda,
                              const void* B, int64_t ldb, const float* bias, int32_t activation,
                              float* C, int64_t ldc, void* cuda_stream);

/* ---------------------------------------------------------------------------------------
 * Learned surrogate (no counterpart in the paper).  A network maps 8 active-region parameters
 *   x = (spot latitude deg, spot longitude deg, spot radius R*, spot temperature K, phase,
 *        inclination deg, vsini km/s, facula filling)
 * to 128 PCA coefficients of the residual spectrum F - F_q (soap_active_batch with
 * SOAP_BATCH_RESIDUAL) and to log10 of its own RV error in cm/s.  Inputs are scaled linearly to
 * [-1, 1] from the ranges given at creation; a query outside them, or with a predicted error
 * above the caller's threshold, is not accepted and belongs to the plain method.
 * Network: 8 -> 4 x 256 (GELU, erf form) -> 129; BF16 weights and activations as tensor-core
 * operands with FP32 accumulation; FP32 master weights; Adam (beta 0.9, 0.999, eps 1e-8).
 * Flat parameter order: W1 [256][8], b1, W2 [256][256], b2, W3, b3, W4, b4, W5 [129][256], b5;
 * output 128 of the last layer is the RV-error head.
 * ------------------------------------------------------------------------------------- */
typedef struct soap_surrogate soap_surrogate;

typedef struct {
    int32_t n_in;          /* 8 */
    int32_t hidden;        /* 256 */
    int32_t n_hidden;      /* 4 */
    int32_t n_coef;        /* 128 */
    int32_t batch;         /* training rows per step, a positive multiple of 128 */
    const float* in_lo;    /* host [n_in] lower ends of the input ranges */
    const float* in_hi;    /* host [n_in] upper ends */
} soap_surrogate_desc;

soap_status soap_surrogate_create(const soap_surrogate_desc* desc, void* cuda_stream, soap_surrogate** out);
soap_status soap_surrogate_num_params(const soap_surrogate* s, int64_t* n);
/* Host float32 [n_params] in the flat order above; set_params also clears the Adam state. */
soap_status soap_surrogate_set_params(soap_surrogate* s, const float* flat);
soap_status soap_surrogate_get_params(soap_surrogate* s, float* flat);
/* Targets are standardised coefficients: c = y * coef_std + coef_mean (host [n_coef] each). */
soap_status soap_surrogate_set_scaling(soap_surrogate* s, const float* coef_mean, const float* coef_std);
/* Loss and gradients of one batch (n = batch rows; x device [n][8] raw inputs, t device [n][129]
 * targets: standardised coefficients and log10 RV error), L = sum_b sum_j w_j (y - t)^2 / n with
 * w_out host [129].  loss host, grads host [n_params].  For checking the backward pass. */
soap_status soap_surrogate_gradients(soap_surrogate* s, const float* x, const float* t, int32_t n,
                                     const float* w_out, double* loss, float* grads);
/* Adam over `epochs` passes of shuffled full batches of (x, t) (device, as above; rows beyond
 * the last full batch of an epoch are skipped).  lr_per_epoch host [epochs]; stage 0 trains
 * everything except the RV-error head, stage 1 only the head, stage 2 everything.
 * loss_per_epoch host [epochs] or NULL.  One training step is a CUDA graph replayed per batch. */
soap_status soap_surrogate_train(soap_surrogate* s, const float* x, const float* t, int64_t n, int32_t epochs,
                                 const float* lr_per_epoch, const float* w_out, int32_t stage, uint64_t seed,
                                 double* loss_per_epoch);
/* Network outputs for n queries x (device [n][8]): coefficients in data units (device [n][128]
 * or NULL), predicted RV error in cm/s (device [n] or NULL) and acceptance (device uint8 [n] or
 * NULL: 1 if every input is inside its range and the predicted error <= rv_err_max_cms). */
soap_status soap_surrogate_predict(soap_surrogate* s, const float* x, int64_t n, float rv_err_max_cms,
                                   float* coef, float* pred_err_cms, uint8_t* accepted);
/* Take the predicted RV error from output n_coef of another network of the same shape and
 * input ranges (trained with stage 2 on the plain-method errors), instead of this network's own head;
 * NULL restores the own head.  The error network must outlive its use. */
soap_status soap_surrogate_set_error_net(soap_surrogate* s, soap_surrogate* error_net);
/* PCA basis of the residuals: mean device [n_px], basis device [n_coef][n_px] (orthonormal rows). */
soap_status soap_surrogate_set_basis(soap_surrogate* s, const float* mean, const float* basis, int64_t n_px);
/* Residual spectra mean + coef . basis for device coef [n][128] into device out [n][n_px]; both
 * factors split into BF16 high and low parts on the tensor cores (error ~1e-5 of |coef| |basis|). */
soap_status soap_surrogate_reconstruct(soap_surrogate* s, const float* coef, int64_t n, float* out);
/* predict + reconstruct: out device [n][n_px] residual spectra for every query (accepted or
 * not), accepted device uint8 [n] (required), pred_err_cms device [n] or NULL.  The caller
 * replaces the rows that were not accepted with the plain method's. */
soap_status soap_surrogate_query(soap_surrogate* s, const float* x, int64_t n, float rv_err_max_cms, float* out,
                                 float* pred_err_cms, uint8_t* accepted);
void soap_surrogate_free(soap_surrogate* s);

/* Network inputs of n surrogate queries (device float32 [n][8] -> device float32 [n][8],
 * asynchronous on the stream).  Query parameters: latitude (deg), longitude (deg), radius (R*),
 * spot temperature (K), phase, inclination (deg), vsini (km/s), facula filling.  Inputs: the
 * region's centre at that phase in the observer frame of the disk integration (Sect. 2.1 and
 * Alg. 5: star-frame (cos lat sin L, sin lat, cos lat cos L), L = lon + 360 phase, tilted so that
 * the rotation axis is (0, sin i, cos i); x across the disk, y up, z toward the observer, rigid
 * rotation) as (y, x, radius, temperature, z, vsini * x, vsini, filling): the spectrum depends on
 * latitude, longitude, phase and inclination only through that point.  FP32 (sincosf). */
soap_status soap_surrogate_encode(const float* params, int64_t n, float* x, void* cuda_stream);

/* y[i] += alpha x[i] for device float arrays of n elements (asynchronous on the stream). */
soap_status soap_axpy_f32(int64_t n, float alpha, const float* x, float* y, void* cuda_stream);

/* PCA by randomized SVD with n_power power iterations (Halko, Martinsson & Tropp 2011):
 * X device [n][p] float32 rows, omega device [p][l] a Gaussian test matrix (the caller draws it),
 * k <= l <= 512 components kept.  mean device [p], basis device [k][p] (orthonormal rows, in
 * decreasing singular value), sv host [k] singular values of the centred data or NULL.
 * Synchronises the stream. */
soap_status soap_pca_fit(const float* X, int64_t n, int64_t p, const float* omega, int32_t l, int32_t k,
                         int32_t n_power, float* mean, float* basis, double* sv, void* cuda_stream);
/* coef device [n][k] = (X - mean) basis^T. */
soap_status soap_pca_project(const float* X, int64_t n, int64_t p, const float* mean, const float* basis,
                             int32_t k, float* coef, void* cuda_stream);

/* Number of kernels this context has launched so far (for launch accounting). */
soap_status soap_get_launch_count(const soap_ctx* ctx, uint64_t* out);

/* For testing error reporting only: mark the context's device status word (stream-ordered) as a
 * tensor-core kernel does when one of its bounded barrier waits gives up.  The next call that
 * reads the status word (a call with host outputs, or soap_synchronize) then returns
 * SOAP_ETIMEOUT and clears it.  No kernel is made to wait or fail. */
soap_status soap_debug_inject_timeout(soap_ctx* ctx);

/* Release the context and all device memory it owns.  NULL is a no-op.  Synchronises the
 * context's stream first. */
void soap_free(soap_ctx* ctx);

/* Description of the last failure on the calling thread ("" if none).  The string stays
 * valid until the next call on this thread. */
const char* soap_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* SOAP_H */
