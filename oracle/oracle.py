"""Python face of the FP64 CPU oracle (soap_oracle.c) plus the Gaussian RV fit.

TEST INFRASTRUCTURE.  Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg
of ``bench.py`` may import this module.  It shares no code with the CUDA library and never
calls it.

Functions follow the paper (arXiv 2301.04259):
  quiet(...)       Alg. 1 (Sect. 2.1): sum over disk cells of I_XY x Doppler-shifted,
                   re-interpolated local spectrum (Eqs. 6, 9-11).
  active(...)      Alg. 5 (Sect. 3.3) with Eqs. 1-4 (Sect. 2.1).
  contrast(...)    Sect. 4.3.1: ratio of two Planck functions.
  ccf(...)         Sect. 4.1: cross-correlation with a line mask.
  fit_gaussian(...) Sect. 4.1: RV = mean of a Gaussian fitted to the CCF (least squares,
                   Levenberg-Marquardt from scipy/MINPACK, used as a library step).
  evolution_area(...), evolution_radius(...)  Sect. 4.2.1: active-region size evolution
                   (linear growth, linear decay, asymmetric Gaussian); active(..., radii=) takes
                   per-phase radii.
  inject_bisectors(...) Sect. 4.3 (Convec.model): each point of a normalised local spectrum
                   moved by the velocity of its normalised depth on a target bisector minus the
                   original one, then re-sampled on the grid.
  lower_resolution(...) Sect. 3.3 after Eq. 4 (Alg. 5): the integrated spectra degraded to an
                   instrument's resolving power (Gaussian line-spread function; reading in
                   instrument_kernel).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from pathlib import Path

import numpy as np

HERE = Path(__file__).resolve().parent
SRC = HERE / "soap_oracle.c"
BUILD = HERE / "_build"
LIB = BUILD / "liboracle.so"

C_KMS = 299792.458

_lib = None


def build(force: bool = False) -> Path:
    """Compile the oracle with gcc (IEEE FP64, no contraction, OpenMP)."""
    BUILD.mkdir(exist_ok=True)
    if LIB.exists() and not force and LIB.stat().st_mtime >= SRC.stat().st_mtime:
        return LIB
    tmp = LIB.with_suffix(f".{os.getpid()}.tmp.so")
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
           "-fno-fast-math", str(SRC), "-o", str(tmp), "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, LIB)
    return LIB


def _load():
    global _lib
    if _lib is not None:
        return _lib
    build()
    lib = ctypes.CDLL(str(LIB))
    d, i32, i64, u32 = ctypes.c_double, ctypes.c_int, ctypes.c_int64, ctypes.c_uint32
    P = ctypes.c_void_p
    lib.or_delta.restype = d
    lib.or_delta.argtypes = [d, d, i64]
    lib.or_grid.restype = None
    lib.or_grid.argtypes = [d, d, i64, P]
    lib.or_cell_geometry.restype = None
    lib.or_cell_geometry.argtypes = [i32, d, d, d, d, d, i32, P, P, P, P, P]
    lib.or_shift_interp.restype = d
    lib.or_shift_interp.argtypes = [P, P, i64, d, d, i64]
    lib.or_quiet.restype = i32
    lib.or_quiet.argtypes = [i32, d, d, d, d, d, i32, P, d, d, i64, P, P, i64, P]
    lib.or_planck_ratio.restype = d
    lib.or_planck_ratio.argtypes = [d, d, d]
    lib.or_contrast.restype = None
    lib.or_contrast.argtypes = [P, i64, d, d, P]
    lib.or_infomap_grid.restype = i32
    lib.or_infomap_grid.argtypes = [i32, d, d, i32, P, P, P, d, P]
    lib.or_active.restype = i32
    lib.or_active.argtypes = [i32, d, d, d, d, d, i32, P, d, d, i64, d, P, P,
                              i32, P, P, P, P, P, i32, P, u32, P, i64, P, P, i32]
    lib.or_ccf.restype = i32
    lib.or_ccf.argtypes = [P, i32, i64, d, d, P, P, i32, d, d, d, i32, P]
    lib.or_num_threads.restype = i32
    lib.or_num_threads.argtypes = []
    _lib = lib
    return lib


def _p(a):
    return ctypes.c_void_p(a.ctypes.data) if a is not None else None


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def num_threads() -> int:
    return int(_load().or_num_threads())


# ---------------------------------------------------------------------------------------
def delta(lambda_start, lambda_end, n_px) -> float:
    return float(_load().or_delta(lambda_start, lambda_end, n_px))


def grid(lambda_start, lambda_end, n_px) -> np.ndarray:
    out = np.empty(n_px, np.float64)
    _load().or_grid(lambda_start, lambda_end, n_px, _p(out))
    return out


def cell_geometry(star):
    """(I, v, mu, bin) on the N x N grid, index j*N+i; invisible cells: I=0, bin=-1."""
    N = star.grid_n
    I = np.empty(N * N); v = np.empty(N * N); mu = np.empty(N * N)
    b = np.empty(N * N, np.int32)
    muv = _f64(star.mu_values)
    _load().or_cell_geometry(N, star.vsini_kms, star.incl_deg, star.u1, star.u2,
                             star.diff_rot_alpha, len(muv), _p(muv), _p(I), _p(v), _p(mu), _p(b))
    return I, v, mu, b


def shift_interp(lam, S, beta, m) -> float:
    """S Doppler-shifted by beta and re-interpolated at output pixel m (Eqs. 6, 9-11)."""
    lam = _f64(lam); S = _f64(S)
    dl = float(np.log(lam[-1] / lam[0]) / (lam.size - 1))
    return float(_load().or_shift_interp(_p(lam), _p(S), lam.size, dl, beta, int(m)))


def _pix(pix, n_px):
    if pix is None:
        return None, n_px
    pix = np.ascontiguousarray(pix, dtype=np.int64)
    if pix.size and (pix.min() < 0 or pix.max() >= n_px):
        raise ValueError("pixel index out of range")
    return pix, pix.size


def quiet(star, quiet_local, pix=None) -> np.ndarray:
    """Integrated quiet spectrum (Alg. 1) at pixels `pix` (all pixels if None)."""
    q = _f64(quiet_local)
    assert q.shape == (star.n_mu, star.n_px)
    pix, ns = _pix(pix, star.n_px)
    out = np.empty(ns, np.float64)
    muv = _f64(star.mu_values)
    rc = _load().or_quiet(star.grid_n, star.vsini_kms, star.incl_deg, star.u1, star.u2,
                          star.diff_rot_alpha, star.n_mu, _p(muv), star.lambda_start_A,
                          star.lambda_end_A, star.n_px, _p(q), _p(pix), ns, _p(out))
    if rc != 0:
        raise RuntimeError("or_quiet failed")
    return out


EFFECT_TOT, EFFECT_FLUX, EFFECT_BCONV = 1, 2, 4


def active(star, quiet_local, active_local, regions, phases, effects=EFFECT_TOT, pix=None,
           return_delta=False, radii=None, facula_mu=False):
    """Spectra of the active star per phase (Alg. 5, Eqs. 1-4).

    active_local: dict type -> [n_mu, n_px] (1 spot, 2 facula; facula defaults to spot).
    radii: optional [n_phases, n_regions] region radii per phase (evolving regions); each phase
    is then computed with its own radii.
    facula_mu: facula cells take the temperature T_quiet + dT_f(mu_b) of their mu bin,
    dT_f(mu) = 250.9 - 407.7 mu + 190.9 mu^2 (SOAP 2.0's limb brightening, Sect. 4.3.1), instead
    of their region's temperature.
    Returns F [n_eff, n_phases, n_sample] (and Delta F if return_delta)."""
    if radii is not None:
        import dataclasses
        radii = np.asarray(radii, np.float64)
        parts = []
        for p, ph in enumerate(np.atleast_1d(np.asarray(phases, np.float64))):
            regs = [dataclasses.replace(r, radius_rstar=float(radii[p, q])) for q, r in enumerate(regions)]
            parts.append(active(star, quiet_local, active_local, regs, [ph], effects, pix, return_delta,
                                facula_mu=facula_mu))
        if return_delta:
            return (np.concatenate([a for a, _ in parts], axis=1), np.concatenate([b for _, b in parts], axis=1))
        return np.concatenate(parts, axis=1)
    q = _f64(quiet_local)
    spot = _f64(active_local[1])
    fac = _f64(active_local.get(2, active_local[1]))
    act = np.ascontiguousarray(np.stack([spot, fac]))
    nr = len(regions)
    rtype = np.array([r.type for r in regions], np.int32)
    lat = _f64([r.lat_deg for r in regions]); lon = _f64([r.lon_deg for r in regions])
    rad = _f64([r.radius_rstar for r in regions]); tmp = _f64([r.temp_K for r in regions])
    if nr == 0:
        rtype = np.zeros(1, np.int32); lat = lon = rad = tmp = np.zeros(1)
    ph = _f64(phases)
    pix, ns = _pix(pix, star.n_px)
    n_eff = bin(effects & 7).count("1")
    F = np.empty((n_eff, ph.size, ns)); dF = np.empty_like(F) if return_delta else None
    muv = _f64(star.mu_values)
    rc = _load().or_active(star.grid_n, star.vsini_kms, star.incl_deg, star.u1, star.u2,
                           star.diff_rot_alpha, star.n_mu, _p(muv), star.lambda_start_A,
                           star.lambda_end_A, star.n_px, star.t_quiet_K, _p(q), _p(act), nr,
                           _p(rtype), _p(lat), _p(lon), _p(rad), _p(tmp), ph.size, _p(ph),
                           effects, _p(pix), ns, _p(F), _p(dF), int(bool(facula_mu)))
    if rc != 0:
        raise RuntimeError("or_active failed")
    return (F, dF) if return_delta else F


def infomap(star, regions, phase) -> np.ndarray:
    """InfoMap on the N x N grid [j, i]: owning region index, -1 quiet, -2 off-disk."""
    N = star.grid_n
    out = np.empty(N * N, np.int32)
    lat = _f64([r.lat_deg for r in regions] or [0.0]); lon = _f64([r.lon_deg for r in regions] or [0.0])
    rad = _f64([r.radius_rstar for r in regions] or [0.0])
    rc = _load().or_infomap_grid(N, star.incl_deg, star.diff_rot_alpha, len(regions), _p(lat),
                                 _p(lon), _p(rad), float(phase), _p(out))
    if rc != 0:
        raise RuntimeError("or_infomap_grid failed")
    return out.reshape(N, N)


def planck_ratio(lambda_A, t_active, t_quiet) -> float:
    return float(_load().or_planck_ratio(lambda_A, t_active, t_quiet))


def contrast(lam, t_active, t_quiet) -> np.ndarray:
    lam = _f64(lam)
    out = np.empty_like(lam)
    _load().or_contrast(_p(lam), lam.size, t_active, t_quiet, _p(out))
    return out


def ccf(F, star_or_range, mask_lambda, mask_weight, width_kms, v_lo, v_step, n_v) -> np.ndarray:
    """CCF [n_spec, n_v] of spectra F [n_spec, n_px] with the box mask (Sect. 4.1)."""
    F = _f64(np.atleast_2d(F))
    if hasattr(star_or_range, "lambda_start_A"):
        ls, le = star_or_range.lambda_start_A, star_or_range.lambda_end_A
    else:
        ls, le = star_or_range
    ml = _f64(mask_lambda); mw = _f64(mask_weight)
    out = np.empty((F.shape[0], n_v))
    _load().or_ccf(_p(F), F.shape[0], F.shape[1], ls, le, _p(ml), _p(mw), ml.size, width_kms,
                   v_lo, v_step, n_v, _p(out))
    return out


def gaussian(v, A, B, mu, sigma):
    return A + B * np.exp(-0.5 * ((v - mu) / sigma) ** 2)


def fit_initial(v, c):
    """Starting point of the Gaussian fit: continuum = max, depth at the minimum, width from
    the area of the dip."""
    v = np.asarray(v, np.float64); c = np.asarray(c, np.float64)
    A0 = float(c.max()); k = int(np.argmin(c)); B0 = float(c[k] - A0)
    dv = float(v[1] - v[0]) if v.size > 1 else 1.0
    area = float(np.sum(A0 - c) * dv)
    s0 = area / (abs(B0) * np.sqrt(2 * np.pi)) if B0 != 0 else dv
    return np.array([A0, B0, float(v[k]), max(s0, dv)])


def fit_gaussian(v, c):
    """Least-squares Gaussian A + B exp(-(v-mu)^2 / 2 sigma^2) to one CCF; returns
    (A, B, mu, sigma).  RV = mu (Sect. 4.1)."""
    from scipy.optimize import least_squares
    v = np.asarray(v, np.float64); c = np.asarray(c, np.float64)

    def res(p):
        return gaussian(v, *p) - c

    def jac(p):
        A, B, mu, s = p
        e = np.exp(-0.5 * ((v - mu) / s) ** 2)
        return np.stack([np.ones_like(v), e, B * e * (v - mu) / s ** 2,
                         B * e * (v - mu) ** 2 / s ** 3], axis=1)

    r = least_squares(res, fit_initial(v, c), jac=jac, method="lm", xtol=1e-15, ftol=1e-15,
                      gtol=1e-15, max_nfev=20000)
    p = r.x.copy()
    p[3] = abs(p[3])
    return newton_polish(v, c, p)


def newton_polish(v, c, p, max_iter=20):
    """Newton steps on the exact Hessian of the cost 1/2 sum r^2 from a point near the
    least-squares minimum, so that the result is its stationary point to FP64 rounding.

    MINPACK stops on relative changes of the cost and of the step, which on a CCF that is far
    from a Gaussian (large residuals, slow Gauss-Newton convergence) leaves the centre up to
    ~1e-8 km/s short of the minimum.  H = J^T J + sum_i r_i d2m_i, with, for d = v - mu and
    g = exp(-d^2 / (2 s^2)): d2m/dB dmu = g d/s^2, d2m/dB ds = g d^2/s^3,
    d2m/dmu^2 = B g (d^2/s^4 - 1/s^2), d2m/dmu ds = B g (d^3/s^5 - 2 d/s^3),
    d2m/ds^2 = B g (d^4/s^6 - 3 d^2/s^4).  A step is kept only while H is positive definite,
    the steps shrink and the cost grows by no more than its rounding (1e-12 relative: near the
    minimum the true decrease is far below the rounding of the cost itself)."""
    p = np.array(p, np.float64)

    def parts(q):
        A, B, mu, s = q
        d = v - mu
        g = np.exp(-0.5 * (d / s) ** 2)
        r = A + B * g - c
        J = np.stack([np.ones_like(v), g, B * g * d / s ** 2, B * g * d ** 2 / s ** 3], axis=1)
        H = J.T @ J
        R = [float(np.sum(r * g * d ** j)) for j in range(5)]
        H[1, 2] += R[1] / s ** 2
        H[1, 3] += R[2] / s ** 3
        H[2, 2] += B * (R[2] / s ** 4 - R[0] / s ** 2)
        H[2, 3] += B * (R[3] / s ** 5 - 2 * R[1] / s ** 3)
        H[3, 3] += B * (R[4] / s ** 6 - 3 * R[2] / s ** 4)
        H[2, 1], H[3, 1], H[3, 2] = H[1, 2], H[1, 3], H[2, 3]
        return 0.5 * float(r @ r), J.T @ r, H

    cost, grad, H = parts(p)
    last = np.inf
    for _ in range(max_iter):
        try:
            np.linalg.cholesky(H)
        except np.linalg.LinAlgError:
            break
        dx = -np.linalg.solve(H, grad)
        scale = np.array([abs(p[0]), abs(p[0]), abs(p[3]), abs(p[3])])
        size = float(np.max(np.abs(dx) / scale))
        if not size < last:
            break
        q = p + dx
        cq, gq, Hq = parts(q)
        if not cq <= cost * (1.0 + 1e-12):
            break
        p, cost, grad, H, last = q, cq, gq, Hq, size
        if size <= 1e-15:
            break
    p[3] = abs(p[3])
    return p


def rv(F, star_or_range, mask_lambda, mask_weight, width_kms, v_lo, v_step, n_v):
    """RV (km/s) per spectrum: Gaussian centre of the CCF.  Returns (rv, params, ccf)."""
    c = ccf(F, star_or_range, mask_lambda, mask_weight, width_kms, v_lo, v_step, n_v)
    v = v_lo + v_step * np.arange(n_v)
    params = np.array([fit_gaussian(v, row) for row in c])
    return params[:, 2].copy(), params, c


# ---------------------------------------------------------------------------------------
# instrumental resolution (Sect. 3.3, after Eq. 4)
# ---------------------------------------------------------------------------------------
def instrument_kernel(resolving_power, delta_px):
    """Discrete line-spread function of an instrument of resolving power R on the log grid.

    The paper lowers the resolution of each integrated spectrum to the instrument's without
    giving the method.  Reading: a Gaussian line-spread function of FWHM lambda / R.  On a
    log-uniform grid that is a constant width in pixels, FWHM = 1 / (R Delta), sigma =
    FWHM / (2 sqrt(2 ln 2)).  Each tap is the Gaussian's mass over one pixel,
    g[k] = (erf((k + 1/2) / (sigma sqrt 2)) - erf((k - 1/2) / (sigma sqrt 2))) / 2, for
    |k| <= K = ceil(6 sigma) + 1, divided by their sum (the spectrum's flux is kept).  Off centre
    the mass is taken from erfc differences (no cancellation in the tails), and g[-k] = g[k].
    Returns (g, K) with g[K + k] the weight of a source pixel k pixels away."""
    import math
    sigma = 1.0 / (resolving_power * delta_px * 2.0 * math.sqrt(2.0 * math.log(2.0)))
    K = int(math.ceil(6.0 * sigma)) + 1
    s2 = sigma * math.sqrt(2.0)
    half = [math.erf(0.5 / s2)] + [0.5 * (math.erfc((k - 0.5) / s2) - math.erfc((k + 0.5) / s2))
                                   for k in range(1, K + 1)]
    g = np.array(half[:0:-1] + half)
    return g / g.sum(), K


def lower_resolution(F, resolving_power, delta_px):
    """F [..., n_px] convolved with the instrument kernel: out[m] = sum_k g[k] F[m - k], source
    indices clamped to the grid (the end values repeat, as for the Doppler shifts)."""
    F = np.asarray(F, np.float64)
    g, K = instrument_kernel(resolving_power, delta_px)
    n = F.shape[-1]
    m = np.arange(n)
    out = np.zeros_like(F)
    for k in range(-K, K + 1):
        out += g[K + k] * F[..., np.clip(m - k, 0, n - 1)]
    return out


# ---------------------------------------------------------------------------------------
# active-region size evolution (Sect. 4.2.1)
# ---------------------------------------------------------------------------------------
EVOLVE_NONE, EVOLVE_LINEAR_GROWTH, EVOLVE_LINEAR_DECAY, EVOLVE_ASYM_GAUSSIAN = 0, 1, 2, 3


def evolution_area(law, t, area0_msh=10000.0, rate_msh_per_day=400.0, t_peak_day=0.0,
                   fwhm_day=10.0, asymmetry=0.09):
    """Area (millionths of the solar hemisphere, MSH) of an evolving region at time t (days).

    Sect. 4.2.1 names three laws and their parameters; the formulas are this reading's:
      linear growth:  A = A0 + rate t                  (t >= 0; A0 before)
      linear decay:   A = max(0, A0 - rate t)          (t >= 0; A0 before)
      asymmetric Gaussian (Murakozy et al. 2014): A = A0 exp(-(t - t_peak)^2 / (2 s^2)) with
        s = s_rise before the peak and s_decay after it, s_rise + s_decay = FWHM / sqrt(2 ln 2)
        (the half-maximum points lie FWHM apart) and (s_decay - s_rise) / (s_decay + s_rise)
        = asymmetry (> 0: faster growth than decay)."""
    t = np.asarray(t, np.float64)
    if law == EVOLVE_LINEAR_GROWTH:
        return area0_msh + rate_msh_per_day * np.maximum(t, 0.0)
    if law == EVOLVE_LINEAR_DECAY:
        return np.maximum(0.0, area0_msh - rate_msh_per_day * np.maximum(t, 0.0))
    if law == EVOLVE_ASYM_GAUSSIAN:
        tot = fwhm_day / np.sqrt(2.0 * np.log(2.0))
        s_rise, s_decay = tot * (1.0 - asymmetry) / 2.0, tot * (1.0 + asymmetry) / 2.0
        s = np.where(t < t_peak_day, s_rise, s_decay)
        return area0_msh * np.exp(-0.5 * ((t - t_peak_day) / s) ** 2)
    raise ValueError("unknown evolution law")


def evolution_radius(area_msh):
    """Region radius (R*) of an area in MSH.  Reading: 10000 MSH = 1% of the visible hemisphere
    (Sect. 4.2.1), taken as the region's projected area at disk centre, r^2 = A 1e-6 (the same
    convention as 'a 1% spot' = r 0.1 in Sect. 4.1)."""
    return np.sqrt(np.asarray(area_msh, np.float64) * 1e-6)


# ---------------------------------------------------------------------------------------
# bisector injection (Sect. 4.3, "Convec.model")
# ---------------------------------------------------------------------------------------
def inject_bisectors(F, bis_table, orig_table, delta_px):
    """Local spectra [n_rows, n_px] (normalised: continuum 1) with their line bisectors replaced.

    The paper removes the original bisector and adds the target one per mu by shifting each
    spectral point according to its normalised depth.  Reading: a point n of depth
    d = clip(1 - F_n, 0, 1) moves by v = B_row(d) - B_orig(d) (km/s), i.e. to the pixel position
    u_n = n + atanh(v / c) / Delta on the log grid; the moved points are re-sampled at the pixel
    centres by linear interpolation in wavelength, as in Eq. 11 (for the bracketing moved points
    u_n <= m < u_n+1 the weight is (lambda_m - lambda'_n) / (lambda'_n+1 - lambda'_n) =
    expm1((m - u_n) Delta) / expm1((u_n+1 - u_n) Delta)); the end values repeat outside.
    Bisectors are tables over
    n_depth equally spaced depths 0..1 (linear in between): bis_table [n_rows, n_depth],
    orig_table [n_depth].  The moved positions must stay increasing."""
    F = np.atleast_2d(np.asarray(F, np.float64))
    bis = np.atleast_2d(np.asarray(bis_table, np.float64))
    orig = np.asarray(orig_table, np.float64)
    nd = orig.size
    depths = np.linspace(0.0, 1.0, nd)
    n = np.arange(F.shape[1], dtype=np.float64)
    out = np.empty_like(F)
    for r in range(F.shape[0]):
        d = np.clip(1.0 - F[r], 0.0, 1.0)
        v = np.interp(d, depths, bis[r]) - np.interp(d, depths, orig)
        u = n + np.arctanh(v / C_KMS) / delta_px
        if not np.all(np.diff(u) > 0):
            raise ValueError("moved positions are not increasing")
        k = np.searchsorted(u, n, side="right") - 1          # u[k] <= m < u[k+1]
        inside = (k >= 0) & (k < F.shape[1] - 1)
        kc = np.clip(k, 0, F.shape[1] - 2)
        w = np.expm1((n - u[kc]) * delta_px) / np.expm1((u[kc + 1] - u[kc]) * delta_px)
        val = F[r, kc] + w * (F[r, kc + 1] - F[r, kc])
        out[r] = np.where(inside, val, np.where(k < 0, F[r, 0], F[r, -1]))
    return out
