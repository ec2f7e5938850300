"""Pins of the FP64 oracle against what the paper and the mathematics fix (no GPU).

Each test checks the oracle against something other than itself: closed forms, limits,
special cases that reduce to a library routine, a 50-digit brute-force rendering of the
paper's literal Eq. 11, invariants of Eqs. 1-4, and numbers the paper prints
(tests/golden/paper_values.json).
"""
import json
import math
import os

import numpy as np
import pytest

from oracle import oracle as O
from paper_2301_04259_gb300 import synth
from paper_2301_04259_gb300.synth import Region, Star, SPOT, FACULA

C_KMS = 299792.458
GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")


def _star(N=20, vsini=2.0, incl=90.0, u1=0.29, u2=0.34, l0=6000.0, l1=6010.0, n_px=512,
          mu_values=(0.25, 0.75), alpha=0.0):
    return Star(grid_n=N, vsini_kms=vsini, incl_deg=incl, u1=u1, u2=u2, lambda_start_A=l0,
                lambda_end_A=l1, n_px=n_px, mu_values=np.asarray(mu_values, float),
                diff_rot_alpha=alpha)


def _rand_spectra(rng, n_mu, n_px, n_lines=6):
    lam = synth.wavelength_grid(6000.0, 6010.0, n_px)
    out = np.empty((n_mu, n_px))
    for b in range(n_mu):
        c = rng.uniform(6000.5, 6009.5, n_lines)
        out[b] = synth._line_product(lam, c, rng.uniform(0.2, 0.8, n_lines), rng.uniform(0.05, 0.2, n_lines))
    return out


# ------------------------------------------------------------------------------------
# limb darkening and the sum over cells
# ------------------------------------------------------------------------------------
def test_total_intensity_tends_to_closed_form():
    """Sum_c I_c -> pi (1 - u1/3 - u2/6) for quadratic limb darkening as N grows."""
    u1, u2 = 0.29, 0.34
    exact = math.pi * (1 - u1 / 3 - u2 / 6)
    errs = {}
    for N in (50, 150, 300, 1000):
        I, _, _, _ = O.cell_geometry(_star(N=N, u1=u1, u2=u2))
        errs[N] = abs(I.sum() - exact) / exact
    assert errs[1000] < 2e-4
    assert errs[1000] < errs[50]
    assert errs[300] < errs[50]


def test_nearest_mu_binning_closed_form():
    """With mu values {0.25, 0.75}, cells with mu < 0.5 use bin 0; their total intensity is
    2 pi int_0^0.5 I(mu) mu dmu (since r dr = -mu dmu on the unit disk)."""
    u1, u2 = 0.29, 0.34
    I, _, mu, b = O.cell_geometry(_star(N=1000, u1=u1, u2=u2, mu_values=(0.25, 0.75)))

    def ring(m0, m1):
        f = lambda m: (1 - u1 * (1 - m) - u2 * (1 - m) ** 2) * m
        from scipy.integrate import quad
        return 2 * math.pi * quad(f, m0, m1)[0]

    assert I[b == 0].sum() == pytest.approx(ring(0.0, 0.5), rel=5e-4)
    assert I[b == 1].sum() == pytest.approx(ring(0.5, 1.0), rel=5e-4)
    assert np.all(b[I == 0] == -1)


def test_nonrotating_star_returns_local_spectra_times_total_intensity():
    """vsini = 0: every cell keeps its spectrum, so F = sum_b (sum_{c in b} I_c) S_b; with one
    spectrum for all bins, F = S * pi(1-u1/3-u2/6) up to the grid sum."""
    rng = np.random.default_rng(1)
    st = _star(N=40, vsini=0.0, n_px=256, mu_values=(0.2, 0.5, 0.9))
    S = _rand_spectra(rng, 1, 256)[0]
    q = np.stack([S, S, S])
    F = O.quiet(st, q)
    I, _, _, _ = O.cell_geometry(st)
    np.testing.assert_allclose(F, S * I.sum(), rtol=1e-14, atol=0)
    # distinct spectra per bin: weights per bin are the bin's total intensity
    q2 = _rand_spectra(rng, 3, 256)
    F2 = O.quiet(st, q2)
    _, _, _, b = O.cell_geometry(st)
    wb = np.array([I[b == k].sum() for k in range(3)])
    np.testing.assert_allclose(F2, wb @ q2, rtol=1e-14, atol=0)


# ------------------------------------------------------------------------------------
# Doppler shift + interpolation (Eqs. 6, 9-11)
# ------------------------------------------------------------------------------------
@pytest.mark.parametrize("v_kms", [0.731, -1.9, 5.5, -0.0004, 12.0])
def test_linear_spectrum_is_reproduced_exactly(v_kms):
    """Linear interpolation in lambda reproduces a spectrum linear in lambda: the shifted
    spectrum at lambda_m equals a + b lambda_m / D (D = sqrt((1+beta)/(1-beta)))."""
    lam = synth.wavelength_grid(6000.0, 6010.0, 400)
    a, b = 3.0, -4.0e-4
    S = a + b * lam
    beta = v_kms / C_KMS
    D = math.sqrt((1 + beta) / (1 - beta))
    for m in range(30, 370, 7):
        got = O.shift_interp(lam, S, beta, m)
        assert got == pytest.approx(a + b * lam[m] / D, rel=2e-15, abs=0)


@pytest.mark.parametrize("k", [1, 3, -2, 17])
def test_integer_pixel_velocity_translates_by_k_pixels(k):
    """beta = tanh(k Delta) gives D = exp(k Delta): the output is the input moved by k px."""
    rng = np.random.default_rng(2)
    lam = synth.wavelength_grid(6000.0, 6010.0, 300)
    dl = math.log(lam[-1] / lam[0]) / 299
    S = rng.uniform(0.2, 1.0, 300)
    beta = math.tanh(k * dl)
    for m in range(40, 260):
        assert O.shift_interp(lam, S, beta, m) == pytest.approx(S[m - k], abs=1e-12)


def test_single_cell_reduces_to_numpy_interp():
    """One shifted spectrum equals np.interp of (lambda D, S) at lambda (edge values repeated);
    np.interp uses the lambda-difference form, good to ~1e-10 here."""
    rng = np.random.default_rng(3)
    lam = synth.wavelength_grid(6000.0, 6010.0, 500)
    S = _rand_spectra(rng, 1, 500)[0]
    for v in (0.37, -2.2, 30.0, -45.0):
        beta = v / C_KMS
        D = math.sqrt((1 + beta) / (1 - beta))
        ref = np.interp(lam, lam * D, S)
        got = np.array([O.shift_interp(lam, S, beta, m) for m in range(500)])
        np.testing.assert_allclose(got, ref, rtol=0, atol=2e-10)


def test_redshift_moves_a_line_to_longer_wavelength():
    """v > 0 (receding) shifts a line to lambda_0 D > lambda_0."""
    lam = synth.wavelength_grid(6000.0, 6010.0, 2000)
    S = synth._line_product(lam, [6005.0], [0.6], [0.02])
    beta = 3.0 / C_KMS
    got = np.array([O.shift_interp(lam, S, beta, m) for m in range(2000)])
    c0 = np.sum(lam * (1 - S)) / np.sum(1 - S)
    c1 = np.sum(lam * (1 - got)) / np.sum(1 - got)
    D = math.sqrt((1 + beta) / (1 - beta))
    assert c1 - c0 == pytest.approx(c0 * (D - 1), rel=1e-3)


# ------------------------------------------------------------------------------------
# 50-digit brute force of the literal definitions (Alg. 1, Alg. 5, Eqs. 1-4, 6, 9-11)
# ------------------------------------------------------------------------------------
try:
    import mpmath
except ImportError:  # pragma: no cover
    mpmath = None
needs_mpmath = pytest.mark.skipif(mpmath is None, reason="mpmath not installed")


def _mp_disk(st, prec=60):
    mp = mpmath.mp
    mp.dps = prec
    N = st.grid_n
    cells = []
    incl = mp.mpf(st.incl_deg) * mp.pi / 180
    for j in range(N):
        for i in range(N):
            x = mp.mpf(2 * i + 1 - N) / N
            y = mp.mpf(2 * j + 1 - N) / N
            r2 = x * x + y * y
            if r2 >= 1:
                continue
            mu = mp.sqrt(1 - r2)
            om = 1 - mu
            I = (mp.mpf(2) / N) ** 2 * (1 - mp.mpf(st.u1) * om - mp.mpf(st.u2) * om * om)
            slat = y * mp.sin(incl) + mu * mp.cos(incl)
            v = mp.mpf(st.vsini_kms) * x * (1 + mp.mpf(st.diff_rot_alpha) * slat ** 2)
            b = min(range(st.n_mu), key=lambda k: (abs(mu - mp.mpf(st.mu_values[k])), k))
            cells.append((x, y, mu, I, v / mp.mpf(C_KMS), b))
    return cells


def _mp_grid(st):
    mp = mpmath.mp
    d = mp.log(mp.mpf(st.lambda_end_A) / mp.mpf(st.lambda_start_A)) / (st.n_px - 1)
    return [mp.mpf(st.lambda_start_A) * mp.exp(k * d) for k in range(st.n_px)]


def _mp_shift(lam, S, beta, m):
    """Eq. 6 then Eq. 11 literally: lambda'_n = lambda_n D, bracket, slope x distance."""
    mp = mpmath.mp
    D = mp.sqrt((1 + beta) / (1 - beta))
    lp = [l * D for l in lam]
    t = lam[m]
    if t < lp[0]:
        return S[0]
    if t >= lp[-1]:
        return S[-1]
    n = max(k for k in range(len(lp)) if lp[k] <= t)
    return (S[n + 1] - S[n]) / (lp[n + 1] - lp[n]) * (t - lp[n]) + S[n]


def _brute_case(N, seed):
    rng = np.random.default_rng(seed)
    st = _star(N=N, vsini=25.0, incl=70.0, n_px=64, mu_values=(0.23, 0.61, 0.97), alpha=-0.18)
    q = _rand_spectra(rng, 3, 64, n_lines=4)
    a = _rand_spectra(rng, 3, 64, n_lines=5)
    return st, q, a


@needs_mpmath
@pytest.mark.parametrize("N", [4, 8])
def test_quiet_matches_50_digit_brute_force(N):
    st, q, _ = _brute_case(N, 10 + N)
    mp = mpmath.mp
    cells = _mp_disk(st)
    lam = _mp_grid(st)
    Sm = [[mp.mpf(float(v)) for v in row] for row in q]
    ref = [mp.fsum(I * _mp_shift(lam, Sm[b], be, m) for (_, _, _, I, be, b) in cells)
           for m in range(st.n_px)]
    got = O.quiet(st, q)
    ref = np.array([float(r) for r in ref])
    np.testing.assert_allclose(got, ref, rtol=2e-15, atol=0)


def _mp_centre(lat, lon, incl, alpha, phase):
    mp = mpmath.mp
    la = mp.mpf(lat) * mp.pi / 180
    lo = (mp.mpf(lon) + 360 * mp.mpf(phase) * (1 + mp.mpf(alpha) * mp.sin(la) ** 2)) * mp.pi / 180
    ic = mp.mpf(incl) * mp.pi / 180
    px, py, pz = mp.cos(la) * mp.sin(lo), mp.sin(la), mp.cos(la) * mp.cos(lo)
    return px, py * mp.sin(ic) - pz * mp.cos(ic), py * mp.cos(ic) + pz * mp.sin(ic)


def _mp_planck_ratio(lam_A, ta, tq):
    mp = mpmath.mp
    hck = mp.mpf("6.62607015e-34") * mp.mpf(299792458) / mp.mpf("1.380649e-23") * mp.mpf(10) ** 10
    return mp.expm1(hck / (lam_A * tq)) / mp.expm1(hck / (lam_A * ta))


@needs_mpmath
def test_active_matches_50_digit_brute_force():
    """Alg. 5 + Eqs. 1-4: InfoMap with later regions overwriting, per-cell differences,
    sum, subtraction from the quiet integral; facula listed before an embedded spot."""
    N = 8
    st, q, a = _brute_case(N, 21)
    regs = [Region(FACULA, 15.0, -25.0, 0.55, 6100.0), Region(SPOT, 12.0, -20.0, 0.3, 4800.0)]
    phases = np.array([0.0, 0.07])
    mp = mpmath.mp
    cells = _mp_disk(st)
    lam = _mp_grid(st)
    Sq = [[mp.mpf(float(v)) for v in row] for row in q]
    Sa = [[mp.mpf(float(v)) for v in row] for row in a]
    got = O.active(st, q, {SPOT: a, FACULA: a}, regs, phases, effects=7)
    for p, ph in enumerate(phases):
        owner = []
        for (x, y, mu, I, be, b) in cells:
            o = -1
            for r, rg in enumerate(regs):
                P = _mp_centre(rg.lat_deg, rg.lon_deg, st.incl_deg, st.diff_rot_alpha, ph)
                dot = x * P[0] + y * P[1] + mu * P[2]
                cr = mp.sqrt(1 - mp.mpf(rg.radius_rstar) ** 2)
                assert abs(dot - cr) > 1e-9, "choose a case without cells on a region edge"
                if dot >= cr:
                    o = r
            owner.append(o)
        assert sum(o == 1 for o in owner) > 0 and sum(o == 0 for o in owner) > 0
        for m in range(st.n_px):
            Fq = mp.fsum(I * _mp_shift(lam, Sq[b], be, m) for (_, _, _, I, be, b) in cells)
            tot, flux, bconv = [], [], []
            for (x, y, mu, I, be, b), o in zip(cells, owner):
                if o < 0:
                    continue
                C = _mp_planck_ratio(lam[m], mp.mpf(regs[o].temp_K), mp.mpf(st.t_quiet_K))
                sq = _mp_shift(lam, Sq[b], be, m)
                sa = _mp_shift(lam, Sa[b], be, m)
                tot.append(I * (sq - C * sa))
                flux.append(I * (sq - C * sq))
                bconv.append(I * (sq - sa))
            exp = [Fq - mp.fsum(tot), Fq - mp.fsum(flux), Fq - mp.fsum(bconv)]
            for e in range(3):
                assert got[e, p, m] == pytest.approx(float(exp[e]), rel=3e-15, abs=1e-16)


# ------------------------------------------------------------------------------------
# rotational broadening of a delta line: analytic profile
# ------------------------------------------------------------------------------------
def test_delta_line_broadens_to_analytic_rotation_profile():
    """A one-pixel line on a rotating limb-darkened disk: the integrated deficit at pixel m
    is int G(x) hat(m - n0 - s(x)) dx with G(x) = int I dy = 2a(1-u1-u2) + (pi/2)(u1+2u2)a^2
    - (4/3)u2 a^3, a = sqrt(1-x^2), and s(x) the pixel shift of velocity vsini*x."""
    from scipy.integrate import quad
    u1, u2, vsini, N, n_px = 0.29, 0.34, 50.0, 400, 256
    dv = 2.0                                           # km/s per pixel
    dl = dv / C_KMS
    l0 = 6000.0
    st = _star(N=N, vsini=vsini, u1=u1, u2=u2, l0=l0, l1=l0 * math.exp(dl * (n_px - 1)),
               n_px=n_px, mu_values=(0.5,))
    n0, d = 128, 0.5
    S = np.ones(n_px); S[n0] = 1 - d
    F = O.quiet(st, S[None, :])
    I, _, _, _ = O.cell_geometry(st)
    deficit = (I.sum() - F) / d

    def G(x):
        a = math.sqrt(max(0.0, 1 - x * x))
        return 2 * a * (1 - u1 - u2) + 0.5 * math.pi * (u1 + 2 * u2) * a * a - 4.0 / 3.0 * u2 * a ** 3

    def s_of_x(x):
        return math.atanh(vsini * x / C_KMS) / dl

    def hat(t):
        return max(0.0, 1 - abs(t))

    ref = np.zeros(n_px)
    for m in range(n_px):
        kinks = [x for x in np.linspace(-1, 1, 4001) if abs(m - n0 - s_of_x(x)) < 1.0]
        if not kinks:
            continue
        lo, hi = max(-1.0, min(kinks) - 1e-3), min(1.0, max(kinks) + 1e-3)
        ref[m] = quad(lambda x: G(x) * hat(m - n0 - s_of_x(x)), lo, hi, limit=200)[0]
    peak = ref.max()
    assert np.abs(deficit - ref).max() < 3e-3 * peak
    # the profile is symmetric about the line and spans +-vsini
    np.testing.assert_allclose(deficit[n0 - 20:n0 + 21], deficit[n0 - 20:n0 + 21][::-1], atol=2e-3 * peak)
    assert deficit[n0 + 27] < 1e-12 and deficit[n0 - 27] < 1e-12


# ------------------------------------------------------------------------------------
# geometry readings pinned by the paper's numbers
# ------------------------------------------------------------------------------------
def test_differential_rotation_reading_reproduces_solar_numbers():
    """Sect. 3.4: omega0 = 360/PROT and omega1 = DIFF_ROT * omega0 reproduce the quoted solar
    law; the literal 'DIFF_ROT*PROT' does not.  The oracle's v/(vsini x) at latitude theta
    equals omega(theta)/omega0."""
    g = json.load(open(GOLDEN))["differential_rotation"]
    w0 = 360.0 / g["PROT_days"]
    assert w0 == pytest.approx(g["omega0_deg_per_day"], abs=5e-4)
    assert g["DIFF_ROT"] * w0 == pytest.approx(g["omega1_deg_per_day"], abs=5e-4)
    assert abs(g["DIFF_ROT"] * g["PROT_days"] - g["omega1_deg_per_day"]) > 1.0
    st = _star(N=60, vsini=2.0, incl=90.0, alpha=g["DIFF_ROT"])
    I, v, mu, _ = O.cell_geometry(st)
    N = st.grid_n
    jj, ii = np.divmod(np.arange(N * N), N)
    x = (2 * ii + 1 - N) / N
    y = (2 * jj + 1 - N) / N
    vis = I > 0
    omega = g["omega0_deg_per_day"] + g["omega1_deg_per_day"] * y[vis] ** 2   # i=90: sin(lat)=y
    np.testing.assert_allclose(v[vis], 2.0 * x[vis] * omega / g["omega0_deg_per_day"], rtol=3e-4, atol=1e-12)


def test_one_percent_spot_fits_paper_box():
    """Sect. 4.1: at N = 300 a disk-centre spot of 1% of the disk fits in 34 x 34 cells."""
    g = json.load(open(GOLDEN))["spot_box"]
    st = _star(N=g["grid_n"])
    r = math.sqrt(g["area_fraction"])
    im = O.infomap(st, [Region(SPOT, 0.0, 0.0, r, 4800.0)], 0.0)
    jj, ii = np.nonzero(im == 0)
    w, h = ii.max() - ii.min() + 1, jj.max() - jj.min() + 1
    assert w <= g["box_cells"] and h <= g["box_cells"]
    assert w >= g["box_cells"] - 6
    assert abs((im == 0).sum() / (im >= -1).sum() - g["area_fraction"]) < 1e-3


def test_regions_rotate_toward_the_receding_limb():
    """Rotation carries a region from disk centre toward +x, the side whose cells recede
    (v > 0): the velocity field and the phase motion describe the same rotation."""
    st = _star(N=100)
    reg = [Region(SPOT, 0.0, 0.0, 0.1, 4800.0)]
    _, v, _, _ = O.cell_geometry(st)
    N = st.grid_n
    xs = []
    for ph in (0.0, 0.03, 0.06):
        im = O.infomap(st, reg, ph)
        jj, ii = np.nonzero(im == 0)
        xs.append(np.mean((2 * ii + 1 - N) / N))
        vmean = np.mean(v.reshape(N, N)[jj, ii])
        if ph > 0:
            assert vmean > 0
    assert xs[0] == pytest.approx(0.0, abs=1e-12) and xs[0] < xs[1] < xs[2]
    assert xs[2] == pytest.approx(math.sin(2 * math.pi * 0.06), abs=0.01)
    # half a rotation later the spot is on the far side
    assert (O.infomap(st, reg, 0.5) >= 0).sum() == 0


# ------------------------------------------------------------------------------------
# invariants of Eqs. 1-4 / Alg. 5
# ------------------------------------------------------------------------------------
@pytest.fixture(scope="module")
def small_case():
    return synth.make_case(5, name="pins", grid_n=40, lambda_start=6000.0, lambda_end=6010.0,
                           n_px=600, mu_values=(0.15, 0.45, 0.75, 0.95), n_lines=12,
                           depth_law="uniform", sigma_law="angstrom", vsini_kms=4.0,
                           incl_deg=70.0, n_phases=6,
                           regions=[Region(FACULA, 20.0, 10.0, 0.3, 6100.0),
                                    Region(SPOT, 20.0, 10.0, 0.12, 4800.0)])


def test_zero_radius_region_gives_zero_residual(small_case):
    c = small_case
    F, dF = O.active(c.star, c.quiet, c.active, [Region(SPOT, 20.0, 10.0, 0.0, 4800.0)],
                     c.phases, effects=7, return_delta=True)
    assert np.all(dF == 0.0)


def test_active_equal_to_quiet_with_unit_contrast_gives_zero(small_case):
    c = small_case
    regs = [Region(SPOT, 20.0, 10.0, 0.2, c.star.t_quiet_K)]
    F, dF = O.active(c.star, c.quiet, {SPOT: c.quiet}, regs, c.phases, effects=7, return_delta=True)
    assert np.all(dF == 0.0)


def test_duplicated_region_changes_nothing(small_case):
    c = small_case
    one = O.active(c.star, c.quiet, c.active, c.regions[1:], c.phases, effects=7)
    two = O.active(c.star, c.quiet, c.active, c.regions[1:] * 2, c.phases, effects=7)
    assert np.array_equal(one, two)


def test_full_disk_cap_relates_effects_to_quiet_and_active_integrals(small_case):
    """A cap of radius 1 R* centred on the disk covers every visible cell, so
    Delta_flux = (1-C) F_q, Delta_bconv = F_q - F_a, Delta_tot = F_q - C F_a (Eqs. 1-3)."""
    c = small_case
    st = Star(**{**c.star.__dict__, "incl_deg": 90.0})
    regs = [Region(SPOT, 0.0, 0.0, 1.0, 4800.0)]
    F, dF = O.active(st, c.quiet, c.active, regs, np.array([0.0]), effects=7, return_delta=True)
    Fq = O.quiet(st, c.quiet)
    Fa = O.quiet(st, c.active[SPOT])
    lam = O.grid(st.lambda_start_A, st.lambda_end_A, st.n_px)
    C = O.contrast(lam, 4800.0, st.t_quiet_K)
    np.testing.assert_allclose(dF[0, 0], Fq - C * Fa, rtol=1e-13, atol=1e-14)
    np.testing.assert_allclose(dF[1, 0], (1 - C) * Fq, rtol=1e-13, atol=1e-14)
    np.testing.assert_allclose(dF[2, 0], Fq - Fa, rtol=1e-13, atol=1e-14)
    np.testing.assert_allclose(F[0, 0], C * Fa, rtol=1e-13, atol=1e-14)


def test_later_region_overwrites_earlier(small_case):
    """Alg. 5: a spot listed after a surrounding facula owns its cells; swapping the order
    lets the facula own them and changes the spectrum."""
    c = small_case
    im = O.infomap(c.star, c.regions, 0.0)
    im_swapped = O.infomap(c.star, c.regions[::-1], 0.0)
    spot_only = O.infomap(c.star, c.regions[1:], 0.0)
    assert np.array_equal(im == 1, spot_only == 0)
    assert (im == 0).sum() > 0
    assert np.all(im_swapped[spot_only == 0] == 1)            # facula (now index 1) owns all
    a = O.active(c.star, c.quiet, c.active, c.regions, c.phases[:2])
    b = O.active(c.star, c.quiet, c.active, c.regions[::-1], c.phases[:2])
    assert np.abs(a - b).max() > 1e-6


def test_phase_is_a_longitude_offset(small_case):
    c = small_case
    regs = [Region(SPOT, 20.0, 10.0, 0.2, 4800.0)]
    a = O.active(c.star, c.quiet, c.active, regs, np.array([0.1]), effects=7)
    regs2 = [Region(SPOT, 20.0, 10.0 + 36.0, 0.2, 4800.0)]
    b = O.active(c.star, c.quiet, c.active, regs2, np.array([0.0]), effects=7)
    np.testing.assert_allclose(a, b, rtol=0, atol=1e-14)


# ------------------------------------------------------------------------------------
# contrast (Planck ratio, Sect. 4.3.1)
# ------------------------------------------------------------------------------------
def test_contrast_limits_and_values():
    from scipy import constants as k
    assert O.planck_ratio(5000.0, 5778.0, 5778.0) == 1.0
    hck = k.h * k.c / k.k * 1e10
    # Wien limit (h c / lambda k T >> 1)
    lam, ta, tq = 1000.0, 3000.0, 4000.0
    assert O.planck_ratio(lam, ta, tq) == pytest.approx(math.exp(hck / lam * (1 / tq - 1 / ta)), rel=1e-12)
    # Rayleigh-Jeans limit: C -> Ta/Tq
    lam = 1e9
    xq, xa = hck / (lam * 5778.0), hck / (lam * 4800.0)
    assert O.planck_ratio(lam, 4800.0, 5778.0) == pytest.approx((xq / xa) * (1 + (xq - xa) / 2), rel=1e-9)
    # direct Planck law with scipy's constants at SOAP 2.0's mean wavelength
    g = json.load(open(GOLDEN))["contrast_wavelength"]
    l_m = g["lambda_A"] * 1e-10
    B = lambda T: 2 * k.h * k.c ** 2 / l_m ** 5 / math.expm1(k.h * k.c / (l_m * k.k * T))
    tq = g["t_quiet_K"]; ta = tq - g["delta_t_spot_K"]
    assert O.planck_ratio(g["lambda_A"], ta, tq) == pytest.approx(B(ta) / B(tq), rel=1e-13)


def test_spot_contrast_is_stronger_in_the_blue():
    """Sect. 4.3.1: the contrast of a cool spot departs more from 1 in the blue than the red."""
    c = [O.planck_ratio(l, 4800.0, 5778.0) for l in (3800.0, 5000.0, 6900.0)]
    assert 0 < c[0] < c[1] < c[2] < 1
    f = [O.planck_ratio(l, 6100.0, 5778.0) for l in (3800.0, 5000.0, 6900.0)]
    assert f[0] > f[1] > f[2] > 1


# ------------------------------------------------------------------------------------
# CCF and Gaussian RV (Sect. 4.1)
# ------------------------------------------------------------------------------------
def _ccf_case(n_px=3000, seed=7):
    rng = np.random.default_rng(seed)
    lam = synth.wavelength_grid(6000.0, 6030.0, n_px)
    cen = np.sort(rng.uniform(6001.0, 6029.0, 40))
    dep = rng.uniform(0.1, 0.7, 40)
    S = synth._line_product(lam, cen, dep, np.full(40, 0.04))
    return lam, S, cen, dep


def test_ccf_of_flat_spectrum_is_total_box_weight():
    lam, S, cen, dep = _ccf_case()
    dl = math.log1p((6030.0 - lam[0]) / lam[0]) / (lam.size - 1)
    W = 0.82
    c = O.ccf(np.ones_like(S), (lam[0], 6030.0), cen, dep, W, -10.0, 0.5, 41)
    np.testing.assert_allclose(c, dep.sum() * W / (C_KMS * dl), rtol=2e-15)


def test_ccf_matches_fine_riemann_sum():
    """Box integral of the piecewise-constant spectrum by a 4001-point midpoint rule."""
    lam, S, cen, dep = _ccf_case()
    dl = math.log(lam[-1] / lam[0]) / (lam.size - 1)
    W = 0.82
    vs = [-3.1, 0.0, 2.7]
    c = O.ccf(S, (lam[0], 6030.0), cen, dep, W, -3.1, 2.9, 2)
    h = W / (2 * C_KMS * dl)
    for k, v in enumerate([-3.1, -0.2]):
        tot = 0.0
        for l in range(cen.size):
            uc = (math.log(cen[l] / lam[0]) + math.atanh(v / C_KMS)) / dl
            t = uc - h + (np.arange(4001) + 0.5) * (2 * h / 4001)
            tot += dep[l] * S[np.floor(t + 0.5).astype(int)].sum() * (2 * h / 4001)
        assert c[0, k] == pytest.approx(tot, rel=2e-4)


def test_gaussian_fit_recovers_exact_gaussian():
    v = -20 + 0.25 * np.arange(161)
    p = (1234.5, -400.25, 0.1234567, 3.3)
    got = O.fit_gaussian(v, O.gaussian(v, *p))
    np.testing.assert_allclose(got, p, rtol=1e-10, atol=1e-11)


def _mp_cost(v, c, p, mp):
    A, B, mu, s = (mp.mpf(float(x)) for x in p)
    tot = mp.mpf(0)
    for vi, ci in zip(v, c):
        r = A + B * mp.exp(-((mp.mpf(float(vi)) - mu) / s) ** 2 / 2) - mp.mpf(float(ci))
        tot += r * r
    return tot


@pytest.mark.parametrize("shape", ["flat_bottom", "ccf"])
def test_gaussian_fit_is_the_least_squares_minimum(shape):
    """Sect. 4.1: the RV is the centre of the least-squares Gaussian.  On dips far from a
    Gaussian, the fitted parameters must be a local minimum of the cost at a resolution of
    1e-10 (relative to the width, or to the continuum for A and B): the cost, evaluated in
    40-digit arithmetic, may not drop under a move of that size in any parameter.  A fit that
    stops 2.5e-9 relative short of the minimum (what MINPACK's own stopping rule allowed)
    fails this on one side."""
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 40
    v = -22.0 + 0.25 * np.arange(177)
    if shape == "flat_bottom":
        c = 1000.0 - 300.0 * np.exp(-np.abs(v - 0.3) ** 3 / 60.0) + 4.0 * np.cos(v / 2.0)
    else:
        c = _rotation_ccf(v)
    p = O.fit_gaussian(v, c)
    base = _mp_cost(v, c, p, mp)
    steps = np.array([abs(p[0]), abs(p[0]), p[3], p[3]]) * 1e-10
    for i in range(4):
        for sgn in (1.0, -1.0):
            q = p.copy()
            q[i] += sgn * steps[i]
            assert _mp_cost(v, c, q, mp) >= base, (i, sgn)


def _rotation_ccf(v):
    """CCF-like dip: a rotationally broadened line (vsini 2 km/s, linear limb darkening 0.6)
    convolved with a Gaussian of 2.5 km/s, on a continuum, by direct quadrature."""
    x = np.linspace(-1.0, 1.0, 4001)
    prof = (2 * 0.4 * np.sqrt(1 - x ** 2) + 0.5 * np.pi * 0.6 * (1 - x ** 2))
    prof /= prof.sum()
    out = np.empty_like(v)
    for i, vi in enumerate(v):
        out[i] = 5000.0 - 1800.0 * np.sum(prof * np.exp(-0.5 * ((vi - 2.0 * x - 0.17) / 2.5) ** 2))
    return out


@pytest.mark.parametrize("k", [1, -3])
def test_integer_pixel_shift_changes_rv_by_c_tanh_k_delta(k):
    """Moving the spectrum by k pixels is a Doppler shift with atanh(v/c) = k Delta.  On a
    fixed velocity grid the Gaussian centre moves by c tanh(k Delta) up to the sampling bias
    of a non-Gaussian CCF (< 1 cm/s); on a grid whose step is c tanh(k Delta) and which moves
    with the spectrum, the CCF samples are the same and the centre moves by exactly one step
    (to the tanh curvature over the window, ~1e-7 km/s)."""
    lam, S, cen, dep = _ccf_case(n_px=4000, seed=8)
    dl = math.log1p((lam[-1] - lam[0]) / lam[0]) / (lam.size - 1)
    S2 = np.ones_like(S)
    if k > 0:
        S2[k:] = S[:-k]
    else:
        S2[:k] = S[-k:]
    rng_ = (lam[0], 6030.0)
    rv1, _, _ = O.rv(S[None], rng_, cen, dep, 0.82, -20.0, 0.25, 161)
    rv2, _, _ = O.rv(S2[None], rng_, cen, dep, 0.82, -20.0, 0.25, 161)
    shift = C_KMS * math.tanh(k * dl)
    assert rv2[0] - rv1[0] == pytest.approx(shift, abs=1e-5)
    step = abs(shift) / abs(k)
    sgn = 1 if k > 0 else -1
    v_lo = -60 * step
    rv1, _, _ = O.rv(S[None], rng_, cen, dep, 0.82, v_lo, step, 121)
    rv2, _, _ = O.rv(S2[None], rng_, cen, dep, 0.82, v_lo + sgn * abs(k) * step, step, 121)
    assert rv2[0] - rv1[0] == pytest.approx(shift, abs=2e-7)


@pytest.fixture(scope="module")
def rv_case():
    # isolated symmetric lines, no convective shift, i = 90 deg: only the flux effect acts
    rng = np.random.default_rng(11)
    c = synth.make_case(11, name="rv", grid_n=60, lambda_start=6000.0, lambda_end=6010.0,
                        n_px=4096, mu_values=(0.3, 0.7, 0.95), n_lines=8, depth_law="uniform",
                        sigma_law="angstrom", vsini_kms=2.0, incl_deg=90.0, n_phases=1, regions=[])
    cen = 6000.8 + 1.2 * np.arange(8) + rng.uniform(-0.1, 0.1, 8)
    dep = rng.uniform(0.3, 0.7, 8)
    sig = np.full(8, 0.05)
    lam = synth.wavelength_grid(6000.0, 6010.0, 4096)
    q1 = synth.local_spectra(lam, cen, dep, sig, c.star.mu_values, cb_kms_at_disk_centre=0.0)
    c.mask_lambda, c.mask_weight = cen, dep
    c.extra.update(line_centers=cen, line_depths=dep, line_sigmas=sig)
    return c, q1


def _rv_flux(c, q1, regs, phases):
    F = O.active(c.star, q1, {SPOT: q1}, regs, phases, effects=O.EFFECT_FLUX)[0]
    lo, st, nv = synth.velocity_grid(c.star.vsini_kms)
    r, _, _ = O.rv(F, c.star, c.mask_lambda, c.mask_weight, c.mask_width_kms, lo, st, nv)
    r0, _, _ = O.rv(O.quiet(c.star, q1)[None], c.star, c.mask_lambda, c.mask_weight,
                    c.mask_width_kms, lo, st, nv)
    return (r - r0[0]) * 1e5          # cm/s


def test_spot_on_approaching_limb_gives_redshift(rv_case):
    """A dark spot on the approaching (x < 0) half removes blueshifted light: RV > 0; on the
    receding half RV < 0."""
    c, q1 = rv_case
    regs = [Region(SPOT, 0.0, 0.0, 0.2, 4800.0)]
    rv = _rv_flux(c, q1, regs, np.array([-0.08, 0.08]))
    assert rv[0] > 1.0 and rv[1] < -1.0


def test_mirrored_spots_give_antisymmetric_rv(rv_case):
    c, q1 = rv_case
    ph = np.array([0.02, 0.07, 0.13])
    a = _rv_flux(c, q1, [Region(SPOT, 10.0, 30.0, 0.15, 4800.0)], ph)
    b = _rv_flux(c, q1, [Region(SPOT, 10.0, -30.0, 0.15, 4800.0)], -ph)
    np.testing.assert_allclose(a, -b, atol=0.1 + 1e-3 * np.abs(a).max())


def test_redshifted_quiet_spectrum_as_spot_gives_nonnegative_cb_rv(rv_case):
    """Sect. 4.3.1 check: the quiet spectrum redshifted by 300 m/s injected as the spot
    spectrum never gives a negative convective-blueshift RV."""
    g = json.load(open(GOLDEN))["cb_redshift_experiment"]
    c, q1 = rv_case
    lam = synth.wavelength_grid(6000.0, 6010.0, 4096)
    a = synth.local_spectra(lam, c.extra["line_centers"] * (1 + g["redshift_kms"] / C_KMS),
                            c.extra["line_depths"], c.extra["line_sigmas"], c.star.mu_values,
                            cb_kms_at_disk_centre=0.0)
    regs = [Region(SPOT, 0.0, 0.0, 0.1, 4800.0)]
    ph = np.linspace(-0.24, 0.24, 9)
    F = O.active(c.star, q1, {SPOT: a}, regs, ph, effects=O.EFFECT_BCONV)[0]
    lo, st, nv = synth.velocity_grid(c.star.vsini_kms)
    r, _, _ = O.rv(F, c.star, c.mask_lambda, c.mask_weight, c.mask_width_kms, lo, st, nv)
    r0, _, _ = O.rv(O.quiet(c.star, q1)[None], c.star, c.mask_lambda, c.mask_weight,
                    c.mask_width_kms, lo, st, nv)
    assert np.all((r - r0[0]) * 1e5 >= -1e-3)
    assert (r - r0[0]).max() > 0



# ---------------------------------------------------------------------------------------
# instrumental resolution (Sect. 3.3 after Eq. 4)
# ---------------------------------------------------------------------------------------
@pytest.mark.parametrize("R,delta", [(115000.0, 2.8986e-6), (50000.0, 2.9e-6), (60000.0, 1.0e-5),
                                     (1.0e6, 2.9e-6)])
def test_instrument_kernel_is_a_pixel_integrated_gaussian_of_fwhm_lambda_over_r(R, delta):
    """Taps sum to one and are symmetric; each equals the 50-digit mass of a Gaussian of FWHM
    1/(R Delta) pixels over its pixel (renormalised over the kept taps).  Where sigma >= 1.2 px
    the taps' variance is sigma^2 + 1/12 (a Gaussian convolved with a one-pixel box; by Poisson
    summation the discrete sum differs by terms ~exp(-2 pi^2 sigma^2) < 1e-12, and the truncation
    at 6 sigma by < 1e-8)."""
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 50
    g, K = O.instrument_kernel(R, delta)
    sigma = 1.0 / (R * delta * 2.0 * math.sqrt(2.0 * math.log(2.0)))
    assert abs(g.sum() - 1.0) < 1e-15
    np.testing.assert_array_equal(g, g[::-1])
    k = np.arange(-K, K + 1)
    if sigma >= 1.2:
        assert float(np.sum(k * k * g)) == pytest.approx(sigma ** 2 + 1.0 / 12.0, rel=1e-8)
    s2 = mp.mpf(sigma) * mp.sqrt(2)
    raw = [(mp.erf((mp.mpf(j) + mp.mpf(0.5)) / s2) - mp.erf((mp.mpf(j) - mp.mpf(0.5)) / s2)) / 2
           for j in range(-K, K + 1)]
    tot = mp.fsum(raw)
    for j in range(2 * K + 1):
        assert float(raw[j] / tot) == pytest.approx(g[j], rel=1e-13, abs=1e-300)


def test_lower_resolution_keeps_flux_centroid_and_adds_variance():
    """For lines far from the grid ends a discrete convolution with a unit-sum kernel keeps the
    equivalent width and, with a symmetric kernel, the centroid, and adds the kernel's variance
    to the line's (exact identities of discrete convolution), whatever the line shape."""
    rng = np.random.default_rng(3)
    n = 4001
    m = np.arange(n, dtype=np.float64)
    depth = np.zeros(n)
    for c, w, d in ((1200.3, 3.1, 0.6), (2000.0, 1.2, 0.3), (2890.7, 5.0, 0.45)):
        depth += d * np.exp(-0.5 * ((m - c) / w) ** 2) * (1 + 0.3 * np.sin(m / 7.0)) ** 2
    depth += 0.01 * rng.random(n) * ((m > 1500) & (m < 1510))
    F = 1.0 - depth
    out = O.lower_resolution(F, 115000.0, 2.8986e-6)
    g, K = O.instrument_kernel(115000.0, 2.8986e-6)
    kv = float(np.sum(np.arange(-K, K + 1) ** 2 * g))
    d_in, d_out = 1.0 - F, 1.0 - out
    assert d_out.sum() == pytest.approx(d_in.sum(), rel=1e-13)
    c_in, c_out = (m * d_in).sum() / d_in.sum(), (m * d_out).sum() / d_out.sum()
    assert c_out == pytest.approx(c_in, abs=1e-9)
    v_in = ((m - c_in) ** 2 * d_in).sum() / d_in.sum()
    v_out = ((m - c_out) ** 2 * d_out).sum() / d_out.sum()
    assert v_out == pytest.approx(v_in + kv, rel=1e-11)


def test_lower_resolution_of_a_flat_spectrum_and_at_the_edges():
    """A flat spectrum stays flat (unit-sum kernel); next to the ends the repeated end values
    enter: a step at the first pixel is smoothed only inward."""
    F = np.full((2, 300), 0.75)
    np.testing.assert_allclose(O.lower_resolution(F, 115000.0, 2.9e-6), F, rtol=0, atol=1e-15)
    S = np.zeros(300)
    S[:1] = 1.0
    out = O.lower_resolution(S, 115000.0, 2.9e-6)
    g, K = O.instrument_kernel(115000.0, 2.9e-6)
    # out[m] = sum over k >= m of g[K + k] (the clamped sources of row 0)
    for mm in range(K + 2):
        assert out[mm] == pytest.approx(g[K + mm:].sum(), rel=1e-14, abs=1e-17)



# ---------------------------------------------------------------------------------------
# active-region evolution (Sect. 4.2.1)
# ---------------------------------------------------------------------------------------
def test_evolution_laws_closed_forms():
    t = np.array([-2.0, 0.0, 1.5, 10.0, 30.0])
    np.testing.assert_allclose(O.evolution_area(O.EVOLVE_LINEAR_GROWTH, t),
                               [10000, 10000, 10600, 14000, 22000], rtol=1e-15)
    np.testing.assert_allclose(O.evolution_area(O.EVOLVE_LINEAR_DECAY, t),
                               [10000, 10000, 9400, 6000, 0], rtol=1e-15)
    # asymmetric Gaussian: peak value, half maxima FWHM apart, widths in the asymmetry's ratio
    tp, fwhm, a = 4.0, 10.0, 0.09
    A = lambda x: float(O.evolution_area(O.EVOLVE_ASYM_GAUSSIAN, x, t_peak_day=tp, fwhm_day=fwhm, asymmetry=a))
    assert A(tp) == 10000.0
    from scipy.optimize import brentq
    lo = brentq(lambda x: A(x) - 5000.0, tp - 20, tp)
    hi = brentq(lambda x: A(x) - 5000.0, tp, tp + 20)
    assert hi - lo == pytest.approx(fwhm, rel=1e-12)
    assert ((hi - tp) - (tp - lo)) / ((hi - tp) + (tp - lo)) == pytest.approx(a, rel=1e-10)
    assert O.evolution_radius(10000.0) == pytest.approx(0.1, rel=1e-15)


def test_per_phase_radii_reduce_to_fixed_regions(small_case):
    """Per-phase radii equal to the regions' own radii give the fixed-region spectra; radius 0
    at a phase gives the quiet spectrum there."""
    c = small_case
    phases = c.phases[:4]
    fixed = O.active(c.star, c.quiet, c.active, c.regions, phases, effects=7)
    radii = np.array([[r.radius_rstar for r in c.regions]] * len(phases))
    np.testing.assert_array_equal(O.active(c.star, c.quiet, c.active, c.regions, phases, effects=7, radii=radii),
                                  fixed)
    radii[2, :] = 0.0
    got = O.active(c.star, c.quiet, c.active, c.regions, phases, effects=1, radii=radii)
    q = O.quiet(c.star, c.quiet)
    np.testing.assert_allclose(got[0, 2], q, rtol=0, atol=1e-15 * np.abs(q).max())



# ---------------------------------------------------------------------------------------
# facula limb brightening (Sect. 4.3.1: SOAP 2.0's dT_f(mu))
# ---------------------------------------------------------------------------------------
def _dT_f(mu):
    return 250.9 - 407.7 * mu + 190.9 * mu * mu


def test_facula_mu_model_with_one_mu_bin_is_a_facula_at_that_temperature():
    """With a single tabulated mu every facula cell has dT_f(mu_0): the mu-dependent model must
    equal the plain model with the facula's temperature set to T_quiet + dT_f(mu_0)."""
    import dataclasses
    c = synth.make_case(9, name="fmu1", grid_n=36, lambda_start=6000.0, lambda_end=6010.0, n_px=500,
                        mu_values=(0.62,), n_lines=10, depth_law="uniform", sigma_law="angstrom",
                        vsini_kms=3.0, incl_deg=80.0, n_phases=4,
                        regions=[Region(FACULA, 15.0, 0.0, 0.3, 6100.0), Region(SPOT, 15.0, 5.0, 0.1, 4800.0)])
    got = O.active(c.star, c.quiet, c.active, c.regions, c.phases, effects=7, facula_mu=True)
    regs = [dataclasses.replace(c.regions[0], temp_K=c.star.t_quiet_K + _dT_f(0.62)), c.regions[1]]
    ref = O.active(c.star, c.quiet, c.active, regs, c.phases, effects=7)
    np.testing.assert_allclose(got, ref, rtol=0, atol=1e-14 * np.abs(ref).max())


def test_facula_mu_model_only_changes_facula_cells(small_case):
    """Spots are untouched by the facula model, and so is the convective-blueshift effect
    (Eq. 2 has no contrast); the flux effect of the faculae changes (their temperature now
    follows dT_f(mu) instead of the region's 6100 K)."""
    c = small_case
    spot_only = [r for r in c.regions if r.type == SPOT]
    a = O.active(c.star, c.quiet, c.active, spot_only, c.phases, effects=7, facula_mu=True)
    b = O.active(c.star, c.quiet, c.active, spot_only, c.phases, effects=7)
    np.testing.assert_array_equal(a, b)
    a = O.active(c.star, c.quiet, c.active, c.regions, c.phases, effects=7, facula_mu=True)
    b = O.active(c.star, c.quiet, c.active, c.regions, c.phases, effects=7)
    np.testing.assert_array_equal(a[2], b[2])
    assert np.abs(a[1] - b[1]).max() > 1e-6 * np.abs(b[1]).max()



# ---------------------------------------------------------------------------------------
# bisector injection (Sect. 4.3, Convec.model)
# ---------------------------------------------------------------------------------------
def _line_spectrum(n=800, centre=400.3, sigma=12.0, depth=0.7):
    m = np.arange(n, dtype=np.float64)
    return 1.0 - depth * np.exp(-0.5 * ((m - centre) / sigma) ** 2)


def test_bisector_injection_with_equal_bisectors_is_the_identity():
    F = np.stack([_line_spectrum(), _line_spectrum(centre=300.0)])
    tab = np.tile(np.linspace(-0.3, 0.2, 11), (2, 1))
    np.testing.assert_array_equal(O.inject_bisectors(F, tab, tab[0], 2.9e-6), F)


def test_constant_bisector_is_a_doppler_shift():
    """v(d) = a at every depth moves the whole spectrum by a: the result must equal the oracle's
    own Doppler shift + Eq. 9-11 interpolation (the C code's shift_interp, written separately),
    since both interpolate linearly in wavelength."""
    a = 0.37                                            # km/s
    delta = O.delta(6000.0, 6010.0, 800)
    F = _line_spectrum()
    got = O.inject_bisectors(F, np.full((1, 5), a), np.zeros(5), delta)[0]
    lam = O.grid(6000.0, 6010.0, 800)
    beta = math.tanh(math.atanh(a / C_KMS))             # the shift's v/c
    ref = np.array([O.shift_interp(lam, F, beta, m) for m in range(800)])
    np.testing.assert_allclose(got, ref, rtol=0, atol=1e-14)


def test_injected_linear_bisector_is_measured_back():
    """A symmetric line given the bisector v(d) = k d: the output line's bisector (midpoint of
    the two wing crossings at each flux level, in velocity) follows k d."""
    delta = 1.0e-6                                      # 0.3 km/s per pixel: a well-sampled line
    k = 0.4
    F = _line_spectrum(n=1200, centre=600.0, sigma=20.0, depth=0.8)
    out = O.inject_bisectors(F, np.array([[0.0, k]]), np.zeros(2), delta)[0]
    m = np.arange(out.size, dtype=np.float64)
    c0 = int(np.argmin(out))
    for level in (0.3, 0.5, 0.7, 0.9):
        f = 1.0 - level * 0.8                           # flux at normalised depth d = level * 0.8
        left = np.interp(f, out[:c0 + 1][::-1], m[:c0 + 1][::-1])
        right = np.interp(f, out[c0:], m[c0:])
        v_mid = ((left + right) / 2.0 - 600.0) * delta * C_KMS
        assert v_mid == pytest.approx(k * (1.0 - f), abs=0.01 * k)
