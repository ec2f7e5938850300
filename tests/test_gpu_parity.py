"""GPU parity: the CUDA library (through its C-ABI) against the FP64 oracle, element by element.

Tolerances (1e-12 relative flux for the FP64 path, 2e-6 relative flux and 1 cm/s RV
for the mixed path) are relative to max F_quiet of the oracle.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2301_04259_gb300 import synth
from paper_2301_04259_gb300.synth import FACULA, SPOT, Region, Star

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL64 = 1e-12
TOL32 = 2e-6


@pytest.fixture(scope="module")
def S():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_2301_04259_gb300 import soap
    return soap


DEV = "cuda:0"


def _t(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def gpu_quiet(S, case, form, prec):
    dt = torch.float64 if prec == S.SOAP_FP64 else torch.float32
    with S.Disk(case.star, _t(case.quiet)) as d:
        out = torch.empty(case.star.n_px, dtype=dt, device=DEV)
        S.soap_quiet_spectrum(d.ctx, form, prec, out)
        torch.cuda.synchronize()
    return out.double().cpu().numpy()


def gpu_active(S, case, regions, phases, effects, prec, active=None):
    dt = torch.float64 if prec == S.SOAP_FP64 else torch.float32
    n_eff = bin(effects).count("1")
    act = case.active if active is None else active
    with S.Disk(case.star, _t(case.quiet), {k: _t(v) for k, v in act.items()}) as d:
        out = torch.empty((n_eff, len(phases), case.star.n_px), dtype=dt, device=DEV)
        S.soap_active_phases(d.ctx, regions, phases, effects, prec, out)
        torch.cuda.synchronize()
    return out.double().cpu().numpy()


def rel(a, b, scale):
    return float(np.abs(a - b).max() / scale)


@pytest.fixture(scope="module")
def cfg1():
    return synth.config1(0)


@pytest.fixture(scope="module")
def cfg1_ref(cfg1):
    q = O.quiet(cfg1.star, cfg1.quiet)
    F = O.active(cfg1.star, cfg1.quiet, cfg1.active, cfg1.regions, cfg1.phases, effects=7)
    return q, F


# ------------------------------------------------------------------------------------------
# quiet star
# ------------------------------------------------------------------------------------------
@pytest.mark.parametrize("form", [0, 1], ids=["toeplitz", "direct"])
def test_quiet_config1(S, cfg1, cfg1_ref, form):
    ref, _ = cfg1_ref
    g64 = gpu_quiet(S, cfg1, form, S.SOAP_FP64)
    g32 = gpu_quiet(S, cfg1, form, S.SOAP_FP32)
    assert rel(g64, ref, ref.max()) <= TOL64
    assert rel(g32, ref, ref.max()) <= TOL32


QUIET_CASES = [
    # N, n_px, vsini, incl, alpha, n_mu
    (1, 300, 2.0, 90.0, 0.0, 1),
    (2, 257, 5.0, 60.0, 0.0, 2),
    (37, 1031, 8.0, 45.0, -0.18, 5),
    (64, 2049, 0.0, 90.0, 0.0, 3),
    (25, 700, 60.0, 30.0, 0.2, 4),
    (131, 4099, 3.0, 80.0, 0.0, 20),
]


@pytest.mark.parametrize("N,n_px,vsini,incl,alpha,n_mu", QUIET_CASES)
def test_quiet_ragged_and_edge_cases(S, N, n_px, vsini, incl, alpha, n_mu):
    case = synth.make_case(N + n_px, name="q", grid_n=N, lambda_start=6000.0, lambda_end=6010.0,
                           n_px=n_px, mu_values=np.linspace(0.1, 1.0, n_mu), n_lines=15,
                           depth_law="uniform", sigma_law="angstrom", vsini_kms=vsini,
                           incl_deg=incl, diff_rot_alpha=alpha, regions=[], n_phases=1)
    ref = O.quiet(case.star, case.quiet)
    for form in (0, 1):
        assert rel(gpu_quiet(S, case, form, S.SOAP_FP64), ref, ref.max()) <= TOL64
        assert rel(gpu_quiet(S, case, form, S.SOAP_FP32), ref, ref.max()) <= TOL32


@pytest.mark.parametrize("lam0,lam1,n_px,vsini", [(5000.0, 6000.0, 64, 2.0), (5000.0, 5500.0, 1000, 400.0)])
def test_quiet_library_atanh_and_expm1(S, lam0, lam1, n_px, vsini):
    """A coarse grid (Delta = 2.9e-3) and a 400 km/s rotator (|beta| up to 1.3e-3): the geometry
    takes the library atanh / expm1 instead of their short series."""
    case = synth.make_case(n_px, name="q", grid_n=33, lambda_start=lam0, lambda_end=lam1,
                           n_px=n_px, mu_values=np.linspace(0.1, 1.0, 4), n_lines=15,
                           depth_law="uniform", sigma_law="angstrom", vsini_kms=vsini,
                           incl_deg=70.0, diff_rot_alpha=0.0, regions=[], n_phases=1)
    ref = O.quiet(case.star, case.quiet)
    for form in (0, 1):
        assert rel(gpu_quiet(S, case, form, S.SOAP_FP64), ref, ref.max()) <= TOL64
        assert rel(gpu_quiet(S, case, form, S.SOAP_FP32), ref, ref.max()) <= TOL32


def test_quiet_cells_on_mu_bin_midpoints(S):
    """Cells whose mu lies exactly on the midpoint of two tabulated mu values (a tie: the lower
    bin, as the first minimum of |mu - mu_b|) or 1e-9 above one: the nearest-bin decision leaves
    the float midpoints for the FP64 comparison there and agrees with the oracle's."""
    N = 24
    x = (2 * np.arange(N) + 1 - N) / N
    r2 = x[:, None] * x[:, None] + x[None, :] * x[None, :]
    mu = np.sqrt(1.0 - r2[r2 < 1.0])
    d = 2.0 ** -6
    a = mu[np.argmin(np.abs(mu - 0.35))]             # tie: midpoint of a - d and a + d is a
    b = mu[np.argmin(np.abs(mu - 0.62))]             # just above the midpoint b - 1e-9
    assert a - d >= 0.25 and a + d < 0.5
    table = np.array([a - d, a + d, b - 1e-9 - d, b - 1e-9 + d, 1.0])
    assert 0.5 * (table[0] + table[1]) == a and np.all(np.diff(table) > 1e-4)
    case = synth.make_case(N + 400, name="q", grid_n=N, lambda_start=6000.0, lambda_end=6010.0,
                           n_px=400, mu_values=table, n_lines=15, depth_law="uniform",
                           sigma_law="angstrom", vsini_kms=2.0, incl_deg=90.0, diff_rot_alpha=0.0,
                           regions=[], n_phases=1)
    ref = O.quiet(case.star, case.quiet)
    for form in (0, 1):
        assert rel(gpu_quiet(S, case, form, S.SOAP_FP64), ref, ref.max()) <= TOL64


# ------------------------------------------------------------------------------------------
# active star
# ------------------------------------------------------------------------------------------
def test_active_config1_all_effects(S, cfg1, cfg1_ref):
    q, ref = cfg1_ref
    g64 = gpu_active(S, cfg1, cfg1.regions, cfg1.phases, 7, S.SOAP_FP64)
    g32 = gpu_active(S, cfg1, cfg1.regions, cfg1.phases, 7, S.SOAP_FP32)
    assert rel(g64, ref, q.max()) <= TOL64
    assert rel(g32, ref, q.max()) <= TOL32
    # the residual itself (Delta F = F_q - F), normalised by its own maximum
    dref = q[None, None] - ref
    d64 = q[None, None] - g64
    assert np.abs(d64 - dref).max() <= 1e-10 * np.abs(dref).max()


def test_active_wide_velocity_kernels(S):
    """vsini 8 km/s on the 4096-px grid of config 1: velocity kernels of ~135 taps, so the
    per-phase kernels need ~47 KB of dynamic shared memory on top of the kernel's static tables
    (more than the default 48 KB per launch); FP64 and FP32, all three effects."""
    c = synth.config1(2)
    c.star.vsini_kms = 8.0
    q = O.quiet(c.star, c.quiet)
    ref = O.active(c.star, c.quiet, c.active, c.regions, c.phases, effects=7)
    assert rel(gpu_active(S, c, c.regions, c.phases, 7, S.SOAP_FP64), ref, q.max()) <= TOL64
    assert rel(gpu_active(S, c, c.regions, c.phases, 7, S.SOAP_FP32), ref, q.max()) <= TOL32


@pytest.fixture(scope="module")
def complex_case():
    regs = [Region(FACULA, 25.0, -30.0, 0.3, 6100.0),
            Region(SPOT, 25.0, -30.0, 0.12, 4800.0),
            Region(SPOT, -10.0, 60.0, 0.2, 4300.0),
            Region(FACULA, -12.0, 58.0, 0.25, 6000.0)]
    c = synth.make_case(17, name="complex", grid_n=57, lambda_start=5000.0, lambda_end=5012.0,
                        n_px=3001, mu_values=np.linspace(0.05, 1.0, 9), n_lines=40,
                        depth_law="loguniform", sigma_law="velocity", vsini_kms=6.0,
                        incl_deg=62.0, diff_rot_alpha=-0.18, regions=regs, n_phases=13)
    lam = synth.wavelength_grid(5000.0, 5012.0, 3001)
    rng = np.random.default_rng(4)
    fac = synth.local_spectra(lam, rng.uniform(5000, 5012, 30), rng.uniform(0.1, 0.5, 30),
                              np.full(30, 0.05), c.star.mu_values, cb_kms_at_disk_centre=0.1)
    c.active = {SPOT: c.active[SPOT], FACULA: fac}
    c.phases = np.linspace(-0.3, 1.4, 13)
    return c


def test_active_complex_regions_classes_and_phases(S, complex_case):
    c = complex_case
    q = O.quiet(c.star, c.quiet)
    ref = O.active(c.star, c.quiet, c.active, c.regions, c.phases, effects=7)
    g64 = gpu_active(S, c, c.regions, c.phases, 7, S.SOAP_FP64)
    g32 = gpu_active(S, c, c.regions, c.phases, 7, S.SOAP_FP32)
    assert rel(g64, ref, q.max()) <= TOL64
    assert rel(g32, ref, q.max()) <= TOL32
    # single effects land in the right slot
    for k, e in enumerate((1, 2, 4)):
        one = gpu_active(S, c, c.regions, c.phases[:5], e, S.SOAP_FP64)
        assert rel(one[0], ref[k, :5], q.max()) <= TOL64


def test_active_degenerate_cases(S, cfg1, cfg1_ref):
    q, _ = cfg1_ref
    ph = np.array([0.0, 0.5, 0.77])
    # no regions: every phase is the quiet spectrum
    g = gpu_active(S, cfg1, [], ph, 7, S.SOAP_FP64)
    assert rel(g, np.broadcast_to(q, g.shape), q.max()) <= TOL64
    # zero radius
    g = gpu_active(S, cfg1, [Region(SPOT, 0.0, 0.0, 0.0, 4800.0)], ph, 1, S.SOAP_FP64)
    assert rel(g, np.broadcast_to(q, g.shape), q.max()) <= TOL64
    # a region on the far side at phase 0.5 leaves the quiet spectrum
    g = gpu_active(S, cfg1, [Region(SPOT, 0.0, 0.0, 0.2, 4800.0)], np.array([0.5]), 1, S.SOAP_FP64)
    assert rel(g[0, 0], q, q.max()) <= TOL64
    # cap covering the whole disk, one phase
    regs = [Region(SPOT, 0.0, 0.0, 1.0, 4800.0)]
    ref = O.active(cfg1.star, cfg1.quiet, cfg1.active, regs, np.array([0.0]), effects=7)
    g = gpu_active(S, cfg1, regs, np.array([0.0]), 7, S.SOAP_FP64)
    assert rel(g, ref, q.max()) <= TOL64


def test_active_maximum_sizes(S):
    """At the library's limits: 64 mu bins, 64 regions (overlapping spots and faculae in list
    order) of 8 classes (distinct type and temperature), 6 phases; FP64 and FP32."""
    rng = np.random.default_rng(64)
    temps = [(SPOT, 3900.0), (SPOT, 4300.0), (SPOT, 4700.0), (SPOT, 5100.0),
             (FACULA, 5900.0), (FACULA, 6000.0), (FACULA, 6100.0), (FACULA, 6200.0)]
    regs = []
    for k in range(64):
        typ, tk = temps[k % 8]
        regs.append(Region(typ, float(rng.uniform(-70, 70)), float(rng.uniform(0, 360)),
                           float(rng.uniform(0.02, 0.25)), tk))
    c = synth.make_case(640, name="max", grid_n=41, lambda_start=6000.0, lambda_end=6010.0, n_px=1500,
                        mu_values=(np.arange(64) + 0.5) / 64.0, n_lines=12, depth_law="uniform",
                        sigma_law="angstrom", vsini_kms=3.0, incl_deg=75.0, diff_rot_alpha=0.0,
                        regions=regs, n_phases=6)
    assert c.star.n_mu == S.SOAP_MAX_MU and len(regs) == S.SOAP_MAX_REGIONS
    q = O.quiet(c.star, c.quiet)
    ref = O.active(c.star, c.quiet, c.active, regs, c.phases, effects=7)
    assert rel(gpu_active(S, c, regs, c.phases, 7, S.SOAP_FP64), ref, q.max()) <= TOL64
    assert rel(gpu_active(S, c, regs, c.phases, 7, S.SOAP_FP32), ref, q.max()) <= TOL32


def test_active_is_deterministic_and_host_output_matches(S, complex_case):
    c = complex_case
    a = gpu_active(S, c, c.regions, c.phases, 7, S.SOAP_FP64)
    b = gpu_active(S, c, c.regions, c.phases, 7, S.SOAP_FP64)
    assert np.array_equal(a, b)
    with S.Disk(c.star, c.quiet, c.active) as d:            # host inputs and outputs
        out = np.empty((3, c.phases.size, c.star.n_px))
        S.soap_active_phases(d.ctx, c.regions, c.phases, 7, S.SOAP_FP64, out)
    assert np.array_equal(out, a)


def test_state_and_range_errors(S, cfg1):
    with S.Disk(cfg1.star, _t(cfg1.quiet)) as d:
        out = torch.empty((1, 2, cfg1.star.n_px), dtype=torch.float64, device=DEV)
        with pytest.raises(S.SoapError) as e:
            S.soap_active_phases(d.ctx, cfg1.regions, np.array([0.0, 0.1]), 1, S.SOAP_FP64, out)
        assert e.value.status == S.SOAP_ESTATE
        S.soap_set_active_spectrum(d.ctx, SPOT, _t(cfg1.active[SPOT]))
        regs = [Region(SPOT, 0.0, 0.0, 0.1, 4000.0 + 10 * k) for k in range(9)]
        with pytest.raises(S.SoapError) as e:
            S.soap_active_phases(d.ctx, regs, np.array([0.0, 0.1]), 1, S.SOAP_FP64, out)
        assert e.value.status == S.SOAP_ERANGE


# ------------------------------------------------------------------------------------------
# full size (disk 300x300, 205,800 px, 100 phases) on sampled pixels
# ------------------------------------------------------------------------------------------
@pytest.fixture(scope="module")
def cfg2():
    return synth.config2(0)


def _sample_pixels(n_px, seed=0, n=56):
    rng = np.random.default_rng(seed)
    edges = [0, 1, 2, 3, n_px - 4, n_px - 3, n_px - 2, n_px - 1]
    return np.unique(np.concatenate([edges, rng.integers(0, n_px, n)])).astype(np.int64)


def test_fullsize_config2_sampled_pixels(S, cfg2):
    c = cfg2
    pix = _sample_pixels(c.star.n_px)
    ref = O.active(c.star, c.quiet, c.active, c.regions, c.phases, effects=1, pix=pix)
    qref = O.quiet(c.star, c.quiet, pix=pix)
    g64 = gpu_active(S, c, c.regions, c.phases, 1, S.SOAP_FP64)
    g32 = gpu_active(S, c, c.regions, c.phases, 1, S.SOAP_FP32)
    scale = qref.max()
    assert rel(g64[:, :, pix], ref, scale) <= TOL64
    assert rel(g32[:, :, pix], ref, scale) <= TOL32
    # at every pixel: the two precisions agree, and phases with no visible region equal F_q
    assert np.isfinite(g64).all() and np.isfinite(g32).all()
    assert np.abs(g32 - g64).max() <= TOL32 * scale
    gq = gpu_quiet(S, c, 0, S.SOAP_FP64)
    assert rel(gq[pix], qref, scale) <= TOL64
    gqd = gpu_quiet(S, c, 1, S.SOAP_FP64)
    assert rel(gqd, gq, scale) <= TOL64


# ------------------------------------------------------------------------------------------
# CCF and RV (Sect. 4.1)
# ------------------------------------------------------------------------------------------
def _gpu_rv(S, case, spectra, lo, step, nv):
    with S.Disk(case.star, _t(case.quiet)) as d:
        sp = _t(spectra)
        n = spectra.shape[0]
        rv = torch.empty(n, dtype=torch.float64, device=DEV)
        fit = torch.empty((n, 4), dtype=torch.float64, device=DEV)
        ccf = torch.empty((n, nv), dtype=torch.float64, device=DEV)
        S.soap_rv_ccf(d.ctx, sp, case.mask_lambda, case.mask_weight, case.mask_width_kms, lo, step,
                      nv, rv, fit, ccf)
        torch.cuda.synchronize()
    return rv.cpu().numpy(), fit.cpu().numpy(), ccf.cpu().numpy()


def test_ccf_and_rv_config1(S, cfg1, cfg1_ref):
    _, ref = cfg1_ref
    lo, step, nv = synth.velocity_grid(cfg1.star.vsini_kms)
    F = ref[0]                                    # oracle spectra as input to both sides
    rv_o, fit_o, ccf_o = O.rv(F, cfg1.star, cfg1.mask_lambda, cfg1.mask_weight,
                              cfg1.mask_width_kms, lo, step, nv)
    rv_g, fit_g, ccf_g = _gpu_rv(S, cfg1, F, lo, step, nv)
    assert np.abs(ccf_g - ccf_o).max() <= 1e-12 * np.abs(ccf_o).max()
    assert np.abs(rv_g - rv_o).max() * 1e5 <= 1e-6          # cm/s
    np.testing.assert_allclose(fit_g, fit_o, rtol=1e-8, atol=1e-10)
    rv_32, _, ccf_32 = _gpu_rv(S, cfg1, F.astype(np.float32), lo, step, nv)
    assert np.abs(rv_32 - rv_o).max() * 1e5 <= 1.0


def test_rv_fp32_many_spectra_against_the_oracle(S, cfg1, cfg1_ref):
    """FP32 fits of few spectra take a block each, of many (more than 304) a warp each: 325 float32
    spectra (the 25 phases at 13 brightness scales, which leave the RV unchanged) against the
    oracle's RVs of the same spectra within 1 cm/s, and the 25 of the first scale fitted alone
    (one block each) against the same spectra inside the large call within 0.1 cm/s."""
    _, ref = cfg1_ref
    lo, step, nv = synth.velocity_grid(cfg1.star.vsini_kms)
    base = ref[0]
    F = np.concatenate([base * (1.0 + 0.002 * k) for k in range(13)]).astype(np.float32)
    assert F.shape[0] > 304
    rv_o, _, _ = O.rv(F.astype(np.float64), cfg1.star, cfg1.mask_lambda, cfg1.mask_weight,
                      cfg1.mask_width_kms, lo, step, nv)
    rv_many, _, _ = _gpu_rv(S, cfg1, F, lo, step, nv)
    assert np.isfinite(rv_many).all()
    assert np.abs(rv_many - rv_o).max() * 1e5 <= 1.0
    rv_few, _, _ = _gpu_rv(S, cfg1, F[:25], lo, step, nv)
    assert np.abs(rv_few - rv_many[:25]).max() * 1e5 <= 0.1


def _tile_np(c, width, step, nv, lo):
    """Pixels a group of 4 consecutive velocities can reach for one line (the tiled CCF kernel
    runs for 2..4): box width plus the largest spread of 4 box positions, + 2."""
    st = c.star
    delta = np.log(st.lambda_end_A / st.lambda_start_A) / (st.n_px - 1)
    s = np.arctanh((lo + step * np.arange(nv)) / 299792.458) / delta
    return int(np.floor((s[3:] - s[:-3]).max() + width / (299792.458 * delta) + 1e-6)) + 2


@pytest.mark.parametrize("width,step,n_spec", [(0.82, 0.25, 17), (0.3, 0.15, 1), (1.6, 0.25, 33),
                                               (0.82, 0.5, 16), (0.82, 0.25, 22), (0.82, 0.25, 29)])
def test_ccf_fp32_sorted_mask_matches_oracle(S, cfg2, width, step, n_spec):
    """FP32 spectra, mask sorted by wavelength, full-size grid (205,800 px, 12,946 lines): the
    CCF element by element against the oracle's on the same (FP32-rounded) spectra, for boxes
    of 0.35 / 0.94 / 1.84 px and velocity steps of 0.15 / 0.25 / 0.5 km/s (2, 3 and 4 pixels per
    group of 4 velocities), with 1, 16, 17, 22, 29 and 33 spectra (full rows of 16, and a last
    row of 1, 6 or 13 spectra computed as 4, 8 or 16 over its own line split)."""
    c = cfg2
    half = c.star.vsini_kms + 20.0
    nv = int(np.floor(2 * half / step + 1e-9)) + 1
    lo = -half
    assert 2 <= _tile_np(c, width, step, nv, lo) <= 4
    F = np.concatenate([c.quiet, c.quiet[::-1] * 0.97])[:n_spec].astype(np.float32)
    ccf_o = O.ccf(F.astype(np.float64), c.star, c.mask_lambda, c.mask_weight, width, lo, step, nv)
    with S.Disk(c.star, _t(c.quiet)) as d:
        rv = torch.empty(n_spec, dtype=torch.float64, device=DEV)
        ccf = torch.empty((n_spec, nv), dtype=torch.float64, device=DEV)
        S.soap_rv_ccf(d.ctx, _t(F), c.mask_lambda, c.mask_weight, width, lo, step, nv, rv, None, ccf)
        torch.cuda.synchronize()
    ccf_g = ccf.cpu().numpy()
    assert np.abs(ccf_g - ccf_o).max() <= 2e-6 * np.abs(ccf_o).max()


def test_ccf_unsorted_mask_matches_sorted(S, cfg1, cfg1_ref):
    """The windowed kernel (mask sorted by wavelength) and the generic one (any order) agree."""
    _, ref = cfg1_ref
    lo, step, nv = synth.velocity_grid(cfg1.star.vsini_kms)
    F = ref[0, :7]
    rv_a, _, ccf_a = _gpu_rv(S, cfg1, F, lo, step, nv)
    perm = np.random.default_rng(5).permutation(cfg1.mask_lambda.size)
    c2 = synth.config1(0)
    c2.mask_lambda, c2.mask_weight = cfg1.mask_lambda[perm].copy(), cfg1.mask_weight[perm].copy()
    rv_b, _, ccf_b = _gpu_rv(S, c2, F, lo, step, nv)
    assert np.abs(ccf_a - ccf_b).max() <= 1e-13 * np.abs(ccf_a).max()
    assert np.abs(rv_a - rv_b).max() * 1e5 <= 1e-6
    rv_c, _, ccf_c = _gpu_rv(S, c2, F.astype(np.float32), lo, step, nv)
    assert np.abs(rv_c - rv_a).max() * 1e5 <= 1.0


def test_ccf_and_rv_fullsize(S, cfg2):
    c = cfg2
    lo, step, nv = synth.velocity_grid(c.star.vsini_kms)
    F = c.quiet[::4]                               # seeded local spectra at full size
    rv_o, _, ccf_o = O.rv(F, c.star, c.mask_lambda, c.mask_weight, c.mask_width_kms, lo, step, nv)
    rv_g, _, ccf_g = _gpu_rv(S, c, F, lo, step, nv)
    assert np.abs(ccf_g - ccf_o).max() <= 1e-12 * np.abs(ccf_o).max()
    assert np.abs(rv_g - rv_o).max() * 1e5 <= 1e-6
    rv_32, _, _ = _gpu_rv(S, c, F.astype(np.float32), lo, step, nv)
    assert np.abs(rv_32 - rv_o).max() * 1e5 <= 1.0



@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_evolving_regions_match_oracle(S, cfg1, prec):
    """Sect. 4.2.1: a spot growing and decaying as an asymmetric Gaussian and a second one
    decaying linearly; per-phase radii from soap_evolve_radii, spectra from
    soap_active_phases_radii against the oracle's per-phase computation (all effects)."""
    c = cfg1
    regs = [Region(SPOT, 20.0, 10.0, 0.1, 4800.0), Region(SPOT, -30.0, 200.0, 0.05, 4300.0)]
    phases = np.linspace(0.0, 1.2, 9)
    t = phases * 25.0                                  # days (a 25-day rotation)
    evo = [{"law": 3, "area0_msh": 12000.0, "t_peak_day": 10.0, "fwhm_day": 12.0, "asymmetry": 0.09},
           {"law": 2, "area0_msh": 9000.0, "rate_msh_per_day": 400.0}]
    radii = S.soap_evolve_radii(evo, regs, t)
    ref = O.active(c.star, c.quiet, c.active, regs, phases, effects=7, radii=radii)
    p = S.SOAP_FP64 if prec == "fp64" else S.SOAP_FP32
    dt = torch.float64 if prec == "fp64" else torch.float32
    with S.Disk(c.star, _t(c.quiet), {k: _t(v) for k, v in c.active.items()}) as d:
        out = torch.empty((3, len(phases), c.star.n_px), dtype=dt, device=DEV)
        S.soap_active_phases_radii(d.ctx, regs, phases, radii, 7, p, out)
        torch.cuda.synchronize()
    tol = TOL64 if prec == "fp64" else TOL32
    q = O.quiet(c.star, c.quiet)
    assert rel(out.double().cpu().numpy(), ref, np.abs(q).max()) <= tol



@pytest.mark.parametrize("which", ["complex_facula", "config2_sample"])
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_facula_limb_brightening_matches_oracle(S, complex_case, cfg2, which, prec):
    """Sect. 4.3.1: faculae at T_quiet + dT_f(mu_b) (one contrast row per class and mu bin, each
    bin folded separately in the contraction) against the oracle's per-cell model; all effects.
    The full-size case samples 60 pixels of 3 phases."""
    p = S.SOAP_FP64 if prec == "fp64" else S.SOAP_FP32
    dt = torch.float64 if prec == "fp64" else torch.float32
    tol = TOL64 if prec == "fp64" else TOL32
    if which == "complex_facula":
        c, phases, pix = complex_case, complex_case.phases, None
    else:
        c, phases = cfg2, cfg2.phases[::40]
        pix = _sample_pixels(cfg2.star.n_px, seed=3, n=60)
    ref = O.active(c.star, c.quiet, c.active, c.regions, phases, effects=7, facula_mu=True, pix=pix)
    q = O.quiet(c.star, c.quiet, pix=pix)
    with S.Disk(c.star, _t(c.quiet), {k: _t(v) for k, v in c.active.items()}) as d:
        S.soap_set_facula_limb_brightening(d.ctx, True)
        out = torch.empty((3, len(phases), c.star.n_px), dtype=dt, device=DEV)
        S.soap_active_phases(d.ctx, c.regions, phases, 7, p, out)
        torch.cuda.synchronize()
    got = out.double().cpu().numpy()
    if pix is not None:
        got = got[:, :, pix]
    assert rel(got, ref, np.abs(q).max()) <= tol
