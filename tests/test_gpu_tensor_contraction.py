"""Active-phase contraction on the tensor cores (SOAP_BF16X3: Eqs. 1-4 as a GEMM over pixels x
phases x (class, mu bin, tap), BF16 hi/lo operands, three products, FP32 accumulation) against
the FP64 oracle at the mixed path's tolerances: 2e-6 of max F_quiet, 1 cm/s RV.  Cases: config 1
(all effects), four region classes with differential rotation and wide kernels, eight classes
over 70 phases (five phase groups), per-bin facula contrast (the operand-building kernel), the
full-size configuration (two phase groups, sampled pixels), no regions (every coefficient tile
skipped), RVs through soap_active_rv, and the precision refused where it does not apply."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2301_04259_gb300 import synth
from paper_2301_04259_gb300.synth import FACULA, SPOT, Region

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

DEV = "cuda:0"
TOL = 2e-6


@pytest.fixture(scope="module")
def S():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_2301_04259_gb300 import soap
    return soap


def _t(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def _active(S, case, regions, phases, effects, facula_mu=False):
    n_eff = bin(effects).count("1")
    with S.Disk(case.star, _t(case.quiet), {k: _t(v) for k, v in case.active.items()}) as d:
        if facula_mu:
            S.soap_set_facula_limb_brightening(d.ctx, True)
        out = torch.full((n_eff, len(phases), case.star.n_px), float("nan"), dtype=torch.float32, device=DEV)
        S.soap_active_phases(d.ctx, regions, phases, effects, S.SOAP_BF16X3, out)
        torch.cuda.synchronize()
    return out.double().cpu().numpy()


def _rel(a, b, scale):
    return float(np.abs(a - b).max() / scale)


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


def test_bf16x3_config1_all_effects(S):
    c = synth.config1(0)
    q = O.quiet(c.star, c.quiet)
    ref = O.active(c.star, c.quiet, c.active, c.regions, c.phases, effects=7)
    got = _active(S, c, c.regions, c.phases, 7)
    assert _rel(got, ref, q.max()) <= TOL


def test_bf16x3_four_classes_wide_kernels(S, complex_case):
    c = complex_case
    q = O.quiet(c.star, c.quiet)
    ref = O.active(c.star, c.quiet, c.active, c.regions, c.phases, effects=7)
    got = _active(S, c, c.regions, c.phases, 7)
    assert _rel(got, ref, q.max()) <= TOL


def test_bf16x3_facula_limb_brightening(S, complex_case):
    c = complex_case
    q = O.quiet(c.star, c.quiet)
    ref = O.active(c.star, c.quiet, c.active, c.regions, c.phases, effects=7, facula_mu=True)
    got = _active(S, c, c.regions, c.phases, 7, facula_mu=True)
    assert _rel(got, ref, q.max()) <= TOL


def test_bf16x3_full_size_sampled(S):
    """Disk 300x300, 205,800 px, 100 phases (two tiles of 64 phases): 64 sampled pixels of every
    phase against the oracle; every output finite."""
    c = synth.config2(0)
    rng = np.random.default_rng(5)
    pix = np.unique(np.concatenate([[0, 1, c.star.n_px - 2, c.star.n_px - 1],
                                    rng.integers(0, c.star.n_px, 60)])).astype(np.int64)
    q = O.quiet(c.star, c.quiet, pix=pix)
    ref = O.active(c.star, c.quiet, c.active, c.regions, c.phases, effects=1, pix=pix)
    got = _active(S, c, c.regions, c.phases, 1)
    assert np.isfinite(got).all()
    assert _rel(got[:, :, pix], ref, q.max()) <= TOL


def test_bf16x3_without_regions_is_the_quiet_star(S):
    c = synth.config1(1)
    q = O.quiet(c.star, c.quiet)
    got = _active(S, c, [], c.phases[:5], 1)
    assert _rel(got, np.broadcast_to(q, got.shape), q.max()) <= TOL


def test_bf16x3_rv_matches_oracle(S):
    """soap_active_rv at SOAP_BF16X3 against the oracle's RVs of the oracle's spectra (1 cm/s)."""
    c = synth.config1(3)
    lo, step, nv = synth.velocity_grid(c.star.vsini_kms)
    ref = O.active(c.star, c.quiet, c.active, c.regions, c.phases, effects=1)[0]
    rv_ref = O.rv(ref, c.star, c.mask_lambda, c.mask_weight, c.mask_width_kms, lo, step, nv)[0]
    with S.Disk(c.star, _t(c.quiet), {k: _t(v) for k, v in c.active.items()}) as d:
        spec = torch.empty((len(c.phases), c.star.n_px), dtype=torch.float32, device=DEV)
        rv = torch.empty(len(c.phases), dtype=torch.float64, device=DEV)
        S.soap_active_rv(d.ctx, c.regions, c.phases, S.SOAP_EFFECT_TOT, S.SOAP_BF16X3, c.mask_lambda,
                         c.mask_weight, c.mask_width_kms, lo, step, nv, spec, rv)
        torch.cuda.synchronize()
    assert np.abs(rv.cpu().numpy() - rv_ref).max() * 1e5 <= 1.0


def test_bf16x3_eight_classes_many_phases(S):
    """Eight region classes (every accumulator the tensor memory holds: groups of 16 phases) over 70
    phases (five phase groups, the last ragged), all three effects, against the oracle."""
    c = synth.config1(2)
    regs = [Region(SPOT if k % 2 else FACULA, -40.0 + 11.0 * k, 45.0 * k, 0.08 + 0.02 * k, 4300.0 + 250.0 * k)
            for k in range(8)]
    phases = np.linspace(0.0, 1.0, 70, endpoint=False)
    q = O.quiet(c.star, c.quiet)
    ref = O.active(c.star, c.quiet, c.active, regs, phases, effects=7)
    got = _active(S, c, regs, phases, 7)
    assert np.isfinite(got).all()
    assert _rel(got, ref, q.max()) <= TOL


def test_bf16x3_only_for_active_phases(S):
    c = synth.config1(0)
    with S.Disk(c.star, _t(c.quiet)) as d:
        with pytest.raises(S.SoapError):
            S.soap_quiet_spectrum(d.ctx, S.SOAP_FORM_TOEPLITZ, S.SOAP_BF16X3,
                                  torch.empty(c.star.n_px, dtype=torch.float32, device=DEV))
