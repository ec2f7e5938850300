"""Instrumental resolution (Sect. 3.3, after Eq. 4): the library's line-spread function against
the oracle's, alone (any spectra, both kernel forms, ragged sizes, host and device) and inside
the quiet, active and RV calls.  Tolerances as everywhere: 1e-12 of max |F| for FP64, 2e-6 for
FP32; RVs 1e-6 cm/s (FP64) and 1 cm/s (FP32)."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2301_04259_gb300 import synth

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

DEV = "cuda:0"


@pytest.fixture(scope="module")
def S():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_2301_04259_gb300 import soap
    return soap


@pytest.fixture(scope="module")
def cfg1():
    return synth.config1(0)


def _t(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def _delta(star):
    return O.delta(star.lambda_start_A, star.lambda_end_A, star.n_px)


def _star(n_px, lam0=6000.0, lam1=6010.0):
    c = synth.config1(0)
    st = c.star
    st.n_px = n_px
    st.lambda_start_A, st.lambda_end_A = lam0, lam1
    lam = synth.wavelength_grid(lam0, lam1, n_px)
    rng = np.random.default_rng(n_px)
    q = synth.local_spectra(lam, rng.uniform(lam0, lam1, 20), rng.uniform(0.1, 0.8, 20),
                            rng.uniform(0.005, 0.05, 20), st.mu_values)
    return st, q


@pytest.mark.parametrize("R,n_px,n_spec", [(1.0e6, 4096, 3), (1.0e6, 1001, 1), (115000.0, 4096, 2),
                                           (115000.0, 777, 5), (3.0e6, 333, 2)])
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_lower_resolution_matches_oracle(S, R, n_px, n_spec, prec):
    """Windowed kernel (K <= 12: R = 1e6, 3e6 on this grid) and generic kernel (K = 55 at
    R = 115000), ragged pixel counts, device and host arrays."""
    st, q = _star(n_px)
    rng = np.random.default_rng(7)
    F = 1.0 - 0.5 * rng.random((n_spec, n_px)) ** 4
    dt = np.float64 if prec == "fp64" else np.float32
    F = F.astype(dt)
    ref = O.lower_resolution(F.astype(np.float64), R, _delta(st))
    tol = 1e-12 if prec == "fp64" else 2e-6
    with S.Disk(st, _t(q)) as d:
        S.soap_set_instrument_resolution(d.ctx, R)
        out = torch.empty(F.shape, dtype=torch.float64 if prec == "fp64" else torch.float32, device=DEV)
        S.soap_lower_resolution(d.ctx, _t(F), out)
        torch.cuda.synchronize()
        got = out.cpu().numpy().astype(np.float64)
        host_out = np.empty_like(F)
        S.soap_lower_resolution(d.ctx, F, host_out)
    assert np.abs(got - ref).max() <= tol * np.abs(ref).max()
    np.testing.assert_array_equal(host_out.astype(np.float64), got)


def test_lower_resolution_needs_a_resolution_and_a_kernel_that_fits(S):
    st, q = _star(512)
    F = np.ones((1, 512))
    with S.Disk(st, _t(q)) as d:
        with pytest.raises(S.SoapError):
            S.soap_lower_resolution(d.ctx, F, np.empty_like(F))
        with pytest.raises(S.SoapError):
            S.soap_set_instrument_resolution(d.ctx, 300.0)          # kernel wider than the 512-px grid
        with pytest.raises(S.SoapError):
            S.soap_set_instrument_resolution(d.ctx, -1.0)
        S.soap_set_instrument_resolution(d.ctx, 1.0e6)
        S.soap_set_instrument_resolution(d.ctx, 0.0)                # off again
        with pytest.raises(S.SoapError):
            S.soap_lower_resolution(d.ctx, F, np.empty_like(F))


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("R", [1.0e6, 115000.0])
def test_quiet_active_and_rv_with_the_instrument(S, cfg1, prec, R):
    """soap_quiet_spectrum, soap_active_phases (all three effects) and soap_active_rv with a
    resolution set equal the oracle's spectra degraded by the oracle's line-spread function;
    switching it off gives the undegraded spectra back."""
    c = cfg1
    p = S.SOAP_FP64 if prec == "fp64" else S.SOAP_FP32
    dt = torch.float64 if prec == "fp64" else torch.float32
    tol = 1e-12 if prec == "fp64" else 2e-6
    dl = _delta(c.star)
    q_ref = O.quiet(c.star, c.quiet)
    a_ref = O.active(c.star, c.quiet, c.active, c.regions, c.phases, effects=7)
    q_lsf = O.lower_resolution(q_ref, R, dl)
    a_lsf = O.lower_resolution(a_ref, R, dl)
    lo, step, nv = synth.velocity_grid(c.star.vsini_kms)
    rv_ref = O.rv(a_lsf[0], c.star, c.mask_lambda, c.mask_weight, c.mask_width_kms, lo, step, nv)[0]
    scale = np.abs(q_ref).max()
    with S.Disk(c.star, _t(c.quiet), {k: _t(v) for k, v in c.active.items()}) as d:
        S.soap_set_instrument_resolution(d.ctx, R)
        qo = torch.empty(c.star.n_px, dtype=dt, device=DEV)
        S.soap_quiet_spectrum(d.ctx, S.SOAP_FORM_TOEPLITZ, p, qo)
        ao = torch.empty((3, len(c.phases), c.star.n_px), dtype=dt, device=DEV)
        S.soap_active_phases(d.ctx, c.regions, c.phases, 7, p, ao)
        so = torch.empty((len(c.phases), c.star.n_px), dtype=dt, device=DEV)
        rv = torch.empty(len(c.phases), dtype=torch.float64, device=DEV)
        S.soap_active_rv(d.ctx, c.regions, c.phases, S.SOAP_EFFECT_TOT, p, c.mask_lambda, c.mask_weight,
                         c.mask_width_kms, lo, step, nv, so, rv)
        S.soap_set_instrument_resolution(d.ctx, 0.0)
        a_off = torch.empty((1, len(c.phases), c.star.n_px), dtype=dt, device=DEV)
        S.soap_active_phases(d.ctx, c.regions, c.phases, S.SOAP_EFFECT_TOT, p, a_off)
        torch.cuda.synchronize()
    assert np.abs(qo.double().cpu().numpy() - q_lsf).max() <= tol * scale
    assert np.abs(ao.double().cpu().numpy() - a_lsf).max() <= tol * scale
    assert np.abs(so.double().cpu().numpy() - a_lsf[0]).max() <= tol * scale
    assert np.abs(a_off[0].double().cpu().numpy() - a_ref[0]).max() <= tol * scale
    rv_tol = 1e-6 if prec == "fp64" else 1.0
    assert np.abs(rv.cpu().numpy() - rv_ref).max() * 1e5 <= rv_tol


def test_lower_resolution_full_size_fp32(S):
    """Full-size grid (205,800 px), HARPS-N-like R = 115000 (FWHM 3 px, windowed kernel): the
    library's FP32 line-spread function of 8 seeded spectra against the oracle's."""
    c = synth.config2(0)
    F = np.ascontiguousarray(c.quiet[:8]).astype(np.float32)
    ref = O.lower_resolution(F.astype(np.float64), 115000.0, _delta(c.star))
    with S.Disk(c.star, _t(c.quiet)) as d:
        S.soap_set_instrument_resolution(d.ctx, 115000.0)
        out = torch.empty(F.shape, dtype=torch.float32, device=DEV)
        S.soap_lower_resolution(d.ctx, _t(F), out)
        torch.cuda.synchronize()
    assert np.abs(out.double().cpu().numpy() - ref).max() <= 2e-6 * np.abs(ref).max()
