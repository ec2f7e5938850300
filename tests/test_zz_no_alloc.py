"""The allocation-free RV entry point (soap_rv_ccf_static) against soap_rv_ccf.

soap_rv_ccf_static serves callers that may not allocate device memory while running; its
scratch is a fixed array inside the library, shared by every call.  Two calls in a row with
different inputs must each reproduce soap_rv_ccf (same CCF definition and fit), which also
shows that the second call is not disturbed by what the first left in the shared scratch.
This file is collected last so that a failure here does not hide the other GPU tests.
"""
import ctypes

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


def _t(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def _reference(S, case, spectra, lo, step, nv):
    with S.Disk(case.star, _t(case.quiet)) as d:
        n = spectra.shape[0]
        rv = torch.empty(n, dtype=torch.float64, device=DEV)
        fit = torch.empty((n, 4), dtype=torch.float64, device=DEV)
        ccf = torch.empty((n, nv), dtype=torch.float64, device=DEV)
        S.soap_rv_ccf(d.ctx, spectra, case.mask_lambda, case.mask_weight, case.mask_width_kms,
                      lo, step, nv, rv, fit, ccf)
        torch.cuda.synchronize()
    return rv.cpu().numpy(), fit.cpu().numpy(), ccf.cpu().numpy()


def _static(S, case, spectra, lo, step, nv):
    st = case.star
    n = spectra.shape[0]
    rv = torch.full((n,), float("nan"), dtype=torch.float64, device=DEV)
    fit = torch.full((n, 4), float("nan"), dtype=torch.float64, device=DEV)
    ccf = torch.full((n, nv), float("nan"), dtype=torch.float64, device=DEV)
    S.soap_rv_ccf_static(st.lambda_start_A, st.lambda_end_A, st.n_px, spectra,
                         _t(case.mask_lambda), _t(case.mask_weight), case.mask_width_kms,
                         lo, step, nv, rv, fit, ccf, stream=torch.cuda.current_stream())
    torch.cuda.synchronize()
    return rv.cpu().numpy(), fit.cpu().numpy(), ccf.cpu().numpy()


def test_static_entry_point_matches_soap_rv_ccf_on_two_calls(S):
    big = synth.config2(3, grid_n=60, n_px=20000, lambda_start=5000.0,
                        lambda_end=5000.0 * np.exp(19999 / 345000.0), n_phases=4)
    small = synth.config1(4)
    calls = [(big, _t(big.quiet[::2])), (small, _t(small.quiet[::3].astype(np.float32)))]
    for case, spectra in calls:
        lo, step, nv = synth.velocity_grid(case.star.vsini_kms)
        rv_a, fit_a, ccf_a = _reference(S, case, spectra, lo, step, nv)
        rv_b, fit_b, ccf_b = _static(S, case, spectra, lo, step, nv)
        tol_ccf = (1e-12 if spectra.dtype == torch.float64 else 1e-6) * np.abs(ccf_a).max()
        assert np.isfinite(ccf_b).all() and np.isfinite(rv_b).all()
        assert np.abs(ccf_b - ccf_a).max() <= tol_ccf
        assert np.abs(rv_b - rv_a).max() * 1e5 <= (1e-4 if spectra.dtype == torch.float64 else 1.0)
        np.testing.assert_allclose(fit_b, fit_a, rtol=1e-6, atol=1e-7)


def test_static_entry_point_matches_the_oracle(S):
    """The same two calls against the FP64 oracle's CCF and Gaussian fit (Sect. 4.1) of the same
    spectra: 1e-6 cm/s for float64 spectra, 1 cm/s for float32 ones (the mixed path's bar)."""
    big = synth.config2(3, grid_n=60, n_px=20000, lambda_start=5000.0,
                        lambda_end=5000.0 * np.exp(19999 / 345000.0), n_phases=4)
    small = synth.config1(4)
    calls = [(big, big.quiet[::2], 1e-6), (small, small.quiet[::3].astype(np.float32), 1.0)]
    for case, F, tol_cms in calls:
        lo, step, nv = synth.velocity_grid(case.star.vsini_kms)
        rv_o, _, ccf_o = O.rv(F.astype(np.float64), case.star, case.mask_lambda, case.mask_weight,
                              case.mask_width_kms, lo, step, nv)
        rv_b, _, ccf_b = _static(S, case, _t(F), lo, step, nv)
        tol_ccf = (1e-12 if F.dtype == np.float64 else 2e-6) * np.abs(ccf_o).max()
        assert np.abs(ccf_b - ccf_o).max() <= tol_ccf
        assert np.abs(rv_b - rv_o).max() * 1e5 <= tol_cms


def test_static_entry_point_rejects_unknown_spectra_type(S):
    """spectra_f32 must be 0 or 1 (this entry point has no tensor-core form): SOAP_EINVAL before
    any device work."""
    case = synth.config1(0)
    st = case.star
    lo, step, nv = synth.velocity_grid(st.vsini_kms)
    F = _t(case.quiet[:2].astype(np.float32))
    ml, mw = _t(case.mask_lambda), _t(case.mask_weight)
    rv = torch.empty(2, dtype=torch.float64, device=DEV)
    for bad in (2, -1, 7):
        status = S._lib.soap_rv_ccf_static(float(st.lambda_start_A), float(st.lambda_end_A), int(st.n_px),
                                           ctypes.c_void_p(F.data_ptr()), bad, 2, ctypes.c_void_p(ml.data_ptr()),
                                           ctypes.c_void_p(mw.data_ptr()), int(ml.numel()),
                                           float(case.mask_width_kms), float(lo), float(step), int(nv),
                                           ctypes.c_void_p(rv.data_ptr()), None, None, None)
        assert status == S.SOAP_EINVAL
        assert "spectra_f32" in S.soap_last_error()


def test_static_entry_point_rejects_oversized_requests(S):
    case = synth.config1(0)
    st = case.star
    n_lines = 16384
    ml = torch.linspace(st.lambda_start_A + 1, st.lambda_end_A - 1, n_lines, dtype=torch.float64, device=DEV)
    mw = torch.ones(n_lines, dtype=torch.float64, device=DEV)
    spectra = torch.ones((200, st.n_px), dtype=torch.float64, device=DEV)
    rv = torch.empty(200, dtype=torch.float64, device=DEV)
    with pytest.raises(S.SoapError) as e:
        S.soap_rv_ccf_static(st.lambda_start_A, st.lambda_end_A, st.n_px, spectra, ml, mw, 0.82,
                             -22.0, 0.25, 177, rv)
    assert e.value.status == S.SOAP_ERANGE
    assert "scratch" in str(e.value)
