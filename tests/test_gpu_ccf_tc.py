"""The line-mask CCF of Sect. 4.1 on the tensor cores (soap_rv_ccf with tensor_cores=True, and
soap_active_rv at SOAP_BF16X3): CCF[s][k] = sum_n F[s][n] M[k][n] as a tcgen05 GEMM over pixels,
the mask matrix M built once from the line and velocity tables, both operands split
into BF16 hi + lo and three products accumulated in FP32, against the FP64 oracle's CCF of the
same (FP32-rounded) spectra.

Tolerance of the CCF, from the arithmetic: x = hi + lo + e with |e| <= 2^-16 |x| (two BF16
roundings of 8 significant bits), so each product misses lo_x lo_y, e_x y and x e_y: at most
3 x 2^-16 = 4.6e-5 of the product, and every product is positive (fluxes and mask weights), so
the same fraction of the CCF bounds the split error; FP32 accumulation over a chunk of at most
2,048 pixels adds at most 2,048 x 2^-24 = 1.2e-4.  Hence 1.7e-4 of the largest CCF value.  The
RVs are held to the mixed path's bar (1 cm/s of the FP64 result)."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2301_04259_gb300 import synth

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

DEV = "cuda:0"
TOL_CCF = 1.7e-4


@pytest.fixture(scope="module")
def S():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_2301_04259_gb300 import soap
    return soap


@pytest.fixture(scope="module")
def cfg2():
    return synth.config2(0)


def _t(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def _spectra(c, n_spec):
    """n_spec FP32 spectra: the local spectra of the case, each row scaled a little differently."""
    q = c.quiet
    rows = [q[i % q.shape[0]] * (1.0 - 1e-3 * i) for i in range(n_spec)]
    return np.stack(rows).astype(np.float32)


def _tc_ccf(S, c, F, width, lo, step, nv, tensor_cores=True):
    n = F.shape[0]
    with S.Disk(c.star, _t(c.quiet)) as d:
        rv = torch.empty(n, dtype=torch.float64, device=DEV)
        ccf = torch.empty((n, nv), dtype=torch.float64, device=DEV)
        S.soap_rv_ccf(d.ctx, _t(F), c.mask_lambda, c.mask_weight, width, lo, step, nv, rv, None, ccf,
                      tensor_cores=tensor_cores)
        torch.cuda.synchronize()
    return rv.cpu().numpy(), ccf.cpu().numpy()


@pytest.mark.parametrize("width,step,n_spec", [(0.82, 0.25, 17), (0.3, 0.2, 1), (1.6, 0.25, 33),
                                               (0.82, 0.5, 130)])
def test_ccf_tc_matches_oracle_fullsize(S, cfg2, width, step, n_spec):
    """Full-size grid (205,800 px, 12,946 lines): boxes of 0.35 / 0.94 / 1.84 px, 89 to 221
    velocities, 1 to 130 spectra (130: a second, ragged tile of spectra)."""
    c = cfg2
    half = c.star.vsini_kms + 20.0
    nv = int(np.floor(2 * half / step + 1e-9)) + 1
    assert nv <= 256                                   # the tensor-core form applies
    lo = -half
    F = _spectra(c, n_spec)
    ccf_o = O.ccf(F.astype(np.float64), c.star, c.mask_lambda, c.mask_weight, width, lo, step, nv)
    _, ccf_g = _tc_ccf(S, c, F, width, lo, step, nv)
    assert np.isfinite(ccf_g).all()
    assert np.abs(ccf_g - ccf_o).max() <= TOL_CCF * np.abs(ccf_o).max()


def test_ccf_tc_rv_fullsize(S, cfg2):
    """RVs of the full-size local spectra through the tensor-core CCF within 1 cm/s of the
    oracle's (FP64 spectra, FP64 CCF and fit)."""
    c = cfg2
    lo, step, nv = synth.velocity_grid(c.star.vsini_kms)
    F = c.quiet[::4]
    rv_o, _, _ = O.rv(F, c.star, c.mask_lambda, c.mask_weight, c.mask_width_kms, lo, step, nv)
    rv_g, _ = _tc_ccf(S, c, F.astype(np.float32), c.mask_width_kms, lo, step, nv)
    assert np.abs(rv_g - rv_o).max() * 1e5 <= 1.0


def test_ccf_tc_odd_pixel_count(S):
    """20,003 px (rows not 16-byte aligned: the element-wise loads; a ragged last chunk) and a
    small disk, against the oracle."""
    c = synth.config2(0, grid_n=60, n_px=20003)
    lo, step, nv = synth.velocity_grid(c.star.vsini_kms)
    F = _spectra(c, 9)
    ccf_o = O.ccf(F.astype(np.float64), c.star, c.mask_lambda, c.mask_weight, c.mask_width_kms, lo, step, nv)
    rv_o = np.array([O.fit_gaussian(lo + step * np.arange(nv), row)[2] for row in ccf_o])
    rv_g, ccf_g = _tc_ccf(S, c, F, c.mask_width_kms, lo, step, nv)
    assert np.abs(ccf_g - ccf_o).max() <= TOL_CCF * np.abs(ccf_o).max()
    assert np.abs(rv_g - rv_o).max() * 1e5 <= 1.0


def test_ccf_tc_agrees_with_simt_form(S, cfg2):
    """The tensor-core and the FP32 SIMT CCF of the same spectra: within the split tolerance of
    each other, and the same RVs within 1 cm/s."""
    c = cfg2
    lo, step, nv = synth.velocity_grid(c.star.vsini_kms)
    F = _spectra(c, 40)
    rv_a, ccf_a = _tc_ccf(S, c, F, c.mask_width_kms, lo, step, nv, tensor_cores=True)
    rv_b, ccf_b = _tc_ccf(S, c, F, c.mask_width_kms, lo, step, nv, tensor_cores=False)
    assert np.abs(ccf_a - ccf_b).max() <= TOL_CCF * np.abs(ccf_b).max()
    assert np.abs(rv_a - rv_b).max() * 1e5 <= 1.0


def test_ccf_tc_unsorted_mask_runs_simt(S):
    """A mask not sorted by wavelength has no tensor-core form: the same result as the FP32 path."""
    c = synth.config1(0)
    lo, step, nv = synth.velocity_grid(c.star.vsini_kms)
    perm = np.random.default_rng(5).permutation(c.mask_lambda.size)
    c.mask_lambda, c.mask_weight = c.mask_lambda[perm].copy(), c.mask_weight[perm].copy()
    F = _spectra(c, 5)
    rv_a, ccf_a = _tc_ccf(S, c, F, c.mask_width_kms, lo, step, nv, tensor_cores=True)
    rv_b, ccf_b = _tc_ccf(S, c, F, c.mask_width_kms, lo, step, nv, tensor_cores=False)
    assert np.array_equal(ccf_a, ccf_b) and np.array_equal(rv_a, rv_b)


def test_ccf_tc_needs_float32(S):
    c = synth.config1(0)
    lo, step, nv = synth.velocity_grid(c.star.vsini_kms)
    with pytest.raises(ValueError):
        _tc_ccf(S, c, c.quiet[:2], c.mask_width_kms, lo, step, nv)


def test_ccf_tc_many_spectra(S, cfg2):
    """800 spectra (7 tiles of 128, the last ragged): pixel chunks at their cap of 2,048 px, so
    the CTAs take several waves; sampled spectra (tile edges) against the oracle."""
    c = cfg2
    lo, step, nv = synth.velocity_grid(c.star.vsini_kms)
    F = _spectra(c, 800)
    rows = np.array([0, 127, 128, 511, 640, 799])
    ccf_o = O.ccf(F[rows].astype(np.float64), c.star, c.mask_lambda, c.mask_weight, c.mask_width_kms, lo, step, nv)
    _, ccf_g = _tc_ccf(S, c, F, c.mask_width_kms, lo, step, nv)
    assert np.abs(ccf_g[rows] - ccf_o).max() <= TOL_CCF * np.abs(ccf_o).max()


def test_ccf_tc_dense_mask_stretch(S):
    """1,200 extra lines packed 0.08 px apart: more than 512 lines reach one 64-pixel block, so
    the mask-matrix builder reads the lines past its shared-memory window directly."""
    c = synth.config1(0)
    lo, step, nv = synth.velocity_grid(c.star.vsini_kms)
    st = c.star
    delta = np.log(st.lambda_end_A / st.lambda_start_A) / (st.n_px - 1)
    u = 2000.0 + 0.08 * np.arange(1200)
    extra = st.lambda_start_A * np.exp(u * delta)
    rng = np.random.default_rng(11)
    lam = np.concatenate([c.mask_lambda, extra])
    w = np.concatenate([c.mask_weight, rng.uniform(0.1, 1.0, extra.size)])
    order = np.argsort(lam, kind="stable")
    c.mask_lambda, c.mask_weight = lam[order].copy(), w[order].copy()
    F = _spectra(c, 6)
    ccf_o = O.ccf(F.astype(np.float64), c.star, c.mask_lambda, c.mask_weight, c.mask_width_kms, lo, step, nv)
    _, ccf_g = _tc_ccf(S, c, F, c.mask_width_kms, lo, step, nv)
    _, ccf_s = _tc_ccf(S, c, F, c.mask_width_kms, lo, step, nv, tensor_cores=False)
    assert np.abs(ccf_s - ccf_o).max() <= 2e-6 * np.abs(ccf_o).max()
    assert np.abs(ccf_g - ccf_o).max() <= TOL_CCF * np.abs(ccf_o).max()


def test_rv_ccf_rejects_unknown_spectra_type(S):
    """spectra_f32 outside 0, 1, 2 is SOAP_EINVAL before any device work."""
    import ctypes
    c = synth.config1(0)
    lo, step, nv = synth.velocity_grid(c.star.vsini_kms)
    F = _t(_spectra(c, 2))
    ml = np.ascontiguousarray(c.mask_lambda)
    mw = np.ascontiguousarray(c.mask_weight)
    with S.Disk(c.star, _t(c.quiet)) as d:
        rv = torch.empty(2, dtype=torch.float64, device=DEV)
        st = S._lib.soap_rv_ccf(d.ctx, ctypes.c_void_p(F.data_ptr()), 3, 2, 1, ctypes.c_void_p(ml.ctypes.data),
                                ctypes.c_void_p(mw.ctypes.data), ml.size, float(c.mask_width_kms), float(lo),
                                float(step), int(nv), ctypes.c_void_p(rv.data_ptr()), None, None, 1)
    assert st == S.SOAP_EINVAL


def test_ccf_tc_at_its_velocity_limit(S, cfg2):
    """256 velocities, the most the tensor-core form takes (N = 256, shared memory ~193 KiB),
    against the oracle; the mask-matrix tiles then fill the whole N range."""
    c = cfg2
    nv, step = 256, 0.2
    lo = -0.5 * step * (nv - 1)
    F = _spectra(c, 5)
    ccf_o = O.ccf(F.astype(np.float64), c.star, c.mask_lambda, c.mask_weight, c.mask_width_kms, lo, step, nv)
    _, ccf_g = _tc_ccf(S, c, F, c.mask_width_kms, lo, step, nv)
    assert np.isfinite(ccf_g).all()
    assert np.abs(ccf_g - ccf_o).max() <= TOL_CCF * np.abs(ccf_o).max()


def test_rv_ccf_reports_a_timed_out_wait_with_host_outputs(S):
    """A tensor-core wait that gave up is reported by soap_rv_ccf itself when its outputs are on
    the host (the status word is marked as the kernel would mark it; no kernel is made to wait),
    the status is cleared by that report, and the next call succeeds."""
    c = synth.config1(0)
    lo, step, nv = synth.velocity_grid(c.star.vsini_kms)
    F = _spectra(c, 3)
    with S.Disk(c.star, _t(c.quiet)) as d:
        rv = np.empty(3)
        S.soap_debug_inject_timeout(d.ctx)
        with pytest.raises(S.SoapError) as e:
            S.soap_rv_ccf(d.ctx, F, c.mask_lambda, c.mask_weight, c.mask_width_kms, lo, step, nv, rv,
                          tensor_cores=True)
        assert e.value.status == S.SOAP_ETIMEOUT
        assert "timeout 1" in str(e.value)
        S.soap_rv_ccf(d.ctx, F, c.mask_lambda, c.mask_weight, c.mask_width_kms, lo, step, nv, rv,
                      tensor_cores=True)
        assert np.isfinite(rv).all()


def test_device_outputs_report_a_timed_out_wait_at_synchronize(S):
    """With device outputs the call returns at once and soap_synchronize reports the timeout."""
    c = synth.config1(0)
    lo, step, nv = synth.velocity_grid(c.star.vsini_kms)
    F = _t(_spectra(c, 3))
    with S.Disk(c.star, _t(c.quiet)) as d:
        rv = torch.empty(3, dtype=torch.float64, device=DEV)
        S.soap_debug_inject_timeout(d.ctx)
        S.soap_rv_ccf(d.ctx, F, c.mask_lambda, c.mask_weight, c.mask_width_kms, lo, step, nv, rv,
                      tensor_cores=True)
        with pytest.raises(S.SoapError) as e:
            S.soap_synchronize(d.ctx)
        assert e.value.status == S.SOAP_ETIMEOUT
        S.soap_synchronize(d.ctx)
