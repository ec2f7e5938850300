"""Bisector injection (Sect. 4.3, Convec.model): the library against the oracle, element by
element (FP64, 1e-12 of max |F|), on the small and the full-size local spectra, host and device,
with and without an original bisector to remove; non-increasing moved positions are refused;
injected spectra feed the disk integration like any local spectra."""
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


def _delta(star):
    return O.delta(star.lambda_start_A, star.lambda_end_A, star.n_px)


def _tables(n_rows, n_d, scale, seed):
    """C-shaped synthetic bisectors per row: v(d) = a + b d + c d^2 (km/s), |v| <= ~scale."""
    rng = np.random.default_rng(seed)
    d = np.linspace(0.0, 1.0, n_d)
    a, b, c = (rng.uniform(-1, 1, (3, n_rows, 1)) * np.array([0.3, 1.0, 1.0])[:, None, None]) * scale
    return a + b * d + c * d * d


@pytest.mark.parametrize("with_orig", [False, True])
@pytest.mark.parametrize("n_d", [2, 11, 101])
def test_bisector_injection_matches_oracle(S, with_orig, n_d):
    c = synth.config1(0)
    F = c.quiet
    bis = _tables(F.shape[0], n_d, 0.25, 1)
    orig = _tables(1, n_d, 0.1, 2)[0] if with_orig else np.zeros(n_d)
    ref = O.inject_bisectors(F, bis, orig, _delta(c.star))
    with S.Disk(c.star, _t(F)) as d:
        out = torch.empty(F.shape, dtype=torch.float64, device=DEV)
        S.soap_inject_bisectors(d.ctx, _t(F), out, bis, orig)
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        host = np.empty_like(F)
        S.soap_inject_bisectors(d.ctx, F, host, bis, orig)
    assert np.abs(got - ref).max() <= 1e-12 * np.abs(ref).max()
    np.testing.assert_array_equal(host, got)


def _star(n_px, lam0, lam1):
    c = synth.config1(0)
    st = c.star
    st.n_px = n_px
    st.lambda_start_A, st.lambda_end_A = lam0, lam1
    lam = synth.wavelength_grid(lam0, lam1, n_px)
    rng = np.random.default_rng(n_px)
    q = synth.local_spectra(lam, rng.uniform(lam0, lam1, 20), rng.uniform(0.1, 0.8, 20),
                            rng.uniform(0.005, 0.05, 20) * (lam1 - lam0) / 10.0, st.mu_values)
    return st, q


@pytest.mark.parametrize("n_px,lam0,lam1", [(4096, 6000.0, 6010.0), (100, 5000.0, 5100.0), (64, 5000.0, 6000.0)])
def test_bisector_injection_across_grid_spacings(S, n_px, lam0, lam1):
    """Fine, medium and coarse log grids (Delta 4e-7, 2e-4, 3e-3): the three expm1 forms of the
    kernel (series to e^4, series to e^6, library function) against the oracle."""
    st, q = _star(n_px, lam0, lam1)
    bis = _tables(q.shape[0], 21, 0.3, 5)
    orig = _tables(1, 21, 0.1, 6)[0]
    ref = O.inject_bisectors(q, bis, orig, _delta(st))
    with S.Disk(st, _t(q)) as d:
        out = torch.empty(q.shape, dtype=torch.float64, device=DEV)
        S.soap_inject_bisectors(d.ctx, _t(q), out, bis, orig)
        torch.cuda.synchronize()
    assert np.abs(out.cpu().numpy() - ref).max() <= 1e-12 * np.abs(ref).max()


def test_bisector_injection_full_size(S):
    """The 20 mu rows of the full-size quiet and active local spectra (205,800 px)."""
    c = synth.config2(0)
    for F in (c.quiet, c.active[synth.SPOT]):
        bis = _tables(F.shape[0], 51, 0.3, 3)
        ref = O.inject_bisectors(F, bis, np.zeros(51), _delta(c.star))
        with S.Disk(c.star, _t(c.quiet)) as d:
            out = torch.empty(F.shape, dtype=torch.float64, device=DEV)
            S.soap_inject_bisectors(d.ctx, _t(F), out, bis, np.zeros(51))
            torch.cuda.synchronize()
        assert np.abs(out.cpu().numpy() - ref).max() <= 1e-12 * np.abs(ref).max()


def test_non_increasing_positions_are_refused(S):
    """A bisector steep enough to move neighbouring wing points past each other: the oracle
    refuses it, and so does the library (device flag, SOAP_ERANGE)."""
    c = synth.config1(0)
    F = c.quiet
    d = np.linspace(0.0, 1.0, 11)
    bis = np.tile(6.0 * d, (F.shape[0], 1))                 # 6 km/s over the depth range
    with pytest.raises(ValueError):
        O.inject_bisectors(F, bis, np.zeros(11), _delta(c.star))
    with S.Disk(c.star, _t(F)) as dctx:
        out = torch.empty(F.shape, dtype=torch.float64, device=DEV)
        with pytest.raises(S.SoapError):
            S.soap_inject_bisectors(dctx.ctx, _t(F), out, bis, np.zeros(11))


def test_injected_spectra_integrate_like_any_local_spectra(S):
    """Quiet star from injected local spectra: the library's integral of its own injected rows
    against the oracle's integral of the oracle's injected rows."""
    c = synth.config1(0)
    bis = _tables(c.quiet.shape[0], 21, 0.2, 4)
    inj = O.inject_bisectors(c.quiet, bis, np.zeros(21), _delta(c.star))
    ref = O.quiet(c.star, inj)
    with S.Disk(c.star, _t(c.quiet)) as d:
        rows = torch.empty(c.quiet.shape, dtype=torch.float64, device=DEV)
        S.soap_inject_bisectors(d.ctx, _t(c.quiet), rows, bis, np.zeros(21))
        S.soap_set_quiet_spectrum(d.ctx, rows)
        q = torch.empty(c.star.n_px, dtype=torch.float64, device=DEV)
        S.soap_quiet_spectrum(d.ctx, S.SOAP_FORM_TOEPLITZ, S.SOAP_FP64, q)
        torch.cuda.synchronize()
    assert np.abs(q.cpu().numpy() - ref).max() <= 1e-12 * np.abs(ref).max()
