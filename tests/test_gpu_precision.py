"""Precision study of the mixed path (config 1 over 10 seeds): the FP32 contraction with FP64
positions and FP64 RV fit against the FP64 oracle.  Bars: 2e-6 of max F_quiet in flux and
1 cm/s in RV; the FP64 path is held to 1e-12.  The measured errors are printed per seed."""
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


@pytest.mark.parametrize("seed", list(range(10)))
def test_mixed_precision_errors_config1(S, seed):
    c = synth.config1(seed)
    q = O.quiet(c.star, c.quiet)
    ref = O.active(c.star, c.quiet, c.active, c.regions, c.phases, effects=1)[0]
    lo, step, nv = synth.velocity_grid(c.star.vsini_kms)
    rv_ref = O.rv(ref, c.star, c.mask_lambda, c.mask_weight, c.mask_width_kms, lo, step, nv)[0]
    out = {}
    with S.Disk(c.star, _t(c.quiet), {k: _t(v) for k, v in c.active.items()}) as d:
        for prec, dt in ((S.SOAP_FP32, torch.float32), (S.SOAP_FP64, torch.float64)):
            spec = torch.empty((1, c.phases.size, c.star.n_px), dtype=dt, device=DEV)
            S.soap_active_phases(d.ctx, c.regions, c.phases, S.SOAP_EFFECT_TOT, prec, spec)
            rv = torch.empty(c.phases.size, dtype=torch.float64, device=DEV)
            S.soap_rv_ccf(d.ctx, spec[0], c.mask_lambda, c.mask_weight, c.mask_width_kms, lo, step, nv, rv)
            torch.cuda.synchronize()
            out[prec] = (spec[0].double().cpu().numpy(), rv.cpu().numpy())
    f32, rv32 = out[S.SOAP_FP32]
    f64, rv64 = out[S.SOAP_FP64]
    e32 = np.abs(f32 - ref).max() / q.max()
    e64 = np.abs(f64 - ref).max() / q.max()
    r32 = np.abs(rv32 - rv_ref).max() * 1e5
    r64 = np.abs(rv64 - rv_ref).max() * 1e5
    print(f"seed {seed}: flux FP32 {e32:.2e} FP64 {e64:.2e}; RV FP32 {r32:.4f} cm/s FP64 {r64:.2e} cm/s")
    assert e32 <= 2e-6 and r32 <= 1.0
    assert e64 <= 1e-12 and r64 <= 1e-6
