"""Precision study (config 3: config 1 over 10 seeds) of the mixed forms against the FP64 oracle:
the FP32 contraction and the tensor-core BF16x3 contraction (hi/lo split, three products, FP32
accumulation), both with FP64 positions; their CCFs (FP32 SIMT / BF16x3 tensor cores) and FP32
fits.  Bars: 2e-6 of max F_quiet in flux and 1 cm/s in RV; the FP64 path is held to 1e-12 and
1e-6 cm/s.  The measured errors are printed per seed.  At full size (disk 300x300, 205,800 px,
100 phases) the RVs of every phase are held to the same bars against the oracle's RVs of its own
full-size spectra (tests/golden/cfg2_fullsize_oracle.json)."""
import json
from pathlib import Path

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
        for prec, dt in ((S.SOAP_FP32, torch.float32), (S.SOAP_BF16X3, torch.float32),
                         (S.SOAP_FP64, torch.float64)):
            spec = torch.empty((1, c.phases.size, c.star.n_px), dtype=dt, device=DEV)
            S.soap_active_phases(d.ctx, c.regions, c.phases, S.SOAP_EFFECT_TOT, prec, spec)
            rv = torch.empty(c.phases.size, dtype=torch.float64, device=DEV)
            S.soap_rv_ccf(d.ctx, spec[0], c.mask_lambda, c.mask_weight, c.mask_width_kms, lo, step, nv, rv,
                          tensor_cores=prec == S.SOAP_BF16X3)
            torch.cuda.synchronize()
            out[prec] = (spec[0].double().cpu().numpy(), rv.cpu().numpy())
    err = {}
    for prec, (f, rv) in out.items():
        err[prec] = (np.abs(f - ref).max() / q.max(), np.abs(rv - rv_ref).max() * 1e5)
    (e32, r32), (ebf, rbf), (e64, r64) = err[S.SOAP_FP32], err[S.SOAP_BF16X3], err[S.SOAP_FP64]
    print(f"seed {seed}: flux FP32 {e32:.2e} BF16x3 {ebf:.2e} FP64 {e64:.2e}; "
          f"RV FP32 {r32:.4f} BF16x3 {rbf:.4f} cm/s FP64 {r64:.2e} cm/s")
    assert e32 <= 2e-6 and r32 <= 1.0
    assert ebf <= 2e-6 and rbf <= 1.0
    assert e64 <= 1e-12 and r64 <= 1e-6


GOLDEN = Path(__file__).resolve().parent / "golden" / "cfg2_fullsize_oracle.json"


def test_fullsize_rvs_against_the_oracle():
    """The full-size active star (synth.config2(0): disk 300x300, 205,800 px, 20 mu bins, facula +
    2 spots, 100 phases) through soap_active_rv at every precision, and at SOAP_FP32 with the CCF
    on the tensor cores (soap_set_ccf_tensor_cores): all 100 RVs against the oracle's RVs of its
    own FP64 spectra, and sampled spectrum values against the oracle's.  The option leaves the
    FP32 spectra unchanged, bit for bit."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_2301_04259_gb300 import soap as S
    g = json.loads(GOLDEN.read_text())
    c = synth.config2(g["seed"])
    assert c.star.n_px == g["n_px"] and c.phases.size == g["n_phases"]
    ref = np.asarray(g["rv_kms"])
    sp = np.asarray(g["samples"]["phase_index"])
    px = np.asarray(g["samples"]["pixel"])
    F_ref = np.asarray(g["samples"]["F"])
    lo, step, nv = g["v_lo"], g["v_step"], g["n_v"]
    with S.Disk(c.star, _t(c.quiet), {k: _t(v) for k, v in c.active.items()}) as d:
        qf = torch.empty(c.star.n_px, dtype=torch.float64, device=DEV)
        S.soap_quiet_spectrum(d.ctx, S.SOAP_FORM_TOEPLITZ, S.SOAP_FP64, qf)
        torch.cuda.synchronize()
        scale = float(qf.max())
        spectra = {}
        for prec, dt, tol_f, tol_rv, tc in ((S.SOAP_FP64, torch.float64, 1e-12, 1e-6, False),
                                            (S.SOAP_FP32, torch.float32, 2e-6, 1.0, False),
                                            (S.SOAP_FP32, torch.float32, 2e-6, 1.0, True),
                                            (S.SOAP_BF16X3, torch.float32, 2e-6, 1.0, False)):
            spec = torch.empty((c.phases.size, c.star.n_px), dtype=dt, device=DEV)
            rv = torch.empty(c.phases.size, dtype=torch.float64, device=DEV)
            S.soap_set_ccf_tensor_cores(d.ctx, tc)
            S.soap_active_rv(d.ctx, c.regions, c.phases, S.SOAP_EFFECT_TOT, prec, c.mask_lambda, c.mask_weight,
                             c.mask_width_kms, lo, step, nv, spec, rv)
            S.soap_set_ccf_tensor_cores(d.ctx, False)
            torch.cuda.synchronize()
            spectra[(prec, tc)] = spec
            r = rv.cpu().numpy()
            e_rv = np.abs(r - ref).max() * 1e5
            e_f = np.abs(spec[torch.from_numpy(sp).to(DEV), torch.from_numpy(px).to(DEV)].double().cpu().numpy()
                         - F_ref).max() / scale
            print(f"precision {prec} (tensor-core CCF {tc}): RV max err {e_rv:.3e} cm/s, sampled flux err {e_f:.2e}")
            assert np.isfinite(r).all()
            assert e_rv <= tol_rv, (prec, tc, e_rv)
            assert e_f <= tol_f, (prec, tc, e_f)
        assert torch.equal(spectra[(S.SOAP_FP32, True)], spectra[(S.SOAP_FP32, False)])
