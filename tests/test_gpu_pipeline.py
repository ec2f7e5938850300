"""The fused spectra + RV call and the host-transfer pipeline.

soap_active_rv runs the same kernels as soap_active_phases followed by soap_rv_ccf, so its
results are compared bit for bit with those two calls.  With the host-transfer pipeline on,
uploads, compute and downloads of successive steps overlap; every step's results must still
equal those of the same step run alone, including when the host sources are overwritten by the
caller only after synchronising and when one host output buffer is reused by every step.
"""
import numpy as np
import pytest

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
def case():
    return synth.config1(0)


def _t(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def _pinned(a):
    return torch.from_numpy(np.ascontiguousarray(a)).pin_memory()


def _grid(c):
    return synth.velocity_grid(c.star.vsini_kms)


def _separate(S, c, quiet, active, phases, prec, effect):
    """Spectra and RVs from soap_active_phases + soap_rv_ccf (device outputs)."""
    lo, step, nv = _grid(c)
    dt = torch.float32 if prec == S.SOAP_FP32 else torch.float64
    with S.Disk(c.star, _t(quiet), {S.SOAP_SPOT: _t(active)}) as d:
        spec = torch.empty((1, len(phases), c.star.n_px), dtype=dt, device=DEV)
        S.soap_active_phases(d.ctx, c.regions, phases, effect, prec, spec)
        rv = torch.empty(len(phases), dtype=torch.float64, device=DEV)
        S.soap_rv_ccf(d.ctx, spec[0], c.mask_lambda, c.mask_weight, c.mask_width_kms, lo, step, nv, rv)
        torch.cuda.synchronize()
    return spec[0].cpu().numpy(), rv.cpu().numpy()


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
@pytest.mark.parametrize("effect", ["tot", "flux", "bconv"])
def test_active_rv_equals_active_phases_then_rv_ccf(S, case, prec, effect):
    c = case
    p = {"fp32": S.SOAP_FP32, "fp64": S.SOAP_FP64}[prec]
    e = {"tot": S.SOAP_EFFECT_TOT, "flux": S.SOAP_EFFECT_FLUX, "bconv": S.SOAP_EFFECT_BCONV}[effect]
    lo, step, nv = _grid(c)
    spec_ref, rv_ref = _separate(S, c, c.quiet, c.active[synth.SPOT], c.phases, p, e)
    dt = torch.float32 if p == S.SOAP_FP32 else torch.float64
    with S.Disk(c.star, _t(c.quiet), {S.SOAP_SPOT: _t(c.active[synth.SPOT])}) as d:
        # device outputs
        spec_d = torch.empty((len(c.phases), c.star.n_px), dtype=dt, device=DEV)
        rv_d = torch.empty(len(c.phases), dtype=torch.float64, device=DEV)
        S.soap_active_rv(d.ctx, c.regions, c.phases, e, p, c.mask_lambda, c.mask_weight,
                         c.mask_width_kms, lo, step, nv, spec_d, rv_d)
        # host outputs (returns with the copies done), and RVs only
        spec_h = torch.empty((len(c.phases), c.star.n_px), dtype=dt).pin_memory()
        rv_h = np.empty(len(c.phases))
        S.soap_active_rv(d.ctx, c.regions, c.phases, e, p, c.mask_lambda, c.mask_weight,
                         c.mask_width_kms, lo, step, nv, spec_h, rv_h)
        rv_only = np.empty(len(c.phases))
        S.soap_active_rv(d.ctx, c.regions, c.phases, e, p, c.mask_lambda, c.mask_weight,
                         c.mask_width_kms, lo, step, nv, None, rv_only)
        torch.cuda.synchronize()
    np.testing.assert_array_equal(spec_d.cpu().numpy(), spec_ref)
    np.testing.assert_array_equal(rv_d.cpu().numpy(), rv_ref)
    np.testing.assert_array_equal(spec_h.numpy(), spec_ref)
    np.testing.assert_array_equal(rv_h, rv_ref)
    np.testing.assert_array_equal(rv_only, rv_ref)


def test_active_rv_rejects_two_effects(S, case):
    c = case
    lo, step, nv = _grid(c)
    with S.Disk(c.star, _t(c.quiet), {S.SOAP_SPOT: _t(c.active[synth.SPOT])}) as d:
        with pytest.raises(S.SoapError):
            S.soap_active_rv(d.ctx, c.regions, c.phases, S.SOAP_EFFECT_TOT | S.SOAP_EFFECT_FLUX,
                             S.SOAP_FP32, c.mask_lambda, c.mask_weight, c.mask_width_kms, lo, step,
                             nv, None, np.empty(len(c.phases)))


def _steps(c):
    """Three steps with their own local spectra and phases."""
    out = []
    for k in range(3):
        quiet = c.quiet * (1.0 + 0.01 * k)
        active = c.active[synth.SPOT] * (1.0 - 0.02 * k)
        phases = c.phases[k::2] if k < 2 else c.phases[::-1]
        out.append((quiet, active, phases))
    return out


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_host_async_pipeline_matches_each_step_alone(S, case, prec):
    c = case
    p = {"fp32": S.SOAP_FP32, "fp64": S.SOAP_FP64}[prec]
    dt = torch.float32 if p == S.SOAP_FP32 else torch.float64
    lo, step, nv = _grid(c)
    steps = _steps(c)
    refs = [_separate(S, c, q, a, ph, p, S.SOAP_EFFECT_TOT) for q, a, ph in steps]
    with S.Disk(c.star, _t(c.quiet), {S.SOAP_SPOT: _t(c.active[synth.SPOT])}) as d:
        S.soap_set_host_async(d.ctx, True)
        q_h = [_pinned(q) for q, _, _ in steps]
        a_h = [_pinned(a) for _, a, _ in steps]
        spec_h = [torch.empty((len(ph), c.star.n_px), dtype=dt).pin_memory() for _, _, ph in steps]
        rv_h = [torch.empty(len(ph), dtype=torch.float64).pin_memory() for _, _, ph in steps]
        shared_spec = torch.empty((len(c.phases), c.star.n_px), dtype=dt).pin_memory()
        shared_rv = torch.empty(len(c.phases), dtype=torch.float64).pin_memory()
        for rep in range(2):                      # the second round reuses stages and buffers
            for k, (_, _, ph) in enumerate(steps):
                S.soap_update_star(d.ctx, c.star)
                S.soap_set_quiet_spectrum(d.ctx, q_h[k])
                S.soap_set_active_spectrum(d.ctx, S.SOAP_SPOT, a_h[k])
                S.soap_active_rv(d.ctx, c.regions, ph, S.SOAP_EFFECT_TOT, p, c.mask_lambda,
                                 c.mask_weight, c.mask_width_kms, lo, step, nv, spec_h[k], rv_h[k])
            # one host output reused by every step: it ends with the last step's results
            for k, (_, _, ph) in enumerate(steps):
                S.soap_set_quiet_spectrum(d.ctx, q_h[k])
                S.soap_set_active_spectrum(d.ctx, S.SOAP_SPOT, a_h[k])
                n = len(ph)
                S.soap_active_rv(d.ctx, c.regions, ph, S.SOAP_EFFECT_TOT, p, c.mask_lambda,
                                 c.mask_weight, c.mask_width_kms, lo, step, nv, shared_spec[:n],
                                 shared_rv[:n])
            S.soap_synchronize(d.ctx)
            for k in range(3):
                np.testing.assert_array_equal(spec_h[k].numpy(), refs[k][0])
                np.testing.assert_array_equal(rv_h[k].numpy(), refs[k][1])
            n = len(steps[-1][2])
            np.testing.assert_array_equal(shared_spec[:n].numpy(), refs[-1][0])
            np.testing.assert_array_equal(shared_rv[:n].numpy(), refs[-1][1])
            for t in spec_h + rv_h + [shared_spec, shared_rv]:
                t.fill_(float("nan"))
        S.soap_set_host_async(d.ctx, False)


def test_ccf_tables_follow_mask_and_velocity_changes(S, case):
    """The context keeps its CCF line and velocity tables while the mask, its width and the
    velocity grid stay the same: alternating masks, widths and grids on one context must give
    what a fresh context gives for each."""
    c = case
    lo, step, nv = _grid(c)
    rng = np.random.default_rng(11)
    keep = np.sort(rng.choice(c.mask_lambda.size, c.mask_lambda.size // 2, replace=False))
    masks = [(c.mask_lambda, c.mask_weight, c.mask_width_kms, lo, step, nv),
             (c.mask_lambda[keep].copy(), c.mask_weight[keep].copy(), c.mask_width_kms, lo, step, nv),
             (c.mask_lambda, c.mask_weight * 1.5, c.mask_width_kms, lo, step, nv),
             (c.mask_lambda, c.mask_weight, c.mask_width_kms * 0.8, lo, step, nv),
             (c.mask_lambda, c.mask_weight, c.mask_width_kms, lo + 1.0, step, nv - 8),
             (c.mask_lambda, c.mask_weight, c.mask_width_kms, lo, step, nv)]
    F = _t(c.quiet[:5].astype(np.float32))

    def rv_of(ctx, m):
        ml, mw, w, l0, st, n = m
        rv = torch.empty(F.shape[0], dtype=torch.float64, device=DEV)
        ccf = torch.empty((F.shape[0], n), dtype=torch.float64, device=DEV)
        S.soap_rv_ccf(ctx, F, ml, mw, w, l0, st, n, rv, None, ccf)
        torch.cuda.synchronize()
        return rv.cpu().numpy(), ccf.cpu().numpy()

    fresh = []
    for m in masks:
        with S.Disk(c.star, _t(c.quiet)) as d:
            fresh.append(rv_of(d.ctx, m))
    with S.Disk(c.star, _t(c.quiet)) as d:
        for rep in range(2):
            for m, (rv_f, ccf_f) in zip(masks, fresh):
                rv, ccf = rv_of(d.ctx, m)
                np.testing.assert_array_equal(ccf, ccf_f)
                np.testing.assert_array_equal(rv, rv_f)


def test_float32_local_spectra_give_the_fp32_path_its_own_results(S, case):
    """float32 local spectra (host or device, pipelined or not) give the SOAP_FP32 path exactly
    the results of the float64 ones, which that path rounds to float32 anyway; the FP64 path
    refuses to run on them until float64 spectra are set again."""
    c = case
    lo, step, nv = _grid(c)
    q32, a32 = c.quiet.astype(np.float32), c.active[synth.SPOT].astype(np.float32)
    spec_ref, rv_ref = _separate(S, c, c.quiet, c.active[synth.SPOT], c.phases, S.SOAP_FP32,
                                 S.SOAP_EFFECT_TOT)
    with S.Disk(c.star, _t(c.quiet), {S.SOAP_SPOT: _t(c.active[synth.SPOT])}) as d:
        for src, pipelined in ((lambda a: _t(a), False), (_pinned, False), (_pinned, True)):
            S.soap_set_host_async(d.ctx, pipelined)
            S.soap_set_quiet_spectrum(d.ctx, src(q32))
            S.soap_set_active_spectrum(d.ctx, S.SOAP_SPOT, src(a32))
            spec = torch.empty((len(c.phases), c.star.n_px), dtype=torch.float32).pin_memory()
            rv = torch.empty(len(c.phases), dtype=torch.float64).pin_memory()
            S.soap_active_rv(d.ctx, c.regions, c.phases, S.SOAP_EFFECT_TOT, S.SOAP_FP32, c.mask_lambda,
                             c.mask_weight, c.mask_width_kms, lo, step, nv, spec, rv)
            S.soap_synchronize(d.ctx)
            np.testing.assert_array_equal(spec.numpy(), spec_ref)
            np.testing.assert_array_equal(rv.numpy(), rv_ref)
        S.soap_set_host_async(d.ctx, False)
        out64 = torch.empty((1, len(c.phases), c.star.n_px), dtype=torch.float64, device=DEV)
        with pytest.raises(S.SoapError):
            S.soap_active_phases(d.ctx, c.regions, c.phases, S.SOAP_EFFECT_TOT, S.SOAP_FP64, out64)
        with pytest.raises(S.SoapError):
            S.soap_quiet_spectrum(d.ctx, S.SOAP_FORM_TOEPLITZ, S.SOAP_FP64,
                                  torch.empty(c.star.n_px, dtype=torch.float64, device=DEV))
        S.soap_set_quiet_spectrum(d.ctx, _t(c.quiet))
        with pytest.raises(S.SoapError):                  # the spot spectrum is still float32
            S.soap_active_phases(d.ctx, c.regions, c.phases, S.SOAP_EFFECT_TOT, S.SOAP_FP64, out64)
        S.soap_set_active_spectrum(d.ctx, S.SOAP_SPOT, _t(c.active[synth.SPOT]))
        S.soap_active_phases(d.ctx, c.regions, c.phases, S.SOAP_EFFECT_TOT, S.SOAP_FP64, out64)
        torch.cuda.synchronize()
    ref64, _ = _separate(S, c, c.quiet, c.active[synth.SPOT], c.phases, S.SOAP_FP64, S.SOAP_EFFECT_TOT)
    np.testing.assert_array_equal(out64[0].cpu().numpy(), ref64)


@pytest.mark.parametrize("n_px", [20000, 20003])
def test_float32_rows_any_pixel_count(S, n_px):
    """float32 uploads pad their rows with 16-byte copies when the pixel count allows it (20,000)
    and element by element otherwise (20,003); either way the FP32 path gets the results of the
    float64 uploads, bit for bit (spot and facula spectra, all three effects)."""
    c = synth.config2(3, grid_n=60, n_px=n_px, lambda_start=5000.0, lambda_end=5300.0, n_phases=9)
    outs = []
    for dt in (np.float64, np.float32):
        with S.Disk(c.star, _t(c.quiet)) as d:
            S.soap_set_quiet_spectrum(d.ctx, _t(c.quiet.astype(dt)))
            for k, v in c.active.items():
                S.soap_set_active_spectrum(d.ctx, k, _t(v.astype(dt)))
            out = torch.empty((3, len(c.phases), n_px), dtype=torch.float32, device=DEV)
            S.soap_active_phases(d.ctx, c.regions, c.phases, 7, S.SOAP_FP32, out)
            torch.cuda.synchronize()
            outs.append(out.cpu().numpy())
    np.testing.assert_array_equal(outs[0], outs[1])
