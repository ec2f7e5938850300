"""GPU parity of the batched form (soap_active_batch) through the C-ABI.

Each configuration of a batch is a star of the context's type with its own vsini,
inclination, regions and phases; its rows must equal the oracle's TOT spectra (Alg. 5,
Eqs. 3-4) for that star within the mixed-path tolerance, 2e-6 of max F_quiet.
"""
import dataclasses

import numpy as np
import pytest

from oracle import oracle as O
from paper_2301_04259_gb300 import synth
from paper_2301_04259_gb300.synth import FACULA, SPOT, Region

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL32 = 2e-6
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


@pytest.fixture(scope="module")
def small():
    """Disk 50x50, 4096 px, 11 mu; star vsini 10 km/s bounds the items' vsini."""
    c = synth.config1(3)
    c.star = dataclasses.replace(c.star, vsini_kms=10.0)
    fac = 0.6 * c.active[SPOT] + 0.4 * c.quiet          # a facula spectrum of its own
    c.active = {SPOT: c.active[SPOT], FACULA: fac}
    return c


def _small_batch():
    """Configurations covering: no region, one spot, overlapping spots, a facula with a spot
    inside (list order decides), two temperatures, far-side caps, vsini sign and extremes,
    pole-on and edge-on views, one phase, phases beyond one rotation."""
    cfgs = [
        synth.BatchConfig(2.0, 90.0, [], 3),
        synth.BatchConfig(10.0, 90.0, [Region(SPOT, 20.0, 0.0, 0.1, 4800.0)], 5),
        synth.BatchConfig(-4.0, 60.0, [Region(SPOT, 10.0, 30.0, 0.15, 4800.0),
                                       Region(SPOT, 15.0, 40.0, 0.12, 4800.0)], 4),
        synth.BatchConfig(6.5, 45.0, [Region(FACULA, -20.0, 10.0, 0.2, 6100.0),
                                      Region(SPOT, -20.0, 10.0, 0.08, 4800.0)], 7),
        synth.BatchConfig(3.0, 30.0, [Region(SPOT, 50.0, 200.0, 0.05, 4300.0),
                                      Region(SPOT, -55.0, 90.0, 0.2, 4800.0),
                                      Region(FACULA, 0.0, 180.0, 0.1, 6100.0)], 9),
        synth.BatchConfig(1.0, 0.0, [Region(SPOT, 70.0, 0.0, 0.2, 4800.0)], 1),
        synth.BatchConfig(9.9, 180.0, [Region(SPOT, -10.0, 300.0, 0.01, 4800.0)], 2),
        synth.BatchConfig(0.0, 90.0, [Region(SPOT, 0.0, 0.0, 0.3, 4800.0)], 3),
    ]
    items, regions, phases = synth.batch_layout(cfgs)
    phases = phases.copy()
    phases[-1] = 1.37                                   # outside [0, 1)
    return cfgs, items, regions, phases


def _oracle_rows(case, cfg, phases):
    star = dataclasses.replace(case.star, vsini_kms=cfg.vsini_kms, incl_deg=cfg.incl_deg)
    return O.active(star, case.quiet, case.active, cfg.regions, phases, effects=1)[0]


def _disk(S, case):
    return S.Disk(case.star, _t(case.quiet), {k: _t(v) for k, v in case.active.items()})


def test_batch_matches_oracle_per_configuration(S, small):
    cfgs, items, regions, phases = _small_batch()
    with _disk(S, small) as d:
        out = torch.empty((phases.size, small.star.n_px), dtype=torch.float32, device=DEV)
        S.soap_active_batch(d.ctx, items, regions, phases, out)
        S.soap_synchronize(d.ctx)
        g = out.double().cpu().numpy()
    scale = O.quiet(small.star, small.quiet).max()
    for cfg, it in zip(cfgs, items):
        fp, n = it[4], it[5]
        ref = _oracle_rows(small, cfg, phases[fp:fp + n])
        err = np.abs(g[fp:fp + n] - ref).max() / scale
        assert err <= TOL32, (cfg, err)


def _oracle_batch_rvs(case, cfg, F, lo, step, nv, margin=20.0):
    """RVs of oracle spectra F [n, n_px] the way the batched form defines them: the CCF on the
    common velocity grid (line validity from that grid, Sect. 4.1), the least-squares Gaussian
    fitted at the grid velocities with |v| <= |vsini| + margin."""
    C = O.ccf(F, case.star, case.mask_lambda, case.mask_weight, case.mask_width_kms, lo, step, nv)
    v = lo + step * np.arange(nv)
    H = abs(cfg.vsini_kms) + margin
    k0 = max(0, int(np.ceil((-H - lo) / step - 1e-9)))
    k1 = min(nv - 1, int(np.floor((H - lo) / step + 1e-9)))
    return np.array([O.fit_gaussian(v[k0:k1 + 1], row[k0:k1 + 1])[2] for row in C])


@pytest.mark.parametrize("tensor_cores", [False, True])
def test_batch_rvs_match_oracle_per_configuration(S, small, tensor_cores):
    """soap_active_batch with rv_kms: each phase's RV (CCF on the common grid -30..30 km/s, fit in
    its configuration's window |v| <= |vsini| + 20 km/s) against the oracle's spectra, CCF and
    fit within the mixed path's 1 cm/s; the spectra are unchanged by asking for RVs."""
    cfgs, items, regions, phases = _small_batch()
    lo, step, nv = synth.velocity_grid(10.0)
    with _disk(S, small) as d:
        S.soap_batch_set_rv(d.ctx, small.mask_lambda, small.mask_weight, small.mask_width_kms, lo, step, nv,
                            fit_margin_kms=20.0, tensor_cores=tensor_cores)
        out = torch.empty((phases.size, small.star.n_px), dtype=torch.float32, device=DEV)
        rv = torch.full((phases.size,), float("nan"), dtype=torch.float64, device=DEV)
        S.soap_active_batch(d.ctx, items, regions, phases, out, rv_out=rv)
        plain = torch.empty_like(out)
        S.soap_active_batch(d.ctx, items, regions, phases, plain)
        S.soap_synchronize(d.ctx)
        g = rv.cpu().numpy()
    assert torch.equal(out, plain)
    assert np.isfinite(g).all()
    for cfg, it in zip(cfgs, items):
        fp, n = it[4], it[5]
        ref = _oracle_batch_rvs(small, cfg, _oracle_rows(small, cfg, phases[fp:fp + n]), lo, step, nv)
        err_cms = np.abs(g[fp:fp + n] - ref).max() * 1e5
        assert err_cms <= 1.0, (cfg, err_cms)


def test_batch_rvs_host_output_whole_grid_and_errors(S, small):
    """Host outputs equal device outputs; fit_margin_kms <= 0 fits the whole grid (against the
    oracle); RVs need soap_batch_set_rv and the spectrum output."""
    cfgs, items, regions, phases = _small_batch()
    lo, step, nv = synth.velocity_grid(10.0)
    n_px = small.star.n_px
    with _disk(S, small) as d:
        out = torch.empty((phases.size, n_px), dtype=torch.float32, device=DEV)
        rv = torch.empty(phases.size, dtype=torch.float64, device=DEV)
        with pytest.raises(S.SoapError) as e:
            S.soap_active_batch(d.ctx, items, regions, phases, out, rv_out=rv)
        assert e.value.status == S.SOAP_ESTATE
        S.soap_batch_set_rv(d.ctx, small.mask_lambda, small.mask_weight, small.mask_width_kms, lo, step, nv,
                            fit_margin_kms=0.0)
        with pytest.raises(S.SoapError) as e:
            S.soap_active_batch(d.ctx, items, regions, phases, out, output=S.SOAP_BATCH_RESIDUAL, rv_out=rv)
        assert e.value.status == S.SOAP_EINVAL
        S.soap_active_batch(d.ctx, items, regions, phases, out, rv_out=rv)
        host = np.empty((phases.size, n_px), dtype=np.float32)
        rvh = np.empty(phases.size)
        S.soap_active_batch(d.ctx, items, regions, phases, host, rv_out=rvh)
        S.soap_synchronize(d.ctx)
        g = rv.cpu().numpy()
        S.soap_batch_set_rv(d.ctx, small.mask_lambda, small.mask_weight, small.mask_width_kms, lo, step, nv,
                            fit_margin_kms=0.1)                  # vsini 0 item: 0.1 km/s holds < 5 points
        with pytest.raises(S.SoapError) as e:
            S.soap_active_batch(d.ctx, items, regions, phases, out, rv_out=rv)
        assert e.value.status == S.SOAP_EINVAL
    assert np.array_equal(out.cpu().numpy(), host) and np.array_equal(g, rvh)
    for cfg, it in list(zip(cfgs, items))[1:4]:
        fp, n = it[4], it[5]
        ref = _oracle_batch_rvs(small, cfg, _oracle_rows(small, cfg, phases[fp:fp + n]), lo, step, nv,
                                margin=1e9)
        assert np.abs(g[fp:fp + n] - ref).max() * 1e5 <= 1.0, cfg


def test_batch_variants_agree_bitwise(S, small):
    """Phases per block only widens tap ranges with exact zeros and pixels per thread does not
    touch the arithmetic: every variant gives the same bits."""
    _, items, regions, phases = _small_batch()
    outs = []
    with _disk(S, small) as d:
        for v in range(S.soap_batch_num_variants()):
            S.soap_batch_set_variant(d.ctx, v)
            assert S.soap_batch_get_variant(d.ctx) == v
            out = torch.empty((phases.size, small.star.n_px), dtype=torch.float32, device=DEV)
            S.soap_active_batch(d.ctx, items, regions, phases, out)
            S.soap_synchronize(d.ctx)
            outs.append(out.cpu())
    for o in outs[1:]:
        assert torch.equal(o, outs[0])


def test_batch_graph_replay_sees_new_inputs(S, small):
    """Same shape, other values: the replayed graph must read the new items, regions and
    phases (and a repeat call must reproduce the first)."""
    cfgs, items, regions, phases = _small_batch()
    items_b = [(0.5 * v + 1.0, 90.0 - 0.5 * inc, fr, nr, fp, n) for (v, inc, fr, nr, fp, n) in items]
    regions_b = [Region(r.type, -r.lat_deg, r.lon_deg + 33.0, r.radius_rstar * 0.9, r.temp_K) for r in regions]
    phases_b = phases + 0.11
    n_px = small.star.n_px
    with _disk(S, small) as d:
        o1 = torch.empty((phases.size, n_px), dtype=torch.float32, device=DEV)
        o2 = torch.empty_like(o1)
        o3 = torch.empty_like(o1)
        S.soap_active_batch(d.ctx, items, regions, phases, o1)
        S.soap_active_batch(d.ctx, items_b, regions_b, phases_b, o2)
        S.soap_active_batch(d.ctx, items, regions, phases, o3)
        S.soap_synchronize(d.ctx)
    with _disk(S, small) as d:
        fresh = torch.empty_like(o1)
        S.soap_active_batch(d.ctx, items_b, regions_b, phases_b, fresh)
        S.soap_synchronize(d.ctx)
    assert torch.equal(o1, o3)
    assert torch.equal(o2, fresh)
    assert not torch.equal(o1, o2)


def test_batch_host_output_and_profiling_path(S, small):
    """Host output equals device output; the profiled (ungraphed) run gives the same bits and
    fills the contraction timer."""
    _, items, regions, phases = _small_batch()
    n_px = small.star.n_px
    with _disk(S, small) as d:
        dev = torch.empty((phases.size, n_px), dtype=torch.float32, device=DEV)
        S.soap_active_batch(d.ctx, items, regions, phases, dev)
        host = np.empty((phases.size, n_px), dtype=np.float32)
        S.soap_active_batch(d.ctx, items, regions, phases, host)
        S.soap_set_profiling(d.ctx, True)
        prof = torch.empty_like(dev)
        S.soap_active_batch(d.ctx, items, regions, phases, prof)
        S.soap_synchronize(d.ctx)
        ms, n = S.soap_get_kernel_time(d.ctx, S.SOAP_TIMER_CONTRACT)
        S.soap_set_profiling(d.ctx, False)
    assert np.array_equal(dev.cpu().numpy(), host)
    assert torch.equal(dev, prof)
    assert n >= 1 and ms > 0


def test_batch_matches_single_star_path(S):
    """Configurations drawn like the full batched workload (disk 150x150, 6000-6300 A at
    16,834 px): each item's rows against soap_active_phases (FP32) of that star."""
    case = synth.batch_spectra(0)
    cfgs = synth.batch_configs(1, 24)
    items, regions, phases = synth.batch_layout(cfgs)
    n_px = case.star.n_px
    with _disk(S, case) as d:
        out = torch.empty((phases.size, n_px), dtype=torch.float32, device=DEV)
        S.soap_active_batch(d.ctx, items, regions, phases, out)
        S.soap_synchronize(d.ctx)
        scale = S.soap_get_star_info(d.ctx).total_intensity * float(case.quiet.max())   # >= max F_q
    for cfg, it in zip(cfgs[:8], items[:8]):
        fp, n = it[4], it[5]
        star = dataclasses.replace(case.star, vsini_kms=cfg.vsini_kms, incl_deg=cfg.incl_deg)
        with S.Disk(star, _t(case.quiet), {k: _t(v) for k, v in case.active.items()}) as d1:
            ref = torch.empty((1, n, n_px), dtype=torch.float32, device=DEV)
            S.soap_active_phases(d1.ctx, cfg.regions, phases[fp:fp + n], 1, S.SOAP_FP32, ref)
            torch.cuda.synchronize()
        err = (out[fp:fp + n].double() - ref[0].double()).abs().max().item() / scale
        assert err <= 1e-6, (cfg, err)


def test_batch_fullsize_sampled_pixels(S):
    """The full batched workload (4096 configurations, disk 150x150, 16,834 px) in the launch
    configuration the benchmark times; sampled (configuration, phase, pixel) outputs against
    the oracle, every output finite."""
    case = synth.batch_spectra(0)
    cfgs = synth.batch_configs(1, 4096)
    items, regions, phases = synth.batch_layout(cfgs)
    n_px = case.star.n_px
    lo, step, nv = synth.velocity_grid(10.0)
    with _disk(S, case) as d:
        S.soap_batch_set_rv(d.ctx, case.mask_lambda, case.mask_weight, case.mask_width_kms, lo, step, nv,
                            fit_margin_kms=20.0)
        out = torch.empty((phases.size, n_px), dtype=torch.float32, device=DEV)
        rv = torch.empty(phases.size, dtype=torch.float64, device=DEV)
        S.soap_active_batch(d.ctx, items, regions, phases, out, rv_out=rv)
        S.soap_synchronize(d.ctx)
        assert bool(torch.isfinite(out).all())
        rvg = rv.cpu().numpy()
        assert np.isfinite(rvg).all()
        rng = np.random.default_rng(7)
        pick = sorted(set(rng.integers(0, len(cfgs), 6).tolist()) | {0, len(cfgs) - 1})
        pix = np.unique(np.concatenate([[0, 1, n_px - 2, n_px - 1], rng.integers(0, n_px, 24)]))
        qref = O.quiet(case.star, case.quiet, pix=pix)
        scale = qref.max()
        for k in pick:
            cfg, it = cfgs[k], items[k]
            fp, n = it[4], it[5]
            ph = np.unique(np.concatenate([[0, n - 1], rng.integers(0, n, 3)]))
            star = dataclasses.replace(case.star, vsini_kms=cfg.vsini_kms, incl_deg=cfg.incl_deg)
            ref = O.active(star, case.quiet, case.active, cfg.regions, phases[fp + ph], effects=1, pix=pix)[0]
            g = out[fp + torch.from_numpy(ph).to(DEV)][:, torch.from_numpy(pix).to(DEV)].double().cpu().numpy()
            err = np.abs(g - ref).max() / scale
            assert err <= TOL32, (k, err)
            if k in pick[:4]:
                # RVs of two phases of the configuration: the oracle's whole spectra, CCF and fit
                full = O.active(star, case.quiet, case.active, cfg.regions, phases[fp + ph[:2]], effects=1)[0]
                ref_rv = _oracle_batch_rvs(case, cfg, full, lo, step, nv)
                assert np.abs(rvg[fp + ph[:2]] - ref_rv).max() * 1e5 <= 1.0, k
        del out


def test_batch_errors(S, small):
    cfgs, items, regions, phases = _small_batch()
    n_px = small.star.n_px
    out = torch.empty((phases.size, n_px), dtype=torch.float32, device=DEV)
    with _disk(S, small) as d:
        bad = list(items)
        bad[1] = (10.5,) + tuple(bad[1][1:])                       # |vsini| above the star's
        with pytest.raises(S.SoapError) as e:
            S.soap_active_batch(d.ctx, bad, regions, phases, out)
        assert e.value.status == S.SOAP_EINVAL
        with pytest.raises(S.SoapError) as e:                     # last phase not covered
            S.soap_active_batch(d.ctx, items[:-1], regions, phases, out)
        assert e.value.status == S.SOAP_EINVAL
        dup = list(items)
        dup[0] = dup[0][:4] + (dup[1][4], dup[0][5])               # two items own one phase
        with pytest.raises(S.SoapError) as e:
            S.soap_active_batch(d.ctx, dup, regions, phases, out)
        assert e.value.status == S.SOAP_EINVAL
        with pytest.raises(S.SoapError) as e:
            S.soap_batch_set_variant(d.ctx, S.soap_batch_num_variants())
        assert e.value.status == S.SOAP_ERANGE
        many = [Region(SPOT, 0.0, 0.0, 0.1, 4000.0 + k) for k in range(S.SOAP_MAX_CLASSES + 1)]
        with pytest.raises(S.SoapError) as e:
            S.soap_active_batch(d.ctx, [(1.0, 90.0, 0, len(many), 0, 1)], many, np.zeros(1), out)
        assert e.value.status == S.SOAP_ERANGE
    rot = dataclasses.replace(small.star, diff_rot_alpha=0.1)
    with S.Disk(rot, _t(small.quiet), {k: _t(v) for k, v in small.active.items()}) as d:
        with pytest.raises(S.SoapError) as e:
            S.soap_active_batch(d.ctx, items, regions, phases, out)
        assert e.value.status == S.SOAP_EINVAL
    with S.Disk(small.star, _t(small.quiet)) as d:                 # no active spectrum
        with pytest.raises(S.SoapError) as e:
            S.soap_active_batch(d.ctx, items, regions, phases, out)
        assert e.value.status == S.SOAP_ESTATE


def test_batch_autotune_and_cache(S, small, tmp_path):
    from paper_2301_04259_gb300 import tuning
    _, items, regions, phases = _small_batch()
    out = torch.empty((phases.size, small.star.n_px), dtype=torch.float32, device=DEV)
    path = tmp_path / "tune.json"
    with _disk(S, small) as d:
        n0 = S.soap_get_launch_count(d.ctx)
        e1 = tuning.tune_batch(d.ctx, small.star, items, regions, phases, out, path=path, reps=2)
        assert e1["source"] == "autotune"
        assert 0 <= e1["variant"] < S.soap_batch_num_variants()
        assert S.soap_batch_get_variant(d.ctx) == e1["variant"]
        assert len(e1["ms"]) == S.soap_batch_num_variants() and min(e1["ms"]) > 0
        assert S.soap_get_launch_count(d.ctx) > n0
    with _disk(S, small) as d:
        e2 = tuning.tune_batch(d.ctx, small.star, items, regions, phases, out, path=path)
        assert e2["source"] == "cache" and e2["variant"] == e1["variant"]
        assert S.soap_batch_get_variant(d.ctx) == e1["variant"]


def test_batch_many_temperatures_and_residual_output(S, small):
    """More distinct (type, temperature) pairs over the batch than one item may hold: each item
    against the oracle; the residual output equals the spectrum minus the item's quiet star."""
    temps = np.linspace(3800.0, 5600.0, 12)
    cfgs = [synth.BatchConfig(2.0 + 0.5 * k, 40.0 + 4 * k,
                              [Region(FACULA, -15.0 + 3 * k, 20.0 * k, 0.18, 6000.0 + 10 * k),
                               Region(SPOT, -15.0 + 3 * k, 20.0 * k, 0.06 + 0.005 * k, t)], 2)
            for k, t in enumerate(temps)]
    items, regions, phases = synth.batch_layout(cfgs)
    quiet_items = [(v, inc, 0, 0, fp, n) for (v, inc, fr, nr, fp, n) in items]
    n_px = small.star.n_px
    with _disk(S, small) as d:
        spec = torch.empty((phases.size, n_px), dtype=torch.float32, device=DEV)
        res = torch.empty_like(spec)
        quiet = torch.empty_like(spec)
        S.soap_active_batch(d.ctx, items, regions, phases, spec, output=S.SOAP_BATCH_SPECTRUM)
        S.soap_active_batch(d.ctx, items, regions, phases, res, output=S.SOAP_BATCH_RESIDUAL)
        S.soap_active_batch(d.ctx, quiet_items, [], phases, quiet, output=S.SOAP_BATCH_SPECTRUM)
        S.soap_synchronize(d.ctx)
    g = spec.double().cpu().numpy()
    scale = O.quiet(small.star, small.quiet).max()
    for cfg, it in zip(cfgs, items):
        fp, n = it[4], it[5]
        ref = _oracle_rows(small, cfg, phases[fp:fp + n])
        assert np.abs(g[fp:fp + n] - ref).max() / scale <= TOL32, cfg
    diff = (spec.double() - quiet.double() - res.double()).abs().max().item() / scale
    assert diff <= 1e-6
    assert res.abs().max().item() > 1e-3 * scale                  # the regions do change the flux
