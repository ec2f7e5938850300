#!/usr/bin/env python
"""Benchmark of the stellar-disk integration (SOAP-GPU hot path, arXiv 2301.04259) on GB300.

Workload: disk 300x300, 3800-6900 A log-uniform at 3 px per R=115000 element (205,800 px),
20 mu bins, 20k-line synthetic spectra, 1 facula + 2 spots, 100 rotational phases.
One step = one pass of the whole path over one star: per-cell geometry and quiet velocity
kernels, local spectra into padded rows, quiet integral, contrast, InfoMap + per-phase
velocity kernels, Toeplitz contraction with Eqs. 1-4 (total effect) for the 100 phases,
CCF + Gaussian RV of the 100 spectra.  `value` = active-star spectra/s of the mixed path
(FP32 contraction, FP64 positions and fit), inputs resident in HBM; `e2e` = the same through
the C-ABI with host buffers (host->device inputs and device->host spectra + RVs inside the
timed region).  The FP64 path is timed too.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
Under torchrun each rank integrates its own star (weak scaling, no collective on the path).
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "active-star spectra/s (300^2 grid, 206k px) and RV error cm/s vs FP64"
UNIT = "spectra/s"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--grid", type=int, default=300)
    ap.add_argument("--n-px", type=int, default=205800)
    ap.add_argument("--cpu-sample-px", type=int, default=256)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the batched-form and surrogate measurements (N=1 only)")
    ap.add_argument("--batch-configs", type=int, default=4096)
    ap.add_argument("--sur-train", type=int, default=1_200_000)
    ap.add_argument("--sur-epochs", type=int, default=150)
    ap.add_argument("--sur-queries", type=int, default=1_000_000)
    ap.add_argument("--sur-err", type=int, default=196_608, help="queries the error network trains on")
    ap.add_argument("--sur-err-epochs", type=int, default=60)
    ap.add_argument("--only", default="all", choices=["all", "batched", "surrogate", "gemm", "quiet", "instrument", "bisectors",
                                                      "tensor"],
                    help="run one block alone (for profiling); 'all' is the full benchmark line")
    return ap.parse_args()


def dist():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def workload(args, rank):
    from paper_2301_04259_gb300 import synth
    if args.n_px == 205800 and args.grid == 300:
        case = synth.config2(args.seed + rank)
    else:
        l1 = 3800.0 * np.exp(np.log(6900.0 / 3800.0) * (args.n_px - 1) / 205799.0)
        case = synth.config2(args.seed + rank, grid_n=args.grid, n_px=args.n_px, lambda_end=l1)
    return case


# ------------------------------------------------------------------------------------------
# clocks during the timed region
# ------------------------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.f,
                stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        self.f.flush()
        rows = []
        with open(self.f.name) as fh:
            for line in fh:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    rows.append((float(parts[1]), float(parts[2]), parts[5:9]))
                except ValueError:
                    continue
        os.unlink(self.f.name)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"], "samples": 0}
        sm = [r[0] for r in rows]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[2][k].lower() == "active"})
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": max(r[1] for r in rows),
                "reasons": reasons, "samples": len(rows)}


# ------------------------------------------------------------------------------------------
# our arm
# ------------------------------------------------------------------------------------------
def run_ours(args):
    import torch
    rank, world, local = dist()
    if world > 1:
        import torch.distributed as tdist
        tdist.init_process_group(backend="nccl", device_id=torch.device(f"cuda:{local}"))
    torch.cuda.set_device(local)
    dev = torch.device(f"cuda:{local}")
    from paper_2301_04259_gb300 import soap as S
    from paper_2301_04259_gb300 import synth

    case = workload(args, rank)
    st = case.star
    P = case.phases.size
    n_px = st.n_px
    lo, vstep, nv = synth.velocity_grid(st.vsini_kms)
    stream = torch.cuda.current_stream()
    q_dev = torch.from_numpy(case.quiet).to(dev)
    a_dev = torch.from_numpy(case.active[synth.SPOT]).to(dev)
    out32 = torch.empty((1, P, n_px), dtype=torch.float32, device=dev)
    out64 = torch.empty((1, P, n_px), dtype=torch.float64, device=dev)
    rv32 = torch.empty(P, dtype=torch.float64, device=dev)
    rv64 = torch.empty(P, dtype=torch.float64, device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)   # > 129 MB L2
    ctx = S.soap_init_star(st, q_dev, stream=stream)
    S.soap_set_active_spectrum(ctx, S.SOAP_SPOT, a_dev)

    # the FP32 path reads float32 local spectra (bit-identical results to float64 ones rounded
    # by the library); the FP64 path gets float64 ones
    q_dev32, a_dev32 = q_dev.float(), a_dev.float()

    # the mixed path's CCF runs on the tensor cores (BF16 hi/lo split of spectra and line mask,
    # FP32 accumulation); tc=False times the same step with the FP32 SIMT CCF beside it
    def step(prec, out, rv, tc=False):
        f32 = prec == S.SOAP_FP32
        S.soap_update_star(ctx, st)
        S.soap_set_quiet_spectrum(ctx, q_dev32 if f32 else q_dev)
        S.soap_set_active_spectrum(ctx, S.SOAP_SPOT, a_dev32 if f32 else a_dev)
        S.soap_active_phases(ctx, case.regions, case.phases, S.SOAP_EFFECT_TOT, prec, out)
        S.soap_rv_ccf(ctx, out[0], case.mask_lambda, case.mask_weight, case.mask_width_kms,
                      lo, vstep, nv, rv, tensor_cores=tc)

    def barrier():
        if world > 1:
            import torch.distributed as tdist
            tdist.barrier()

    def timed(prec, out, rv, K, W, profile=False, tc=False):
        for _ in range(W):
            step(prec, out, rv, tc)
        torch.cuda.synchronize()
        S.soap_reset_kernel_times(ctx)
        S.soap_set_profiling(ctx, profile)
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(K)]
        barrier()
        torch.cuda.synchronize()
        l0 = S.soap_get_launch_count(ctx)
        for k in range(K):
            flush.fill_(k & 0xFF)                 # evict L2 between steps (not timed)
            ev[k][0].record(stream)
            step(prec, out, rv, tc)
            ev[k][1].record(stream)
        torch.cuda.synchronize()
        barrier()
        launches = S.soap_get_launch_count(ctx) - l0
        ms = float(np.mean([a.elapsed_time(b) for a, b in ev]))
        timers = {}
        if profile:
            for t, name in enumerate(S.TIMERS):
                tot, n = S.soap_get_kernel_time(ctx, t)
                timers[name] = (tot, n)
            S.soap_set_profiling(ctx, False)
        return ms, launches, timers

    K, W = args.steps, max(3, args.warmup)
    rv32s = torch.empty(P, dtype=torch.float64, device=dev)
    with ClockSampler(local) as clk:
        ms32, launches, timers = timed(S.SOAP_FP32, out32, rv32, K, W, profile=True, tc=True)
        ms32_plain, launches_plain, _ = timed(S.SOAP_FP32, out32, rv32, K, W, tc=True)
        _, _, timers_simt = timed(S.SOAP_FP32, out32, rv32s, K, W, profile=True)
        ms_simt, launches_simt, _ = timed(S.SOAP_FP32, out32, rv32s, K, W)
        K64 = max(3, K // 4)
    ms64, _, timers64 = timed(S.SOAP_FP64, out64, rv64, K64, 3, profile=True)
    clocks = clk.summary()
    ms_step = ms32_plain
    # max over ranks
    if world > 1:
        import torch.distributed as tdist
        t = torch.tensor([ms_step, ms64, ms_simt], device=dev, dtype=torch.float64)
        tdist.all_reduce(t, op=tdist.ReduceOp.MAX)
        ms_step, ms64, ms_simt = float(t[0]), float(t[1]), float(t[2])
    value = world * P / (ms_step * 1e-3)
    value64 = world * P / (ms64 * 1e-3)
    rv_err = float((rv32 - rv64).abs().max().item() * 1e5)          # cm/s
    rv_vs_oracle = oracle_rv_errors(case, args, rv32, rv64)
    if rv_vs_oracle is not None:
        rv_vs_oracle["fp32_simt_ccf"] = oracle_rv_errors(case, args, rv32s, rv64)["fp32"]

    # end to end through the C-ABI with host buffers (pinned), copies inside the timed region:
    # every step uploads the local spectra, computes the phases' spectra and RVs and brings both
    # back (soap_active_rv); with the host-transfer pipeline on, the uploads of one step, the
    # kernels of another and the downloads of a third overlap; the timed region ends with
    # soap_synchronize, when the last step's results are on the host
    # local spectra as the FP32 path reads them (float32: the same results, half the upload)
    q_host = torch.from_numpy(case.quiet.astype(np.float32)).pin_memory()
    a_host = torch.from_numpy(case.active[synth.SPOT].astype(np.float32)).pin_memory()
    out_host = torch.empty((P, n_px), dtype=torch.float32).pin_memory()
    rv_host = torch.empty(P, dtype=torch.float64).pin_memory()
    S.soap_set_host_async(ctx, True)
    S.soap_set_ccf_tensor_cores(ctx, True)

    def step_e2e():
        S.soap_update_star(ctx, st)
        S.soap_set_quiet_spectrum(ctx, q_host)
        S.soap_set_active_spectrum(ctx, S.SOAP_SPOT, a_host)
        S.soap_active_rv(ctx, case.regions, case.phases, S.SOAP_EFFECT_TOT, S.SOAP_FP32,
                         case.mask_lambda, case.mask_weight, case.mask_width_kms, lo, vstep, nv,
                         out_host, rv_host)

    for _ in range(W):
        step_e2e()
    S.soap_synchronize(ctx)
    barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    Ke = max(3, K)
    for _ in range(Ke):
        step_e2e()
    S.soap_synchronize(ctx)
    e2e_ms = (time.perf_counter() - t0) * 1e3 / Ke
    S.soap_set_host_async(ctx, False)
    e2e_rv_err = float(np.abs(rv_host.numpy() - rv32.cpu().numpy()).max() * 1e5)
    if world > 1:
        import torch.distributed as tdist
        t = torch.tensor([e2e_ms], device=dev, dtype=torch.float64)
        tdist.all_reduce(t, op=tdist.ReduceOp.MAX)
        e2e_ms = float(t[0])
    # local spectra, phases, regions in (the mask tables stay on the device while the mask is
    # unchanged); spectra and RVs out
    h2d = q_host.numel() * 4 + a_host.numel() * 4 + P * 8 + len(case.regions) * 48
    d2h = P * n_px * 4 + P * 8

    # rooflines of the two largest kernels of the mixed path; "roofline" is the dominant one
    n_mu = st.n_mu
    n_class = len({(r.type, r.temp_K) for r in case.regions})
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except OSError:
        pass
    hbm_peak = float(peaks.get("hbm_gbs", 6800.0))
    src = "measured" if peaks else "fallback"
    full = (st.grid_n, n_px) == (300, 205800)

    def per_launch(name):
        ms, n = timers[name]
        return ms / max(1, n)

    # contraction: output once + the quiet and active rows, contrast and F_q read once
    bytes_contract = (P * n_px * 4 + 2 * n_mu * n_px * 4 + n_class * n_px * 4 + n_px * 4)
    c_per = per_launch("contract")
    achieved = bytes_contract / (c_per * 1e-3) / 1e9
    rl_contract = {"kernel": "k_contract<float,4,4,128> (Toeplitz contraction, active phases)", "bound": "hbm",
                   "achieved": round(achieved, 1), "peak": hbm_peak, "unit": "GB/s",
                   "frac": round(achieved / hbm_peak, 4),
                   "traffic": profiled_traffic("k_contract_f32_disk300_205800px.md") if full else None,
                   "bytes_per_launch": bytes_contract, "ms_per_launch": round(c_per, 5), "peak_source": src}
    # CCF on the tensor cores: it streams the line-mask matrix (BF16 hi + lo per velocity, padded
    # to 16, and pixel, padded to 64) and the spectra once per launch
    n_pad = -(-nv // 16) * 16
    bytes_ccf_tc = (-(-n_px // 64) * 64) * n_pad * 4 + P * n_px * 4
    t_per = per_launch("ccf")
    ach_tc = bytes_ccf_tc / (t_per * 1e-3) / 1e9
    rl_ccf_tc = {"kernel": "k_ccf_tc (CCF as a tcgen05 GEMM, BF16 hi/lo, warp-specialised)", "bound": "hbm",
                 "achieved": round(ach_tc, 1), "peak": hbm_peak, "unit": "GB/s",
                 "frac": round(ach_tc / hbm_peak, 4),
                 "traffic": profiled_traffic("k_ccf_tc_bf16x3_disk300_205800px.md") if full else None,
                 "bytes_per_launch": bytes_ccf_tc, "ms_per_launch": round(t_per, 5), "peak_source": src}
    # SIMT CCF: 2 pixels per (line, velocity, spectrum), one FMA (2 flop) each, over the lines
    # whose box stays on the grid; FP32 SIMT peak from the unit counts and the maximum SM clock
    delta = np.log(st.lambda_end_A / st.lambda_start_A) / (n_px - 1)
    h = case.mask_width_kms / (2 * 299792.458 * delta)
    u = np.log(case.mask_lambda / st.lambda_start_A) / delta
    s_lo = np.arctanh(lo / 299792.458) / delta
    s_hi = np.arctanh((lo + vstep * (nv - 1)) / 299792.458) / delta
    n_valid = int(np.sum((u + s_lo - h >= -0.5) & (u + s_hi + h <= n_px - 0.5)))
    flops_ccf = 4.0 * P * n_valid * nv
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    max_mhz = float(clocks.get("sm_max_mhz") or 2070.0)
    fp32_peak = sms * 128 * 2 * max_mhz * 1e6 / 1e12
    f_per = timers_simt["ccf"][0] / max(1, timers_simt["ccf"][1])
    ach_ccf = flops_ccf / (f_per * 1e-3) / 1e12
    rl_ccf = {"kernel": "k_ccf_tile (CCF, 4 velocities x 16 spectra per thread)", "bound": "alu",
              "achieved": round(ach_ccf, 2), "peak": round(fp32_peak, 1), "unit": "TFLOP/s",
              "frac": round(ach_ccf / fp32_peak, 4),
              "traffic": profiled_traffic("k_ccf_tile_f32_disk300_205800px.md") if full else None,
              "flops_per_launch": flops_ccf, "ms_per_launch": round(f_per, 5),
              "peak_source": f"derived: {sms} SMs x 128 FP32 lanes x 2 flop x {max_mhz:.0f} MHz"}
    name, (tot, n) = max(timers.items(), key=lambda kv: kv[1][0])
    roofline = dict(rl_ccf_tc if c_per < t_per else rl_contract)
    roofline.update({"dominant_kernel": name, "dominant_ms_per_step": round(tot / K, 5)})
    rooflines = {"contract": rl_contract, "ccf": rl_ccf_tc, "ccf_simt": rl_ccf}
    kernel_ms_per_step = {k: round(v[0] / K, 5) for k, v in timers.items() if v[1]}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(case, args.cpu_sample_px)
    extras = {}
    if rank == 0 and world == 1 and not args.no_extras:
        S.soap_free(ctx)
        ctx = None
        del out32, out64, flush
        torch.cuda.empty_cache()
        extras["batched"] = measure_batched(args, dev, hbm_peak)
        torch.cuda.empty_cache()
        extras["surrogate"] = measure_surrogate(args, dev)
        torch.cuda.empty_cache()
        extras["quiet_forms"] = measure_quiet_forms(args, dev)
        torch.cuda.empty_cache()
        extras["instrument"] = measure_instrument(args, dev, hbm_peak)
        torch.cuda.empty_cache()
        extras["bisectors"] = measure_bisectors(args, dev, hbm_peak)
        torch.cuda.empty_cache()
        extras["tensor_contraction"] = measure_tensor_contraction(args, dev, float(peaks.get("bf16_tflops", 1913.8)))

    res = {"metric": METRIC, "value": round(value, 2), "unit": UNIT, "n_gpus": world,
           "steps": K, "warmup": W, "ms_per_step": round(ms_step, 5), "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f32+bf16x3",
           "data": "synthetic (seeded 20k-line spectra, random-init regions)",
           "config": {"workload": case.name, "grid": st.grid_n, "n_px": n_px, "n_mu": n_mu,
                      "phases_per_step": P, "effects": "total (Eq. 3)",
                      "precision": "FP32 local spectra, contraction and fit; CCF as BF16 hi/lo tcgen05 GEMM "
                                   "with FP32 accumulation; FP64 positions and weights",
                      "l2": "flushed between timed steps (256 MB write)",
                      "parallelism": f"replicas{world}"},
           "rv_err_cms_vs_fp64": rv_err,
           "rv_err_cms_vs_oracle": rv_vs_oracle,
           "fp32_simt_ccf": {"value": round(world * P / (ms_simt * 1e-3), 2), "unit": UNIT,
                             "ms_per_step": round(ms_simt, 5), "gpu_launches": int(launches_simt),
                             "rv_max_diff_cms_vs_tensor_ccf": float((rv32 - rv32s).abs().max().item() * 1e5),
                             "kernel_ms_per_step": {k: round(v[0] / K, 5) for k, v in timers_simt.items() if v[1]}},
           "fp64_path": {"value": round(value64, 2), "unit": UNIT, "ms_per_step": round(ms64, 5),
                         "kernel_ms_per_step": {k: round(v[0] / K64, 5)
                                                for k, v in timers64.items() if v[1]}},
           "roofline": roofline, "rooflines": rooflines, "kernel_ms_per_step": kernel_ms_per_step,
           "e2e": {"value": round(world * P / (e2e_ms * 1e-3), 2), "unit": UNIT,
                   "ms_per_step": round(e2e_ms, 4), "h2d_bytes_per_step": int(h2d),
                   "d2h_bytes_per_step": int(d2h), "api": "soap_active_rv, host-transfer pipeline",
                   "rv_max_diff_cms_vs_device_path": e2e_rv_err},
           "gpu_launches": int(launches_plain), "clocks": clocks}
    if cpu is not None:
        res["cpu_baseline"] = cpu
    res.update(extras)
    if ctx is not None:
        S.soap_free(ctx)
    if rank == 0:
        print(json.dumps(res), flush=True)
    if world > 1:
        import torch.distributed as tdist
        tdist.destroy_process_group()


def oracle_rv_errors(case, args, rv32, rv64):
    """Max |RV - RV_oracle| (cm/s) of the FP32 and FP64 paths over the 100 phases, against the FP64
    oracle's RVs of its own full-size spectra (tests/golden/cfg2_fullsize_oracle.json, written by
    tests/golden/make_cfg2_fullsize.py for seed 0); None for any other workload."""
    path = os.path.join(ROOT, "tests", "golden", "cfg2_fullsize_oracle.json")
    if (args.seed, case.star.grid_n, case.star.n_px) != (0, 300, 205800) or not os.path.exists(path):
        return None
    g = json.load(open(path))
    ref = np.asarray(g["rv_kms"])
    if ref.size != rv32.numel():
        return None
    return {"fp32": round(float(np.abs(rv32.cpu().numpy() - ref).max() * 1e5), 6),
            "fp64": float(np.abs(rv64.cpu().numpy() - ref).max() * 1e5),
            "oracle": "FP64 oracle, all 205,800 px x 100 phases (tests/golden/cfg2_fullsize_oracle.json)"}


def profiled_traffic(name):
    """DRAM bytes read + written per launch from a committed ncu summary (profiles/), or None."""
    try:
        text = open(os.path.join(ROOT, "profiles", name)).read()
    except OSError:
        return None
    tot = 0.0
    for key in ("DRAM read", "DRAM write"):
        for line in text.splitlines():
            if line.startswith(f"| {key} |"):
                val, unit = line.split("|")[2].split()[:2]
                tot += float(val) * {"byte": 1, "Kbyte": 1e3, "Mbyte": 1e6, "Gbyte": 1e9,
                                     "B": 1, "KB": 1e3, "MB": 1e6, "GB": 1e9}[unit]
                break
        else:
            return None
    return int(tot)


# ------------------------------------------------------------------------------------------
# batched form and surrogate (N = 1)
# ------------------------------------------------------------------------------------------
def _disk(S, case, dev):
    import torch
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    return S.Disk(case.star, t(case.quiet), {k: t(v) for k, v in case.active.items()})


def measure_batched(args, dev, hbm_peak):
    """4096 independent configurations (disk 150x150, 6000-6300 A at 16,834 px, 10-200 phases,
    1-4 spots, vsini 1-10 km/s, i 30-90 deg): one autotuned, graph-captured soap_active_batch per
    step; the 29 GB of output exceed L2, so no flush is needed between steps."""
    import torch
    from paper_2301_04259_gb300 import soap as S
    from paper_2301_04259_gb300 import synth
    case = synth.batch_spectra(args.seed)
    cfgs = synth.batch_configs(args.seed + 1, args.batch_configs)
    items, regions, phases = synth.batch_layout(cfgs)
    it, rg, ph = S.batch_columns_arrays({
        "vsini": [c[0] for c in items], "incl": [c[1] for c in items], "first_region": [c[2] for c in items],
        "n_regions": [c[3] for c in items], "first_phase": [c[4] for c in items],
        "n_phases": [c[5] for c in items], "type": [r.type for r in regions], "lat": [r.lat_deg for r in regions],
        "lon": [r.lon_deg for r in regions], "radius": [r.radius_rstar for r in regions],
        "temp": [r.temp_K for r in regions], "phases": phases})
    n_px = case.star.n_px
    out = torch.empty((phases.size, n_px), dtype=torch.float32, device=dev)
    with _disk(S, case, dev) as d:
        best, ms_var = S.soap_batch_autotune(d.ctx, items, regions, phases, out, reps=2)
        stream = torch.cuda.current_stream()
        for _ in range(3):
            S.soap_active_batch_arrays(d.ctx, it, rg, ph, out)
        torch.cuda.synchronize()
        K = 5
        l0 = S.soap_get_launch_count(d.ctx)
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(K)]
        for k in range(K):
            ev[k][0].record(stream)
            S.soap_active_batch_arrays(d.ctx, it, rg, ph, out)
            ev[k][1].record(stream)
        torch.cuda.synchronize()
        launches = (S.soap_get_launch_count(d.ctx) - l0) // K
        ms = float(np.mean([a.elapsed_time(b) for a, b in ev]))
        S.soap_set_profiling(d.ctx, True)
        S.soap_reset_kernel_times(d.ctx)
        S.soap_active_batch_arrays(d.ctx, it, rg, ph, out)
        S.soap_synchronize(d.ctx)
        kernels = {name: round(S.soap_get_kernel_time(d.ctx, t)[0], 4) for t, name in enumerate(S.TIMERS)
                   if S.soap_get_kernel_time(d.ctx, t)[1]}
        S.soap_set_profiling(d.ctx, False)
        S.soap_synchronize(d.ctx)
        # the same batch with the RV of every spectrum (Sect. 4.1): CCF on one grid -30..30 km/s
        # (0.25 km/s), each configuration fitted within |v| <= |vsini| + 20 km/s, inside the graph
        lo, step, nv = synth.velocity_grid(10.0)
        rv = torch.empty(phases.size, dtype=torch.float64, device=dev)
        with_rv = {}
        for form, tcf in (("simt_ccf", False), ("tensor_ccf", True)):
            S.soap_batch_set_rv(d.ctx, case.mask_lambda, case.mask_weight, case.mask_width_kms, lo, step, nv,
                                20.0, tcf)
            for _ in range(2):
                S.soap_active_batch_arrays(d.ctx, it, rg, ph, out, rv_out=rv)
            torch.cuda.synchronize()
            K2 = 3
            l0 = S.soap_get_launch_count(d.ctx)
            ev2 = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(K2)]
            for k in range(K2):
                ev2[k][0].record(stream)
                S.soap_active_batch_arrays(d.ctx, it, rg, ph, out, rv_out=rv)
                ev2[k][1].record(stream)
            torch.cuda.synchronize()
            launches_rv = (S.soap_get_launch_count(d.ctx) - l0) // K2
            ms_rv = float(np.mean([a.elapsed_time(b) for a, b in ev2]))
            S.soap_set_profiling(d.ctx, True)
            S.soap_reset_kernel_times(d.ctx)
            S.soap_active_batch_arrays(d.ctx, it, rg, ph, out, rv_out=rv)
            S.soap_synchronize(d.ctx)
            krv = {name: round(S.soap_get_kernel_time(d.ctx, t)[0], 4) for t, name in enumerate(S.TIMERS)
                   if name in ("ccf", "ccf_aux", "fit") and S.soap_get_kernel_time(d.ctx, t)[1]}
            S.soap_set_profiling(d.ctx, False)
            S.soap_synchronize(d.ctx)
            r = rv.cpu().numpy()
            with_rv[form] = {"ms_per_batch": round(ms_rv, 3), "spectra_and_rvs_per_s": round(phases.size / (ms_rv * 1e-3), 1),
                             "gpu_launches_per_batch": int(launches_rv), "rv_kernel_ms": krv,
                             "rv_finite_frac": round(float(np.isfinite(r).mean()), 6)}
    out_bytes = out.numel() * 4
    del out
    c_ms = kernels.get("contract", ms)
    return {"workload": f"batch{len(cfgs)}_disk150_{n_px}px", "configs": len(cfgs), "spectra": int(phases.size),
            "ms_per_batch": round(ms, 3), "spectra_per_s": round(phases.size / (ms * 1e-3), 1),
            "variant": {"index": best, "phases_per_block": S.soap_batch_variant_info(best)[0],
                        "px_per_thread": S.soap_batch_variant_info(best)[1]},
            "autotune_ms": [round(float(v), 3) for v in ms_var], "gpu_launches_per_batch": int(launches),
            "kernel_ms": kernels, "output_bytes": int(out_bytes),
            "with_rv": with_rv, "rv_velocity_grid": {"v_lo": lo, "v_step": step, "n_v": nv, "fit_margin_kms": 20.0},
            "contract_hbm_write_gbs": round(out_bytes / (c_ms * 1e-3) / 1e9, 1),
            "contract_frac_of_hbm": round(out_bytes / (c_ms * 1e-3) / 1e9 / hbm_peak, 4),
            "precision": "FP32 contraction, FP64 positions"}


def measure_surrogate(args, dev):
    """Surrogate trained on the batched method's residual spectra; checked accuracy on held-out
    queries (true RVs from the plain method), and throughput on --sur-queries queries."""
    import torch
    from paper_2301_04259_gb300 import soap as S
    from paper_2301_04259_gb300 import synth
    from paper_2301_04259_gb300 import surrogate_pipeline as SP
    case = synth.batch_spectra(args.seed)
    n_px = case.star.n_px
    res = {}
    with _disk(S, case, dev) as d:
        t0 = time.perf_counter()
        model = SP.train(d.ctx, case, n_train=args.sur_train, epochs=args.sur_epochs, seed=args.seed,
                         n_err=args.sur_err, err_epochs=args.sur_err_epochs)
        res["train_wall_s"] = round(time.perf_counter() - t0, 2)
        res["train"] = {k: (round(v, 4) if isinstance(v, float) else v) for k, v in model.log.items()
                        if k not in ("loss", "head_loss", "rv_sens_cms_per_sd")}
        res["train"]["final_loss"] = model.log["loss"][-1]
        xe = synth.surrogate_params(args.seed + 99, 8192)
        err = SP.plain_rv_errors(d.ctx, case, model, xe)
        acc = torch.empty(len(xe), dtype=torch.uint8, device=dev)
        S.soap_surrogate_predict(model.handle, SP.encode_dev(xe), model.accept_thr_cms, accepted=acc)
        a = acc.cpu().numpy().astype(bool)
        res["heldout_vs_plain"] = {
            "queries": len(xe), "accepted_frac": round(float(a.mean()), 4),
            "rv_err_cms_all_median": round(float(np.median(err)), 3),
            "rv_err_cms_accepted_p50_p95_p99_max": [round(float(np.percentile(err[a], q)), 3) for q in (50, 95, 99, 100)]
            if a.any() else None,
            "accepted_over_10cms_frac": round(float((err[a] > SP.RV_ERR_MAX_CMS).mean()), 4) if a.any() else None,
            "accept_threshold_pred_cms": round(model.accept_thr_cms, 4)}
        # throughput on n queries in chunks of 65536 (one reused output buffer): answers as 128
        # PCA coefficients (plain: residual spectra + projection; network) and as residual spectra
        # (plain; surrogate for every query; hybrid = surrogate where accepted, plain elsewhere)
        nq, ch = args.sur_queries, 65536
        xq = synth.surrogate_params(args.seed + 123, nq)
        xqd = SP.encode_dev(xq)          # the network's inputs
        out = torch.empty((ch, n_px), dtype=torch.float32, device=dev)
        coef = torch.empty((nq, 128), dtype=torch.float32, device=dev)
        accq = torch.empty(nq, dtype=torch.uint8, device=dev)

        def plain_coef():
            for a0 in range(0, nq, ch):
                m = min(ch, nq - a0)
                SP.plain_residuals(d.ctx, xq[a0:a0 + m], out[:m])
                S.soap_pca_project(out[:m], model.mean, model.basis, coef[a0:a0 + m])

        def surrogate_coef():
            S.soap_surrogate_predict(model.handle, xqd, model.accept_thr_cms, coef=coef, accepted=accq)

        def plain_spec():
            for a0 in range(0, nq, ch):
                m = min(ch, nq - a0)
                SP.plain_residuals(d.ctx, xq[a0:a0 + m], out[:m])

        def surrogate_spec():
            for a0 in range(0, nq, ch):
                m = min(ch, nq - a0)
                S.soap_surrogate_query(model.handle, xqd[a0:a0 + m], model.accept_thr_cms, out[:m], accq[a0:a0 + m])

        def hybrid_spec():
            SP.query(d.ctx, model, xq, chunk=ch)

        def hybrid_coef():
            SP.query_coefficients(d.ctx, model, xq, coef, chunk=ch)

        timing = {}
        for name, fn in (("plain_coefficients", plain_coef), ("surrogate_coefficients", surrogate_coef),
                         ("hybrid_coefficients", hybrid_coef), ("plain_spectra", plain_spec),
                         ("surrogate_spectra", surrogate_spec), ("hybrid_spectra", hybrid_spec)):
            fn()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            fn()
            torch.cuda.synchronize()
            timing[name] = time.perf_counter() - t0
        res["queries"] = nq
        res["queries_per_s"] = {k: round(nq / v, 1) for k, v in timing.items()}
        res["accepted_frac_queries"] = round(float(accq.float().mean().item()), 4)
        res["gain_coefficients_vs_plain"] = round(timing["plain_coefficients"] / timing["surrogate_coefficients"], 2)
        res["gain_hybrid_coefficients_vs_plain"] = round(timing["plain_coefficients"] / timing["hybrid_coefficients"], 3)
        res["gain_hybrid_spectra_vs_plain"] = round(timing["plain_spectra"] / timing["hybrid_spectra"], 3)
        res["precision"] = "BF16 weights/activations, FP32 accumulation; split-BF16 reconstruction"
        res["note"] = ("coefficients: 128 PCA coefficients of F - F_q per query; spectra: F - F_q in "
                       "chunks of 65536; surrogate_* answers every query from the network, hybrid_* "
                       "only the accepted ones (the plain method, projected for coefficients, "
                       "elsewhere: the answer that keeps the acceptance guarantee); wall-clock incl. "
                       "host bookkeeping")
        model.free()
    return res


# ------------------------------------------------------------------------------------------
# CPU oracle (cpu_baseline leg and the reference arm)
# ------------------------------------------------------------------------------------------
def oracle_step_seconds(case, n_sample, seed):
    """Oracle time for one step's worth of work, from a pixel sample of the spectra and two
    of the RV fits, scaled to all pixels and all phases."""
    from oracle import oracle as O
    from paper_2301_04259_gb300 import synth
    st = case.star
    rng = np.random.default_rng(seed)
    pix = np.sort(rng.choice(st.n_px, n_sample, replace=False)).astype(np.int64)
    t0 = time.perf_counter()
    O.active(st, case.quiet, case.active, case.regions, case.phases, effects=1, pix=pix)
    t_spec = (time.perf_counter() - t0) * st.n_px / n_sample
    lo, vstep, nv = synth.velocity_grid(st.vsini_kms)
    t0 = time.perf_counter()
    O.rv(case.quiet[:2], st, case.mask_lambda, case.mask_weight, case.mask_width_kms, lo, vstep, nv)
    t_rv = (time.perf_counter() - t0) * case.phases.size / 2
    return t_spec + t_rv


def cpu_baseline(case, n_sample):
    from oracle import oracle as O
    t = oracle_step_seconds(case, n_sample, 1)
    P = case.phases.size
    return {"value": round(P / t, 5), "unit": UNIT, "cores": O.num_threads(), "kind": "oracle",
            "sample": f"{n_sample} of {case.star.n_px} px for all {P} phases + 2 of {P} CCF/RV fits, "
                      f"scaled to the full step ({t:.1f} s per {P} spectra)"}


def run_reference(args):
    rank, world, local = dist()
    if rank != 0:
        return
    from oracle import oracle as O
    case = workload(args, 0)
    P = case.phases.size
    n_sample = max(8, args.cpu_sample_px // 4)
    for k in range(max(0, args.warmup)):
        oracle_step_seconds(case, 8, 100 + k)
    times = [oracle_step_seconds(case, n_sample, k) for k in range(args.steps)]
    t = float(np.mean(times))
    value = P / t
    res = {"impl": "reference", "metric": METRIC, "value": round(value, 5), "unit": UNIT,
           "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(t * 1e3, 2),
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic", "config": {"workload": case.name, "grid": case.star.grid_n,
                                           "n_px": case.star.n_px, "phases_per_step": P},
           "cpu_baseline": {"value": round(value, 5), "unit": UNIT, "cores": O.num_threads(),
                            "kind": "oracle",
                            "sample": f"per step {n_sample} px of all {P} phases + 2 RV fits, scaled"},
           "e2e": {"value": round(value, 5), "unit": UNIT, "h2d_bytes_per_step": 0,
                   "d2h_bytes_per_step": 0}}
    print(json.dumps(res), flush=True)


def measure_gemm(args, dev, bf16_peak):
    """The surrogate's reconstruction GEMM alone: 65536 residual spectra of 16,834 px from 128
    coefficients with BF16 high/low splitting (K = 3 x 128) on the tcgen05 tensor cores."""
    import torch
    from paper_2301_04259_gb300 import soap as S
    from paper_2301_04259_gb300 import synth
    rng = np.random.default_rng(args.seed)
    n, p, k = 65536, synth.n_px_for_sampling(6000.0, 6300.0), 128
    basis = torch.from_numpy(np.linalg.qr(rng.standard_normal((p, k)))[0].T.astype(np.float32)).to(dev).contiguous()
    mean = torch.zeros(p, dtype=torch.float32, device=dev)
    coef = torch.from_numpy(rng.standard_normal((n, k)).astype(np.float32)).to(dev)
    out = torch.empty((n, p), dtype=torch.float32, device=dev)
    s = S.soap_surrogate_create(synth.SURROGATE_LO, synth.SURROGATE_HI, 128)
    try:
        S.soap_surrogate_set_basis(s, mean, basis)
        for _ in range(3):
            S.soap_surrogate_reconstruct(s, coef, out)
        torch.cuda.synchronize()
        stream = torch.cuda.current_stream()
        K = max(3, args.steps)
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(K)]
        for a, b in ev:
            a.record(stream)
            S.soap_surrogate_reconstruct(s, coef, out)
            b.record(stream)
        torch.cuda.synchronize()
        ms = float(np.median([a.elapsed_time(b) for a, b in ev]))
    finally:
        S.soap_surrogate_free(s)
    flops = 2.0 * n * p * (3 * k)
    tf = flops / (ms * 1e-3) / 1e12
    return {"kernel": "k_gemm_tn<256> (tcgen05 BF16, split reconstruction)", "M": n, "N": p, "K": 3 * k,
            "ms": round(ms, 4), "achieved_tflops": round(tf, 1), "bf16_peak_tflops": bf16_peak,
            "frac": round(tf / bf16_peak, 4), "output_gbs": round(n * p * 4 / (ms * 1e-3) / 1e9, 1),
            "note": "includes the split of the coefficient rows (one small kernel per chunk)"}


def measure_quiet_forms(args, dev):
    """The quiet-star sum (Alg. 1) of the full-size star in its two forms: the direct gather
    (every visible cell shifts, interpolates and adds its local spectrum: 2 FMA per cell-pixel)
    and the Toeplitz contraction (per-mu-bin velocity kernels), FP32 and FP64, kernel time from
    the library's timers (geometry excluded)."""
    import torch
    from paper_2301_04259_gb300 import soap as S
    from paper_2301_04259_gb300 import synth
    case = workload(args, 0)
    st = case.star
    n_px = st.n_px
    q_dev = torch.from_numpy(case.quiet).to(dev)
    ctx = S.soap_init_star(st, q_dev)
    res = {"workload": case.name, "visible_cells": None}
    try:
        info = S.soap_get_star_info(ctx)
        vis = int(getattr(info, "n_visible", 0)) or int(round(np.pi / 4 * st.grid_n ** 2))
        res["visible_cells"] = vis
        sms = torch.cuda.get_device_properties(dev).multi_processor_count
        fp32_tfma = sms * 128 * 2.07e9 / 1e12
        for form, fname in ((S.SOAP_FORM_DIRECT, "direct"), (S.SOAP_FORM_TOEPLITZ, "toeplitz")):
            for prec, pname, dt in ((S.SOAP_FP32, "fp32", torch.float32), (S.SOAP_FP64, "fp64", torch.float64)):
                out = torch.empty(n_px, dtype=dt, device=dev)
                reps = 2 if (form == S.SOAP_FORM_DIRECT and prec == S.SOAP_FP64) else 5
                S.soap_quiet_spectrum(ctx, form, prec, out)
                torch.cuda.synchronize()
                S.soap_reset_kernel_times(ctx)
                S.soap_set_profiling(ctx, True)
                for _ in range(reps):
                    S.soap_quiet_spectrum(ctx, form, prec, out)
                torch.cuda.synchronize()
                timer = S.TIMERS.index("direct" if form == S.SOAP_FORM_DIRECT else "contract_quiet")
                tot, n = S.soap_get_kernel_time(ctx, timer)
                S.soap_set_profiling(ctx, False)
                ms = tot / max(1, n)
                entry = {"ms": round(ms, 4), "spectra_per_s": round(1e3 / ms, 1)}
                if form == S.SOAP_FORM_DIRECT:
                    fma = 2.0 * vis * n_px
                    entry["cell_px_per_s"] = float(f"{vis * n_px / (ms * 1e-3):.4g}")
                    if prec == S.SOAP_FP32:
                        entry["fma_frac_of_fp32_peak"] = round(fma / (ms * 1e-3) / 1e12 / fp32_tfma, 4)
                    entry["hbm_gbs_algorithmic"] = round((st.n_mu * n_px + n_px) * (4 if prec == S.SOAP_FP32 else 8)
                                                         / (ms * 1e-3) / 1e9, 1)
                res[f"{fname}_{pname}"] = entry
    finally:
        S.soap_free(ctx)
    res["note"] = ("direct: 2 FMA per visible cell-pixel, rows read through L1 (HBM is not its limit: the "
                   "rows are 16.5 MB); toeplitz: the same sum as per-mu-bin banded convolutions")
    return res


def measure_instrument(args, dev, hbm_peak):
    """Instrumental resolution lowering (Sect. 3.3 after Eq. 4) of the step's 100 full-size
    spectra at R = 115000 (FWHM 3 px, 19 taps): kernel time from the library's timer and its
    HBM roofline (each spectrum read once and written once)."""
    import torch
    from paper_2301_04259_gb300 import soap as S
    case = workload(args, 0)
    st = case.star
    P, n_px = case.phases.size, st.n_px
    ctx = S.soap_init_star(st, torch.from_numpy(case.quiet).to(dev))
    res = {"workload": case.name, "resolving_power": 115000.0, "spectra": P}
    try:
        S.soap_set_instrument_resolution(ctx, 115000.0)
        for dt, name, esz in ((torch.float32, "fp32", 4), (torch.float64, "fp64", 8)):
            src = torch.rand((P, n_px), dtype=dt, device=dev)
            dst = torch.empty_like(src)
            S.soap_lower_resolution(ctx, src, dst)
            torch.cuda.synchronize()
            S.soap_reset_kernel_times(ctx)
            S.soap_set_profiling(ctx, True)
            reps = max(3, args.steps)
            for _ in range(reps):
                S.soap_lower_resolution(ctx, src, dst)
            torch.cuda.synchronize()
            tot, n = S.soap_get_kernel_time(ctx, S.TIMERS.index("lsf"))
            S.soap_set_profiling(ctx, False)
            ms = tot / max(1, n)
            gbs = 2.0 * P * n_px * esz / (ms * 1e-3) / 1e9
            res[name] = {"ms": round(ms, 4), "hbm_gbs": round(gbs, 1), "frac_of_hbm": round(gbs / hbm_peak, 4)}
            del src, dst
    finally:
        S.soap_free(ctx)
    res["note"] = "inputs 329/165 MB > L2 (FP64/FP32); timed without an L2 flush between repetitions"
    return res


def measure_bisectors(args, dev, hbm_peak):
    """Bisector injection (Sect. 4.3) into the 20 mu rows of the full-size quiet local spectra
    (FP64): kernel time from the library's timer, whole-call time (table upload, kernel, status
    check) from CUDA events around the call, and the HBM rate of the kernel's algorithmic bytes
    (each row read once and written once)."""
    import torch
    from paper_2301_04259_gb300 import soap as S
    case = workload(args, 0)
    st = case.star
    F = torch.from_numpy(case.quiet).to(dev)
    out = torch.empty_like(F)
    d = np.linspace(0.0, 1.0, 101)
    bis = np.tile(0.25 * (d - 1.5 * d * d) + 0.05, (F.shape[0], 1))   # a C-shaped bisector, km/s
    orig = np.zeros(101)
    ctx = S.soap_init_star(st, F)
    try:
        for _ in range(3):
            S.soap_inject_bisectors(ctx, F, out, bis, orig)
        torch.cuda.synchronize()
        stream = torch.cuda.current_stream()
        reps = max(3, args.steps)
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(reps)]
        S.soap_reset_kernel_times(ctx)
        S.soap_set_profiling(ctx, True)
        for a, b in ev:
            a.record(stream)
            S.soap_inject_bisectors(ctx, F, out, bis, orig)
            b.record(stream)
        torch.cuda.synchronize()
        tot, n = S.soap_get_kernel_time(ctx, S.TIMERS.index("bisectors"))
        S.soap_set_profiling(ctx, False)
        call_ms = float(np.median([a.elapsed_time(b) for a, b in ev]))
    finally:
        S.soap_free(ctx)
    ms = tot / max(1, n)
    gbs = 2.0 * F.numel() * 8 / (ms * 1e-3) / 1e9
    return {"workload": case.name, "rows": int(F.shape[0]), "n_px": int(F.shape[1]), "kernel_ms": round(ms, 4),
            "call_ms": round(call_ms, 4), "hbm_gbs": round(gbs, 1), "frac_of_hbm": round(gbs / hbm_peak, 4),
            "note": "FP64; call_ms adds the table upload and the status-word check (a stream synchronisation)"}


def measure_tensor_contraction(args, dev, bf16_peak):
    """The active-phase contraction of the headline step in its two forms: SIMT FP32 (per-tap
    Toeplitz tiles, SOAP_FP32) and tcgen05 BF16 split precision (dense GEMM over pixels x phases x
    (class, mu bin, tap), SOAP_BF16X3).  Kernel time from the library's timer; for the tensor
    form the executed tensor work (3 products over the padded GEMM) against the BF16 peak."""
    import torch
    from paper_2301_04259_gb300 import soap as S
    case = workload(args, 0)
    st = case.star
    P, n_px = case.phases.size, st.n_px
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    ctx = S.soap_init_star(st, t(case.quiet))
    res = {"workload": case.name, "phases": P}
    outs = {}
    try:
        for k, v in case.active.items():
            S.soap_set_active_spectrum(ctx, k, t(v))
        info = S.soap_get_star_info(ctx)
        n_class = len({(r.type, r.temp_K) for r in case.regions})
        for name, prec in (("simt_fp32", S.SOAP_FP32), ("tcgen05_bf16x3", S.SOAP_BF16X3)):
            out = torch.empty((1, P, n_px), dtype=torch.float32, device=dev)
            for _ in range(3):
                S.soap_active_phases(ctx, case.regions, case.phases, S.SOAP_EFFECT_TOT, prec, out)
            torch.cuda.synchronize()
            S.soap_reset_kernel_times(ctx)
            S.soap_set_profiling(ctx, True)
            for _ in range(max(3, args.steps)):
                S.soap_active_phases(ctx, case.regions, case.phases, S.SOAP_EFFECT_TOT, prec, out)
            torch.cuda.synchronize()
            tot, n = S.soap_get_kernel_time(ctx, S.TIMERS.index("contract"))
            S.soap_set_profiling(ctx, False)
            res[name] = {"ms": round(tot / max(1, n), 4)}
            outs[name] = out
        # k_toeplitz_tma: M = pixels, N = phase groups of 64, K = (term, 8-bin planes, taps) with one
        # accumulator per term (Q and each class); all-zero coefficient tiles are skipped, so the
        # dense product below is an upper bound of the executed work
        n_acc = n_class + 1
        k_dense = n_acc * (-(-st.n_mu // 8) * 8) * (-(-info.n_taps // 2) * 2)
        p_pad = -(-P // 64) * 64
        m_pad = -(-n_px // 128) * 128
        flops = 2.0 * 3 * m_pad * p_pad * k_dense
        ms = res["tcgen05_bf16x3"]["ms"]
        tf = flops / (ms * 1e-3) / 1e12
        res["tcgen05_bf16x3"].update({"kernel": "k_toeplitz_tma", "dense_gemm": [m_pad, p_pad, k_dense],
                                      "dense_tflop_upper_bound": round(flops / 1e12, 4),
                                      "dense_tflops_upper_bound": round(tf, 1),
                                      "frac_of_bf16_peak_upper_bound": round(tf / bf16_peak, 4)})
        res["max_abs_diff_vs_fp32"] = float((outs["tcgen05_bf16x3"] - outs["simt_fp32"]).abs().max().item())
        # the CCF of the same spectra in its two forms (soap_rv_ccf, FP32 spectra in HBM)
        from paper_2301_04259_gb300 import synth
        spec = outs["simt_fp32"][0]
        lo, vstep, nv = synth.velocity_grid(st.vsini_kms)
        ccf, rvs = {}, {}
        for name, tcf in (("simt_fp32", False), ("tcgen05_bf16x3", True)):
            rv = torch.empty(P, dtype=torch.float64, device=dev)
            call = lambda: S.soap_rv_ccf(ctx, spec, case.mask_lambda, case.mask_weight, case.mask_width_kms,
                                         lo, vstep, nv, rv, tensor_cores=tcf)
            for _ in range(3):
                call()
            torch.cuda.synchronize()
            S.soap_reset_kernel_times(ctx)
            S.soap_set_profiling(ctx, True)
            for _ in range(max(3, args.steps)):
                call()
            torch.cuda.synchronize()
            tot, n = S.soap_get_kernel_time(ctx, S.TIMERS.index("ccf"))
            S.soap_set_profiling(ctx, False)
            ccf[name] = {"ms": round(tot / max(1, n), 4)}
            rvs[name] = rv.cpu().numpy()
        # executed tensor work: 3 products over M = 128 spectra, N = velocities rounded up to 16,
        # K = each pixel chunk rounded up to 64 (one wave of CTAs over the pixels)
        sms = torch.cuda.get_device_properties(dev).multi_processor_count
        per = -(-(n_px * -(-P // 128)) // sms)
        chunk = max(64, -(-per // 64) * 64)
        k_exec = sum(-(-min(chunk, n_px - p0) // 64) * 64 for p0 in range(0, n_px, chunk))
        flops = 2.0 * 3 * 128 * (-(-nv // 16) * 16) * k_exec * (-(-P // 128))
        tf = flops / (ccf["tcgen05_bf16x3"]["ms"] * 1e-3) / 1e12
        ccf["tcgen05_bf16x3"].update({"gemm": [128 * (-(-P // 128)), -(-nv // 16) * 16, k_exec],
                                      "executed_tflop": round(flops / 1e12, 4), "achieved_tflops": round(tf, 1),
                                      "frac_of_bf16_peak": round(tf / bf16_peak, 4)})
        ccf["max_rv_diff_cm_s"] = float(np.nanmax(np.abs(rvs["tcgen05_bf16x3"] - rvs["simt_fp32"])) * 1e5)
        res["ccf"] = ccf
    finally:
        S.soap_free(ctx)
    res["note"] = ("tensor form k_toeplitz_tma: operand windows by TMA, taps as descriptor offsets, one accumulator "
                   "per term, all-zero coefficient tiles skipped; bound by the operand fetch of the no-swizzle "
                   "layout (profiles/k_toeplitz_tma_bf16x3_disk300_205800px.md). The SIMT kernel visits only the "
                   "non-zero taps of each block of 4 phases (~50 FMA per phase and pixel)")
    return res


def run_block(args):
    import torch
    torch.cuda.set_device(0)
    dev = torch.device("cuda:0")
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except OSError:
        pass
    if args.only == "batched":
        res = measure_batched(args, dev, float(peaks.get("hbm_gbs", 6800.0)))
    elif args.only == "surrogate":
        res = measure_surrogate(args, dev)
    elif args.only == "quiet":
        res = measure_quiet_forms(args, dev)
    elif args.only == "instrument":
        res = measure_instrument(args, dev, float(peaks.get("hbm_gbs", 6800.0)))
    elif args.only == "bisectors":
        res = measure_bisectors(args, dev, float(peaks.get("hbm_gbs", 6800.0)))
    elif args.only == "tensor":
        res = measure_tensor_contraction(args, dev, float(peaks.get("bf16_tflops", 1913.8)))
    else:
        res = measure_gemm(args, dev, float(peaks.get("bf16_tflops", 1900.0)))
    print(json.dumps({"block": args.only, **res}), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    elif args.only != "all":
        run_block(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
