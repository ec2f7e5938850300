"""Write tests/golden/cfg2_fullsize_oracle.json: the FP64 oracle's answer for the full-size
active-star workload (disk 300 x 300, 3800-6900 A at 205,800 px, 20 mu bins, a facula with a
spot inside it plus a second spot, 100 phases, vsini 2 km/s; seed 0 of synth.config2).

It stores
  - the 100 radial velocities (km/s) and Gaussian fit parameters (A, B, mu, sigma) of the
    oracle's TOT spectra (Alg. 5 with Eqs. 3-4; CCF and least-squares Gaussian of Sect. 4.1);
  - a few hundred sampled (phase, pixel) values of those spectra and the matching values of the
    quiet spectrum (Alg. 1), for the flux tolerance normalisation.

Only the oracle computes anything here (the synthetic inputs come from synth.py, which holds
none of the method's arithmetic).  It takes about 12 minutes on 8 cores:

    python tests/golden/make_cfg2_fullsize.py [--out PATH]

The synthetic spectra depend on the platform's float64 exp at the 1e-12 level: numpy's
vectorised exp rounds differently on x86-64 (AVX-512) and aarch64, and on a 6000 A grid a
one-ulp change of a wavelength moves a line-flank value by ~1e-11 relative (the wavelength is
~4e4 times the distance to the line centre in units of its own rounding).  The oracle's answer
inherits that, so the stored values are written on the platform the GPU tests run on (aarch64)
and the file records the platform.
"""
from __future__ import annotations

import argparse
import json
import platform
import sys
import time
from pathlib import Path

import numpy as np

ROOT = Path(__file__).resolve().parents[2]
sys.path.insert(0, str(ROOT))

from oracle import oracle as O                      # noqa: E402
from paper_2301_04259_gb300 import synth           # noqa: E402

OUT = Path(__file__).resolve().parent / "cfg2_fullsize_oracle.json"
SEED = 0
N_SAMPLES = 400
SAMPLE_SEED = 20230110


def main() -> None:
    ap = argparse.ArgumentParser()
    ap.add_argument("--out", default=str(OUT))
    out = Path(ap.parse_args().out)
    O.build()
    t0 = time.time()
    case = synth.config2(SEED)
    st = case.star
    F = O.active(st, case.quiet, case.active, case.regions, case.phases)[0]       # [100, n_px]
    t1 = time.time()
    v_lo, v_step, n_v = synth.velocity_grid(st.vsini_kms)
    rv, params, _ = O.rv(F, st, case.mask_lambda, case.mask_weight, case.mask_width_kms, v_lo, v_step, n_v)
    t2 = time.time()
    rng = np.random.default_rng(SAMPLE_SEED)
    sp = rng.integers(0, F.shape[0], N_SAMPLES)
    px = np.sort(rng.choice(st.n_px, N_SAMPLES, replace=False))
    Fq = O.quiet(st, case.quiet, pix=px.astype(np.int64))
    doc = {
        "about": ("FP64 oracle results for the full-size active-star workload: synth.config2(seed=0), "
                  "disk 300x300, 3800-6900 A at 205,800 px, 20 mu bins, 1 facula + 2 spots, 100 phases, "
                  "vsini 2 km/s.  RVs from the box-mask CCF and least-squares Gaussian (Sect. 4.1) of the "
                  "TOT spectra (Alg. 5, Eqs. 3-4).  Written by tests/golden/make_cfg2_fullsize.py, which "
                  "calls only oracle/."),
        "seed": SEED,
        "n_px": int(st.n_px),
        "n_phases": int(F.shape[0]),
        "mask_width_kms": case.mask_width_kms,
        "v_lo": v_lo, "v_step": v_step, "n_v": int(n_v),
        "rv_kms": [float(x) for x in rv],
        "fit_params": [[float(x) for x in p] for p in params],
        "samples": {
            "phase_index": [int(x) for x in sp],
            "pixel": [int(x) for x in px],
            "F": [float(F[s, p]) for s, p in zip(sp, px)],
            "F_quiet": [float(x) for x in Fq],
        },
        "max_F_quiet_sampled": float(Fq.max()),
        "oracle_seconds": {"spectra": round(t1 - t0, 1), "rv": round(t2 - t1, 1)},
        "oracle_threads": O.num_threads(),
        "platform": {"machine": platform.machine(), "numpy": np.__version__},
    }
    out.write_text(json.dumps(doc, indent=1) + "\n")
    print(f"wrote {out} ({t1 - t0:.0f} s spectra, {t2 - t1:.0f} s RVs)")


if __name__ == "__main__":
    main()
