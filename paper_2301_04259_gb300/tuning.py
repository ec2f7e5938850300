"""Persisted variant choice of the batched form (soap_active_batch).

The fastest variant (phases per block, pixels per thread) depends on the shape of the
problem: pixels per spectrum, velocity-kernel taps, mu bins, grid size and the GPU.  The first
run on a shape calls soap_batch_autotune and stores the winner in a JSON table keyed by that
shape; later runs read it back and set it with soap_batch_set_variant.
"""
from __future__ import annotations

import json
import os
from pathlib import Path
from typing import Callable, Optional

DEFAULT_PATH = Path(os.environ.get("SOAP_TUNING_CACHE",
                                   Path.home() / ".cache" / "soap_gb300" / "batch_tuning.json"))


def tuning_key(n_px: int, n_taps: int, n_mu: int, grid_n: int, device: str) -> str:
    return f"{device}|npx={int(n_px)}|taps={int(n_taps)}|mu={int(n_mu)}|grid={int(grid_n)}"


def load_table(path: Path) -> dict:
    try:
        with open(path) as f:
            table = json.load(f)
        return table if isinstance(table, dict) else {}
    except (OSError, ValueError):
        return {}


def save_table(path: Path, table: dict) -> None:
    path = Path(path)
    path.parent.mkdir(parents=True, exist_ok=True)
    tmp = path.with_suffix(path.suffix + ".tmp")
    with open(tmp, "w") as f:
        json.dump(table, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def choose_variant(key: str, autotune: Callable[[], tuple], set_variant: Callable[[int], None],
                   n_variants: int, path: Optional[Path] = None, retune: bool = False) -> dict:
    """Set the stored variant for `key`, or run `autotune() -> (best, ms_per_variant)`, store
    and set its winner.  Returns the table entry (with "source": "cache" or "autotune")."""
    path = Path(path) if path is not None else DEFAULT_PATH
    table = load_table(path)
    entry = table.get(key)
    if (not retune and isinstance(entry, dict) and isinstance(entry.get("variant"), int)
            and 0 <= entry["variant"] < n_variants):
        set_variant(entry["variant"])
        return dict(entry, source="cache")
    best, ms = autotune()
    entry = {"variant": int(best), "ms": [float(x) for x in ms]}
    table[key] = entry
    save_table(path, table)
    set_variant(int(best))
    return dict(entry, source="autotune")


def tune_batch(ctx, star, items, regions, phases, out, path: Optional[Path] = None,
               reps: int = 3, retune: bool = False) -> dict:
    """choose_variant for a context and a device batch (soap_batch_autotune on a miss)."""
    import torch

    from . import soap

    info = soap.soap_get_star_info(ctx)
    key = tuning_key(star.n_px, info.n_taps, len(star.mu_values), star.grid_n,
                     torch.cuda.get_device_name(out.device))
    return choose_variant(
        key,
        lambda: soap.soap_batch_autotune(ctx, items, regions, phases, out, reps=reps),
        lambda v: soap.soap_batch_set_variant(ctx, v),
        soap.soap_batch_num_variants(), path=path, retune=retune)
