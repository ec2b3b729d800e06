"""Autotuner for libmw3 launch shapes.

For a workload's grid shape and precision it times short propagations through the
library's own per-kernel CUDA-event timers (mw3_kernel_times) over a sweep of
  kin_warp    half-warp FFT kinetic kernels (2: spectral partners through shared
              memory, 3: by shuffles), warp-register ones (1) or the shared-memory
              ones (0),
  kin_fused   both radial terms in one launch of thread-block clusters (1 cluster size
              chosen by the library, 2/4/8 that size) or the two kernels (0),
  rows_pairs  line pairs per CTA of the R-direction kinetic kernel,
  cols_tile   R columns per CTA of the r-direction kinetic kernel,
  tc_persist  form of the tensor-core angular step (mixed precision): 4 tile-major
              parity-split (one electronic state), 2 group-major parity-split,
              1 persistent without the split, 0 one tile per CTA (the library falls
              back to the nearest form a shape supports),
  tc_tma      tile copies of the tile-major angular step by the tensor memory
              accelerator (1) or cp.async (0),
  flush_tc    energy-sum flush on the tensor cores (1) or the CUDA cores (0),
  prod_gather product-channel node sums from stencil columns gathered plane-major
              first (1) or from 4 x 4 stencils read straight from the state (0),
  kb          iterations per energy-sum flush (ring depth),
and keeps, for each knob, the value with the lowest time of the kernels it
controls. Results are cached in a JSON file keyed by the shape, so a later
Propagator(..., tuning="auto") reuses them without measuring again.
"""
from __future__ import annotations

import copy
import json
import os

from . import mw3

DEFAULT_CACHE = os.environ.get("MW3_TUNE_CACHE",
                               os.path.join(os.path.expanduser("~"), ".cache", "mw3_tuning.json"))

SWEEP = dict(kin_warp=[2, 3, 1, 0], kin_fused=[0, 1, 2, 4, 8], rows_pairs=[2, 4, 8, 16], cols_tile=[8, 16, 32, 64],
             tc_persist=[4, 2, 1, 0], tc_tma=[0, 1], flush_tc=[1, 0], prod_gather=[1, 0],
             kb=[32, 64, 128])
RADIAL = ["kinetic_rows", "kinetic_cols", "kinetic_radial"]
CONTROLS = dict(kin_warp=RADIAL, kin_fused=RADIAL, rows_pairs=["kinetic_rows"],
                cols_tile=["kinetic_cols"],
                tc_persist=["angular_tc", "gamma_to_dvr", "gamma_update"], tc_tma=["angular_tc"],
                flush_tc=["sums_flush"], prod_gather=["products"], kb=["sums_flush"])


def shape_key(cfg: dict, precision: str) -> str:
    g = cfg["grid"]
    nblk = sum(min(J, cfg["omega_max"]) + 1 for J in cfg["J"]) * cfg["nelec"]
    return (f"{precision}:NR{g['NR']}:nr{g['nr']}:ng{g['ngamma']}:blk{nblk}:"
            f"nE{cfg['analysis']['nE']}")


def load_cache(path=DEFAULT_CACHE) -> dict:
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def save_cache(cache: dict, path=DEFAULT_CACHE):
    os.makedirs(os.path.dirname(path) or ".", exist_ok=True)
    tmp = path + ".tmp"
    with open(tmp, "w") as f:
        json.dump(cache, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def _time_setting(cfg, precision, setting, steps, device):
    pr = mw3.Propagator(cfg, device=device, precision=precision, tuning=setting)
    pr.propagate(2)                       # first-iteration and set-up effects
    pr.kernel_times(enable=True)
    pr.propagate(steps)
    t = pr.kernel_times()
    pr.close()
    return {k: ms for k, (ms, n) in t.items() if n}


def tune(cfg: dict, precision: str = "mixed", steps: int = 0, device: int = 0,
         cache_path: str = DEFAULT_CACHE, force: bool = False, verbose: bool = False) -> dict:
    """Best launch shapes for this workload shape (measured once, then cached)."""
    key = shape_key(cfg, precision)
    cache = load_cache(cache_path)
    if key in cache and not force:
        return dict(cache[key]["best"])
    best = {}
    report = {}
    for knob, values in SWEEP.items():
        scores = {}
        for v in values:
            setting = dict(best)
            setting[knob] = v
            # a flush costs the same however much of the ring is filled, so the
            # ring-depth sweep always runs whole rings
            n = max(steps, 2 * v) if knob == "kb" else (steps or 8)
            try:
                ms = _time_setting(cfg, precision, setting, n, device)
            except mw3.MW3Error:
                continue
            scores[v] = sum(ms.get(k, 0.0) for k in CONTROLS[knob]) / n
            if verbose:
                print(f"tune {knob}={v}: {scores[v]:.4f} ms/step")
        if scores:
            best[knob] = min(scores, key=scores.get)
            report[knob] = {str(k): round(s, 5) for k, s in scores.items()}
    cache[key] = dict(best=best, ms_per_step=report)
    save_cache(cache, cache_path)
    return dict(best)
