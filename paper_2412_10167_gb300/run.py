"""Command-line runner: propagate one of the synthetic workloads for a number of
Chebyshev iterations and print the step rate and the summed probabilities.

  python -m paper_2412_10167_gb300.run --config c2 --precision mixed --steps 3

Configurations: c1, c2, c3, c4 (the full workloads), c1, c2s, c3s, c4s (their
parity-sized copies) and c2p (the config-2 grid with 8 blocks and 16 energies, the
kernel-profiling case). The step rate printed here is wall-clock around
mw3_propagate (synchronous) and includes graph capture on the first full chunk; the
timed measurement is bench.py.
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np


def main(argv=None):
    import workloads as W
    from . import mw3
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--config", default="c2")
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--tuning", default=None, help="JSON dictionary of mw3_set_tuning keys")
    ap.add_argument("--compare", action="store_true",
                    help="also run the FP64 path and report max |dP| of the mixed form")
    args = ap.parse_args(argv)
    table = dict(W.CONFIGS)
    table.update(W.SMALL)
    table.update(W.PROFILE)
    cfg = table[args.config]
    tuning = json.loads(args.tuning) if args.tuning else None
    pr = mw3.Propagator(cfg, precision=args.precision, tuning=tuning)
    t0 = time.perf_counter()
    pr.propagate(args.steps)
    dt = time.perf_counter() - t0
    E, P, _ = pr.probabilities()
    out = dict(config=cfg["name"], precision=args.precision, steps=args.steps,
               steps_per_s=args.steps / dt, iteration=pr.iteration,
               P_total_max=float(np.max(P)))
    has_prod = bool(cfg["analysis"].get("products"))
    if has_prod:
        out["P_products_max"] = float(np.max(pr.product_probabilities().sum(axis=(1, 2, 3))))
    if args.compare:
        Pp = pr.product_probabilities() if has_prod else None
        _, _, Pin = pr.probabilities()
        ref = mw3.Propagator(cfg, precision="fp64", tuning=tuning)
        t0 = time.perf_counter()
        ref.propagate(args.steps)
        out["fp64_steps_per_s"] = args.steps / (time.perf_counter() - t0)
        _, P64, Pin64 = ref.probabilities()
        out["max_abs_dP"] = {"total": float(np.max(np.abs(P - P64))),
                             "reactant_channels": float(np.max(np.abs(Pin - Pin64)))
                             if Pin is not None else None}
        out["max_P"] = {"total": float(np.max(np.abs(P64))),
                        "reactant_channels": float(np.max(np.abs(Pin64))) if Pin64 is not None else None}
        if has_prod:
            Pp64 = ref.product_probabilities()
            out["max_abs_dP"]["product_channels"] = float(np.max(np.abs(Pp - Pp64)))
            out["max_P"]["product_channels"] = float(np.max(np.abs(Pp64)))
        ref.close()
    pr.close()
    print(json.dumps(out))


if __name__ == "__main__":
    main()
