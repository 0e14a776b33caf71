"""Write ``fullsize_fix.json``: the FP64 oracle's own fix of the full-size
synthetic workloads, so GPU tests at those sizes can compare their final
functional F with the oracle's.

Calls only the oracle (``oracle/lgf_oracle.py``) and the seeded input
generator (``lgf_inputs``); nothing here comes from the CUDA path.  The
method (steepest descent with Fourier acceleration, paper Sec. 1) has no
closed-form end point, so the stored values are the oracle's: the number of
updates it applied, F and theta of its final links, with theta < 1e-15.

Cases (lattice, seed, link scale; gauge scale 1.0, alpha 0.08):
* the single 32^4 lattice, link scale 0.5, seed 0;
* the paper-shaped finite-temperature lattices 48^3 x 8 and 48^3 x 12, link
  scale 0.6, seed 0;
* the first member of each shape of the 64-lattice mixed batch: member i
  has seed i and shape (16^4, 24^3 x 48, 32^3 x 8, 20^4)[i mod 4], link
  scale 0.5.

Usage: ``python tests/golden/make_fullsize_fix.py [--jobs N] [case ...]``.
Each case runs in its own process (started with ``spawn``); the 32^4 case
takes a few minutes on one core.  Existing entries of the JSON file are kept
unless recomputed.
"""
from __future__ import annotations

import argparse
import json
import multiprocessing as mp
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
OUT = os.path.join(HERE, "fullsize_fix.json")

ALPHA = 0.08
TOL = 1e-15
MAX_ITER = 2000

CASES = {
    "32^4": ((32, 32, 32, 32), 0, 0.5),
    "48^3x8": ((48, 48, 48, 8), 0, 0.6),
    "48^3x12": ((48, 48, 48, 12), 0, 0.6),
    "batch member 0 16^4": ((16, 16, 16, 16), 0, 0.5),
    "batch member 1 24^3x48": ((24, 24, 24, 48), 1, 0.5),
    "batch member 2 32^3x8": ((32, 32, 32, 8), 2, 0.5),
    "batch member 3 20^4": ((20, 20, 20, 20), 3, 0.5),
}


def run_case(name: str) -> tuple[str, dict]:
    if ROOT not in sys.path:
        sys.path.insert(0, ROOT)
    import lgf_inputs as I
    from oracle import lgf_oracle as O

    dims, seed, scale = CASES[name]
    U = I.synthetic_config(dims, seed=seed, link_scale=scale, gauge_scale=1.0)
    F0, th0 = O.functional(U)
    t0 = time.perf_counter()
    res = O.fix(U, TOL, MAX_ITER, ALPHA)
    dt = time.perf_counter() - t0
    return name, {
        "dims": list(dims), "seed": seed, "link_scale": scale, "gauge_scale": 1.0,
        "alpha": ALPHA, "theta_tol": TOL,
        "iterations": res["iterations"], "converged": bool(res["converged"]),
        "F": res["F"], "theta": res["theta"], "F_input": F0, "theta_input": th0,
        "oracle_seconds": round(dt, 1),
    }


def main() -> None:
    ap = argparse.ArgumentParser()
    ap.add_argument("cases", nargs="*", default=list(CASES))
    ap.add_argument("--jobs", type=int, default=2)
    args = ap.parse_args()
    for c in args.cases:
        if c not in CASES:
            raise SystemExit(f"unknown case {c!r}; known: {list(CASES)}")
    data = {}
    if os.path.exists(OUT):
        with open(OUT) as f:
            data = json.load(f)
    data.setdefault("source", (
        "FP64 oracle (oracle/lgf_oracle.py, fix) on the seeded synthetic inputs "
        "(lgf_inputs.synthetic_config); written by tests/golden/make_fullsize_fix.py"))
    data.setdefault("cases", {})
    ctx = mp.get_context("spawn")
    with ctx.Pool(max(1, min(args.jobs, len(args.cases)))) as pool:
        for name, rec in pool.imap_unordered(run_case, args.cases):
            print(f"{name}: {rec['iterations']} iterations, F = {rec['F']!r}, "
                  f"theta = {rec['theta']:.3e}, {rec['oracle_seconds']} s", flush=True)
            data["cases"][name] = rec
            with open(OUT, "w") as f:
                json.dump(data, f, indent=1, sort_keys=True)
                f.write("\n")


if __name__ == "__main__":
    main()
