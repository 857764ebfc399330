"""Write the time-to-fit targets: the FP64 oracle's converged global Fit on
the seeded synthetic workloads.

Only the oracle and the seeded input generator are called.  The data are
the FP32 tensors the benchmark uploads (upcast to FP64), the initial factors
are the benchmark's, and the run is plain CoNCPD-APG (Algorithm 1) with the
termination rule of Section III-C (|RelErr_k - RelErr_{k-1}| < 1e-8, at most
1000 iterations).  Fit = 1 - RelErr (Section IV settings).

    python tests/golden/make_fit_targets.py [workload ...]

writes tests/golden/fit_targets.json (one record per workload).
"""

import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

from oracle import cncpd_oracle as O  # noqa: E402
import synth  # noqa: E402

OUT = os.path.join(HERE, "fit_targets.json")


def target(name, eps=1e-8, max_it=1000):
    w = synth.workload(name)
    Xs, _ = synth.make_tensors(w, dtype=np.float32)
    X64 = [X.astype(np.float64) for X in Xs]
    del Xs
    U0 = synth.init_factors(w.dims, w.R, w.seed)
    prob = O.Problem(X64, [w.R] * w.K, w.L)
    fits = []
    t0 = time.perf_counter()

    def progress(it, st, info):
        fits.append(1.0 - info["relerr"])
        if it % 10 == 0:
            print(f"{name}: iteration {it}, fit {fits[-1]:.9f}, {time.perf_counter() - t0:.0f} s",
                  file=sys.stderr, flush=True)

    res = O.apg(prob, U0, max_it=max_it, eps=eps, callback=progress)
    dt = time.perf_counter() - t0
    return {
        "workload": name, "seed": w.seed, "K": w.K, "dims": [list(d) for d in w.dims], "R": w.R, "L": w.L,
        "data": "synth.make_tensors(dtype=float32) upcast to float64; synth.init_factors(seed)",
        "eps": eps, "max_it": max_it, "iterations": res["iters"],
        "reupdates": int(sum(res["hist"]["redo"])),
        "fit": fits[-1],
        "first_iteration_within_1e-4": next(i + 1 for i, f in enumerate(fits) if f >= fits[-1] - 1e-4),
        "oracle_seconds": dt,
    }


def main():
    names = sys.argv[1:] or ["bf16_512x512x256"]
    table = {}
    if os.path.exists(OUT):
        with open(OUT) as f:
            table = json.load(f)
    for name in names:
        rec = target(name)
        table[name] = rec
        print(json.dumps(rec), flush=True)
        with open(OUT, "w") as f:
            json.dump(table, f, indent=1, sort_keys=True)
            f.write("\n")


if __name__ == "__main__":
    main()
