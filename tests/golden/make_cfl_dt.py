"""Write tests/golden/cfl_dt.json: the explicit stability limit of each workload.

Each workload steps at dt = 2 x the explicit (central-difference,
consistent-mass) limit dt_CFL = 2 / sqrt(lambda_max(T^-1 S)).  lambda_max is
computed here by the CPU oracle only (ARPACK on the pencil (S, T)), once, and
stored so that the GPU tests and the benchmark share the same time step
without importing the oracle.

Usage: python tests/golden/make_cfl_dt.py [config ids ...]   (default: 1 2 4 5 3)
"""
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import fem, newmark  # noqa: E402
from paper_2204_13254_gb300 import workloads as W  # noqa: E402

OUT = os.path.join(HERE, "cfl_dt.json")


def main(ids):
    table = json.load(open(OUT)) if os.path.exists(OUT) else {}
    for i in ids:
        t = time.time()
        w = W.config(i)
        space = fem.EdgeSpace(w.xyz, w.tets, w.eps, w.mu)
        T, S = space.assemble()
        dt_cfl = newmark.cfl_dt(T, S)
        table[f"config{i}"] = {"workload": w.name, "n_dof": int(space.n), "dt_cfl": float(dt_cfl),
                               "dt": float(2.0 * dt_cfl)}
        print(f"config{i} {w.name}: n={space.n} dt_cfl={dt_cfl:.17g} ({time.time() - t:.1f}s)", flush=True)
        json.dump(table, open(OUT, "w"), indent=1, sort_keys=True)


if __name__ == "__main__":
    main([int(a) for a in sys.argv[1:]] or [1, 2, 4, 5, 3])
