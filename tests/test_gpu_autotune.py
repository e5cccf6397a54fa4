"""GEMV tile autotuner: picks valid tiles, keeps results (up to summation order)
and reuses its on-disk cache."""
import json
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2204_13254_gb300 import dd as D
from paper_2204_13254_gb300 import workloads as W

pytestmark = pytest.mark.gpu
GOLD = os.path.join(os.path.dirname(__file__), "golden")


def run(fs, w, dt, n):
    fs.set_state(torch.zeros(fs.n_dof, dtype=torch.float64, device="cuda"),
                 torch.zeros(fs.n_dof, dtype=torch.float64, device="cuda"), 0)
    dofs = fs.dof_of_pairs(w.source_pairs)
    d2g = w.d2G(dt, n)
    sv = torch.zeros(fs.n_dof, dtype=torch.float64, device="cuda")
    out = torch.empty_like(sv)
    for k in range(n):
        sv.zero_()
        sv[dofs] = float(d2g[k])
        fs.step(sv, out)
    return out.cpu().numpy()


def test_autotune_results_and_cache(tmp_path):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    w = W.config(1)
    dt = json.load(open(os.path.join(GOLD, "cfl_dt.json")))["config1"]["dt"]
    for prm in (D.make_params(tol=1e-13), D.make_params(precision=D.DD_MIXED, tol=1e-6, refine_tol=1e-12, max_refine=6,
                                                        use_graph=1)):
        fs = D.FieldSolver(w.xyz, w.tets, w.part, w.n_sub, params=prm).bind()
        fs.factor(dt)
        ref = run(fs, w, dt, 30)
        cache = str(tmp_path / "tiles.txt")
        t1 = D.dd_autotune(fs.h, cache)
        tiles = D.dd_get_tiles(fs.h)
        for p in tiles.values():
            for lpr, rows in p.values():
                assert lpr in (8, 16, 32) and rows in (8, 16, 32, 64, 128)
        got = run(fs, w, dt, 30)
        assert np.linalg.norm(got - ref) <= 1e-10 * np.linalg.norm(ref)
        D.dd_autotune(fs.h, cache)               # complete cache entry: tiles read back, no timing
        assert D.dd_get_tiles(fs.h) == tiles
        # one line per dense kind and precision, one per packed kind (cluster size, ring depth, L2 kept, form)
        assert sum(1 for _ in open(cache)) == 2 * len(D.GEMV_KINDS) + len(D.dd_get_sym_config(fs.h))
        fs.close()
