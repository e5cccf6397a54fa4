"""Full-size GPU runs checked by properties that hold at any size.

The oracle cannot march these meshes step by step in seconds, so each GPU field
is checked against the recurrence itself, assembled independently by the
oracle: the FP64 residual A e^{k+1} - B e^k + A e^{k-1} + d2g^k relative to the
size of the right-hand side, and the discrete Gauss law D0^T T e^k (the z-line
current closes on the PEC walls, so no charge is deposited).  Same launch
configuration as bench.py (same workload, dt, precision modes).
"""
import json
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import fem, newmark
from paper_2204_13254_gb300 import dd as D
from paper_2204_13254_gb300 import workloads as W

pytestmark = pytest.mark.gpu
GOLD = os.path.join(os.path.dirname(__file__), "golden")
DT = json.load(open(os.path.join(GOLD, "cfl_dt.json")))


def run_and_check(cfg, n_steps, runs, autotune=False):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    w = W.config(cfg)
    dt = DT[f"config{cfg}"]["dt"]
    space = fem.EdgeSpace(w.xyz, w.tets, w.eps, w.mu)
    T, S = space.assemble()
    A, B = newmark.newmark_matrices(T, S, dt)
    D0 = space.gradient_matrix()
    src = np.zeros(space.n)
    src[space.dof_of_pairs(w.source_pairs)] = 1.0
    d2g = w.d2G(dt, n_steps)
    fs = D.FieldSolver(w.xyz, w.tets, w.part, w.n_sub, w.eps, w.mu).bind()
    fs.factor(dt)
    if autotune:
        D.dd_autotune(fs.h, None)
    dofs = fs.dof_of_pairs(w.source_pairs)
    sv = torch.zeros(fs.n_dof, dtype=torch.float64, device="cuda")
    out = torch.empty_like(sv)
    results = {}
    for name, prm, bound in runs:
        fs.set_params(prm)
        fs.set_state(torch.zeros_like(sv), torch.zeros_like(sv), 0)
        f = [np.zeros(fs.n_dof), np.zeros(fs.n_dof)]
        worst, gauss = 0.0, 0.0
        for k in range(n_steps):
            sv.zero_()
            sv[dofs] = float(d2g[k])
            st = fs.step(sv, out)
            assert st["status"] == 0
            f.append(out.cpu().numpy().copy())
            r = A @ f[-1] - B @ f[-2] + A @ f[-3] + d2g[k] * src
            scale = np.linalg.norm(B @ f[-2]) + np.linalg.norm(A @ f[-3]) + np.linalg.norm(d2g[k] * src)
            worst = max(worst, np.linalg.norm(r) / scale)
            Te = T @ f[-1]
            gauss = max(gauss, np.abs(D0.T @ Te).max() / max(np.abs(Te).max(), 1e-300))
        assert worst <= bound, (name, worst)
        assert gauss <= 1e3 * bound, (name, gauss)
        results[name] = (worst, gauss, np.array(f[2:]))
    fs.close()
    return results


def test_config4_cavity48_fp64_and_mixed():
    res = run_and_check(4, 30, [("fp64", D.make_params(tol=1e-12), 1e-11),
                                ("mixed", D.make_params(precision=D.DD_MIXED, tol=1e-5, refine_tol=1e-10,
                                                        max_refine=6), 1e-9)])
    f64, f32 = res["fp64"][2], res["mixed"][2]
    rel = np.linalg.norm(f32[-1] - f64[-1]) / np.linalg.norm(f64[-1])
    assert rel <= 1e-8, rel


def test_config3_jittered_rcb300_fp64():
    run_and_check(3, 12, [("fp64", D.make_params(tol=1e-12), 1e-11)])


def test_config4_bench_launch_configuration():
    """The configuration bench.py times: autotuned tiles, CUDA-graph steps, both precisions."""
    res = run_and_check(4, 30, [("fp64", D.make_params(tol=1e-10, use_graph=1, chunk=2), 1e-9),
                                ("mixed", D.make_params(precision=D.DD_MIXED, tol=1e-5, refine_tol=1e-10,
                                                        max_refine=6, use_graph=1, chunk=2), 1e-9)], autotune=True)
    f64, f32 = res["fp64"][2], res["mixed"][2]
    assert np.linalg.norm(f32[-1] - f64[-1]) / np.linalg.norm(f64[-1]) <= 1e-8
