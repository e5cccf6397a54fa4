"""CUDA-graph mode of dd_step (CG loop as a conditional WHILE node, refinement
passes as conditional IF nodes) reproduces the eager launches bit for bit."""
import json
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2204_13254_gb300 import dd as D
from paper_2204_13254_gb300 import workloads as W

pytestmark = pytest.mark.gpu
GOLD = os.path.join(os.path.dirname(__file__), "golden")


def march(w, dt, n, prm, stats=True):
    fs = D.FieldSolver(w.xyz, w.tets, w.part, w.n_sub, w.eps, w.mu, prm).bind()
    fs.factor(dt)
    dofs = fs.dof_of_pairs(w.source_pairs)
    d2g = w.d2G(dt, n)
    sv = torch.zeros(fs.n_dof, dtype=torch.float64, device="cuda")
    out = torch.empty_like(sv)
    F, S = [], []
    for k in range(n):
        sv.zero_()
        sv[dofs] = float(d2g[k])
        st = fs.step(sv, out, stats=stats)
        S.append((st["iters"], st["refinements"], st["status"]))
        F.append(out.cpu().numpy().copy())
    fs.close()
    return np.array(F), S


@pytest.mark.parametrize("prec,warm", [(D.DD_FP64, 1), (D.DD_MIXED, 1), (D.DD_FP64, 2), (D.DD_MIXED, 2)])
def test_graph_equals_eager(prec, warm):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    w = W.config(1)
    dt = json.load(open(os.path.join(GOLD, "cfl_dt.json")))["config1"]["dt"]
    kw = dict(precision=prec, tol=1e-12 if prec == D.DD_FP64 else 1e-6, refine_tol=1e-12, max_refine=5, warm_start=warm)
    Fe, Se = march(w, dt, 40, D.make_params(**kw, chunk=8, use_graph=0))
    Fg, Sg = march(w, dt, 40, D.make_params(**kw, chunk=2, use_graph=1))
    assert np.array_equal(Fe, Fg)
    assert Se == Sg


def test_graph_ragged_and_no_stats():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    nx, ny, nz = 8, 6, 6
    L = (1.2, 1.0, 1.0)
    xyz, tets = W.kuhn_box(nx, ny, nz, *L)
    xyz, rng = W.jitter_nodes(xyz, L[0] / nx, L, 0.2, seed=5)
    part = W.rcb_partition(W.tet_centroids(xyz, tets), 7, rng.uniform(0.6, 1.4, size=7))
    w = W.Workload("ragged", xyz, tets, part, 7, None, 1.0, 30, W.z_line_node_pairs(nx, ny, nz, 4, 3))
    dt = 0.03
    Fe, _ = march(w, dt, 30, D.make_params(tol=1e-12))
    Fg, _ = march(w, dt, 30, D.make_params(tol=1e-12, use_graph=1, chunk=1), stats=False)
    assert np.array_equal(Fe, Fg)


@pytest.mark.parametrize("ws", [0, 1, 5])
def test_packed_forms_are_deterministic(ws):
    """Two marches of the same mixed-precision problem with every packed kind on one
    kernel form give bitwise equal fields (fixed summation order, no races), on a
    cavity whose subdomains span many tiles (8^3-cube subdomains)."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    w = W.cavity(16, 2, steps=12)
    dt = 0.03
    fs = D.FieldSolver(w.xyz, w.tets, w.part, w.n_sub,
                       params=D.make_params(precision=D.DD_MIXED, tol=1e-5, refine_tol=1e-10, max_refine=6,
                                            solver=D.DD_SOLVER_COUPLED_GMRES)).bind()
    fs.factor(dt)
    for kind in ("local", "recover", "iface_rows", "coupled"):
        # the persistent form: one consumer group where x and y of a whole subdomain are staged
        # (local solve, recovery), two groups (a ring depth that is a multiple of 2) for the others
        cl, st = ((1, 3) if kind in ("local", "recover") else (2, 4)) if ws == 5 else (2, 3)
        D.dd_set_sym_config(fs.h, kind, cl, st, 0, ws)
    pat = torch.zeros(fs.n_dof, dtype=torch.float64, device="cuda")
    pat[torch.as_tensor(fs.dof_of_pairs(w.source_pairs), device="cuda")] = 1.0
    d2g = w.d2G(dt, 12)
    zero = torch.zeros(fs.n_dof, dtype=torch.float64, device="cuda")
    runs = []
    for _ in range(2):
        fs.set_state(zero, zero, 0)
        out = torch.empty_like(zero)
        its = []
        for k in range(12):
            its.append(D.dd_step_scaled(fs.h, pat, d2g[k], out)["iters"])
        runs.append((out.clone(), its))
    fs.close()
    assert torch.equal(runs[0][0], runs[1][0])
    assert runs[0][1] == runs[1][1]
