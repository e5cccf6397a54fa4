"""The elimination's trailing updates on the tensor cores (DD_FACTOR_TENSOR: BF16
slices of the panels, exact FP32 class sums in tensor memory, FP64 combination)
give the FP64 factorisation: the Schur operator of Eq. f1schur equals the CPU
oracle's to 1e-12, the coupled operator the FP64-path's to 1e-13, and the march
equals the oracle's monolithic solve."""
import json
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import dd as odd
from oracle import fem, newmark
from paper_2204_13254_gb300 import dd as D
from paper_2204_13254_gb300 import workloads as W

pytestmark = pytest.mark.gpu
GOLD = os.path.join(os.path.dirname(__file__), "golden")
DT = json.load(open(os.path.join(GOLD, "cfl_dt.json")))
T_ = D.DD_FACTOR_TENSOR


def need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def test_tensor_factor_schur_operator_matches_oracle():
    need_gpu()
    w = W.cavity(6, 3)
    dt = 0.05
    space = fem.EdgeSpace(w.xyz, w.tets)
    m = odd.DDMaps(space, w.part, w.n_sub)
    solver = odd.DDSolver(space, m, dt)
    fs = D.FieldSolver(w.xyz, w.tets, w.part, w.n_sub, params=D.make_params(factor_mode=T_)).bind()
    fs.factor(dt)
    rng = np.random.default_rng(0)
    for _ in range(3):
        lam = rng.standard_normal(m.n_lambda)
        got = fs.schur_apply(torch.tensor(lam, device="cuda")).cpu().numpy()
        ref = solver.schur_apply(lam)
        assert np.linalg.norm(got - ref) <= 1e-12 * np.linalg.norm(ref)
    fs.close()


def _coupled(w, dt, mode, u, eps=None):
    fs = D.FieldSolver(w.xyz, w.tets, w.part, w.n_sub, eps if eps is not None else w.eps, w.mu,
                       params=D.make_params(solver=D.DD_SOLVER_COUPLED_GMRES, factor_mode=mode)).bind()
    fs.factor(dt)
    out = fs.coupled_apply(torch.tensor(u, device="cuda")).cpu().numpy()
    fs.close()
    return out


@pytest.mark.parametrize("case", ["cavity24_k4", "ragged_rcb"])
def test_tensor_factor_coupled_operator_equals_fp64_path(case):
    """Subdomains of 6^3 cubes (1854 local unknowns: fifteen 128-row blocks per
    panel), and a jittered mesh with a ragged RCB split and eps ~ U[1, 4]."""
    need_gpu()
    if case == "cavity24_k4":
        w = W.cavity(24, 4)
        dt = DT["config4"]["dt"] * 2.0
    else:
        nx, ny, nz = 10, 8, 8
        L = (1.2, 1.0, 1.0)
        xyz, tets = W.kuhn_box(nx, ny, nz, *L)
        xyz, rng = W.jitter_nodes(xyz, L[0] / nx, L, 0.2, seed=9)
        part = W.rcb_partition(W.tet_centroids(xyz, tets), 6, rng.uniform(0.6, 1.4, size=6))
        w = W.Workload("ragged", xyz, tets, part, 6, rng.uniform(1, 4, size=len(tets)), 1.0, 30,
                       W.z_line_node_pairs(nx, ny, nz, 5, 4))
        dt = 0.02
    h = D.dd_setup(w.xyz, w.tets, w.part, w.n_sub, w.eps, w.mu)
    sz = D.dd_get_sizes(h)
    D.dd_destroy(h)
    u = np.random.default_rng(3).standard_normal(int(sz.n_lambda + sz.n_corner))
    ref = _coupled(w, dt, D.DD_FACTOR_FP64, u)
    got = _coupled(w, dt, T_, u)
    assert np.linalg.norm(got - ref) <= 1e-13 * np.linalg.norm(ref), np.linalg.norm(got - ref) / np.linalg.norm(ref)


def test_tensor_factor_march_matches_monolithic():
    need_gpu()
    w = W.config(1)
    dt = DT["config1"]["dt"]
    n = 30
    space = fem.EdgeSpace(w.xyz, w.tets)
    T, S = space.assemble()
    src = np.zeros(space.n)
    src[space.dof_of_pairs(w.source_pairs)] = 1.0
    d2g = w.d2G(dt, n)
    ref = newmark.run(T, S, dt, src, d2g, n, keep=True)["fields"]
    for solver in (D.DD_SOLVER_SCHUR_CG, D.DD_SOLVER_COUPLED_GMRES):
        fs = D.FieldSolver(w.xyz, w.tets, w.part, w.n_sub,
                           params=D.make_params(tol=1e-13, solver=solver, max_it=3000, factor_mode=T_)).bind()
        fs.factor(dt)
        pat = torch.zeros(fs.n_dof, dtype=torch.float64, device="cuda")
        pat[torch.as_tensor(fs.dof_of_pairs(w.source_pairs), device="cuda")] = 1.0
        out = torch.empty_like(pat)
        worst = 0.0
        for k in range(n):
            D.dd_step_scaled(fs.h, pat, d2g[k], out)
            nr = np.linalg.norm(ref[k])
            if nr > 0:
                worst = max(worst, np.linalg.norm(out.cpu().numpy() - ref[k]) / nr)
        fs.close()
        assert worst <= 1e-10, (solver, worst)
