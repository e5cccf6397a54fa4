"""GPU coupled MFETI-DP1 solve (Eqs. F1lr + F1uc, restarted GMRES with the
diagonal preconditioner) against the CPU FP64 oracle.

* the coupled operator (dd_coupled_apply) equals the oracle's to 1e-12;
* at the paper's setting (GMRES(20), tol 1e-6) single cold-start solves take
  the same number of Arnoldi steps as the oracle's GMRES (the GPU
  orthogonalises with classical Gram-Schmidt applied twice, the oracle with
  modified Gram-Schmidt: the same iterates up to rounding, so only a residual
  that lands on the threshold can differ), and a warm-started march agrees
  with the oracle's to the tolerance;
* with a tight tolerance and a short restart (several cycles per solve) the
  fields equal the monolithic sparse-direct march;
* the CUDA-graph form (nested conditional WHILE nodes) reproduces the eager
  launches bit for bit;
* full size (48^3 cavity, 512 subdomains): step residual and Gauss law at the
  level the tolerance implies;
* bad parameters and an exhausted iteration budget come back as status codes.
"""
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


def need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def gmres_params(**kw):
    kw.setdefault("tol", 1e-6)
    kw.setdefault("restart", 20)
    return D.make_params(solver=D.DD_SOLVER_COUPLED_GMRES, **kw)


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


def oracle_dd(w, dt, n, tol, restart):
    space = fem.EdgeSpace(w.xyz, w.tets, w.eps, w.mu)
    m = odd.DDMaps(space, w.part, w.n_sub)
    src = np.zeros(space.n)
    src[space.dof_of_pairs(w.source_pairs)] = 1.0
    return odd.run(space, m, dt, src, w.d2G(dt, n), n, tol=tol, keep=True, solver="gmres", restart=restart)


def rel_err(a, b):
    return np.linalg.norm(a - b, axis=-1) / np.maximum(np.linalg.norm(b, axis=-1), 1e-300)


def test_coupled_operator_matches_oracle():
    need_gpu()
    w = W.cavity(6, 3)
    dt = 0.05
    space = fem.EdgeSpace(w.xyz, w.tets)
    m = odd.DDMaps(space, w.part, w.n_sub)
    solver = odd.DDSolver(space, m, dt)
    fs = D.FieldSolver(w.xyz, w.tets, w.part, w.n_sub).bind()
    fs.factor(dt)
    assert m.n_corner > 0
    rng = np.random.default_rng(0)
    for _ in range(3):
        u = rng.standard_normal(m.n_lambda + m.n_corner)
        got = fs.coupled_apply(torch.tensor(u, device="cuda")).cpu().numpy()
        ref = solver.coupled_apply(u)
        assert np.linalg.norm(got - ref) <= 1e-12 * np.linalg.norm(ref)
    fs.close()


def test_paper_setting_march_matches_oracle_gmres():
    """GMRES(20), tol 1e-6, diagonal preconditioner, warm start: config-1 cavity.

    The library solves each step for the increment delta = e^{n+1} - 2e^n + e^{n-1}
    (A delta = -dt^2 S e^n - d2g), the oracle march for e^{n+1} itself: the warm
    starts differ, so per-step counts agree only to a few steps here; the
    single-solve test below compares them exactly."""
    need_gpu()
    w = W.config(1)
    dt = DT["config1"]["dt"]
    n = 25
    ref = oracle_dd(w, dt, n, 1e-6, 20)
    F, S = march(w, dt, n, gmres_params())
    its = np.array([s[0] for s in S])
    assert all(s[2] == 0 for s in S)
    assert np.all(np.abs(its - ref["iters"]) <= 3), (its, ref["iters"])
    err = rel_err(F, ref["fields"])
    assert err[2:].max() <= 2e-5, err.max()


def test_single_solves_same_arnoldi_counts_as_oracle():
    """Cold-start solves of the increment system from random states: the GPU and
    the oracle run GMRES(20) on the same coupled system, so the Arnoldi counts
    are equal (one count may differ by one if a residual lands on the
    threshold) and the increments agree to rounding when the counts do."""
    need_gpu()
    w = W.config(1)
    dt = DT["config1"]["dt"]
    space = fem.EdgeSpace(w.xyz, w.tets, w.eps, w.mu)
    m = odd.DDMaps(space, w.part, w.n_sub)
    solver = odd.DDSolver(space, m, dt)
    src = np.zeros(space.n)
    src[space.dof_of_pairs(w.source_pairs)] = 1.0
    fs = D.FieldSolver(w.xyz, w.tets, w.part, w.n_sub, w.eps, w.mu, gmres_params(warm_start=0)).bind()
    fs.factor(dt)
    rng = np.random.default_rng(4)
    out = torch.empty(fs.n_dof, dtype=torch.float64, device="cuda")
    same, total = 0, 6
    for trial in range(total):
        e_n, e_nm1 = rng.standard_normal(space.n), rng.standard_normal(space.n)
        amp = rng.uniform(-1, 1)
        fs.set_state(torch.tensor(e_n, device="cuda"), torch.tensor(e_nm1, device="cuda"), 0)
        sv = torch.tensor(amp * src, device="cuda")
        st = fs.step(sv, out)
        delta = out.cpu().numpy() - 2 * e_n + e_nm1
        b = solver.newmark_rhs(e_n, 2 * e_n, amp * src)          # (B - 2A) e^n - d2g = -dt^2 S e^n - d2g
        x, _, _, it, _ = solver.solve(b, tol=1e-6, warm=False, solver="gmres", restart=20)
        ref = solver.gather_global(x)
        assert abs(st["iters"] - it) <= 1, (st["iters"], it)
        if st["iters"] == it:
            same += 1
            assert np.linalg.norm(delta - ref) <= 1e-9 * np.linalg.norm(ref)
        else:
            assert np.linalg.norm(delta - ref) <= 1e-5 * np.linalg.norm(ref)
    assert same >= total - 1
    fs.close()


def test_restarted_tight_equals_monolithic():
    """restart 5: every solve runs several cycles; tol 1e-12 reaches the monolithic fields."""
    need_gpu()
    nx, ny, nz = 8, 6, 6
    L = (1.2, 1.0, 1.0)
    xyz, tets = W.kuhn_box(nx, ny, nz, *L)
    xyz, rng = W.jitter_nodes(xyz, L[0] / nx, L, 0.2, seed=5)
    part = W.rcb_partition(W.tet_centroids(xyz, tets), 7, rng.uniform(0.6, 1.4, size=7))
    w = W.Workload("ragged", xyz, tets, part, 7, rng.uniform(1, 4, size=len(tets)), 1.0, 30,
                   W.z_line_node_pairs(nx, ny, nz, 4, 3))
    space = fem.EdgeSpace(xyz, tets, w.eps)
    T, S = space.assemble()
    dt = 2.0 * newmark.cfl_dt(T, S)
    n = 30
    src = np.zeros(space.n)
    src[space.dof_of_pairs(w.source_pairs)] = 1.0
    mono = newmark.run(T, S, dt, src, w.d2G(dt, n), n, keep=True)
    F, St = march(w, dt, n, gmres_params(tol=1e-12, restart=5, max_it=2000))
    assert all(s[2] == 0 for s in St)
    assert max(s[0] for s in St) > 10                         # several restart cycles per solve
    assert rel_err(F, mono["fields"])[2:].max() <= 1e-9
    ref = oracle_dd(w, dt, n, 1e-12, 5)
    its = np.array([s[0] for s in St])
    assert np.all(np.abs(its - ref["iters"]) <= 2), (its, ref["iters"])


def test_graph_equals_eager():
    need_gpu()
    w = W.config(1)
    dt = DT["config1"]["dt"]
    prm = dict(tol=1e-10, restart=8)
    Fe, Se = march(w, dt, 30, gmres_params(**prm, chunk=8, use_graph=0))
    Fg, Sg = march(w, dt, 30, gmres_params(**prm, chunk=2, use_graph=1))
    assert np.array_equal(Fe, Fg)
    assert Se == Sg
    Fn, _ = march(w, dt, 30, gmres_params(**prm, chunk=3, use_graph=1), stats=False)
    assert np.array_equal(Fe, Fn)


@pytest.mark.parametrize("graph", [0, 1])
def test_mixed_precision_matches_monolithic(graph):
    """FP32 coupled GMRES inside the FP64 refinement of the step system: fields
    within 1e-8 of the monolithic march, eager and graph bit for bit alike."""
    need_gpu()
    w = W.config(1)
    dt = DT["config1"]["dt"]
    n = 40
    space = fem.EdgeSpace(w.xyz, w.tets, w.eps, w.mu)
    T, S = space.assemble()
    src = np.zeros(space.n)
    src[space.dof_of_pairs(w.source_pairs)] = 1.0
    mono = newmark.run(T, S, dt, src, w.d2G(dt, n), n, keep=True)
    kw = dict(precision=D.DD_MIXED, tol=1e-5, refine_tol=1e-12, max_refine=6)
    F, St = march(w, dt, n, gmres_params(**kw, use_graph=graph, chunk=8 if graph == 0 else 2))
    assert all(s[2] == 0 for s in St)
    assert all(s[1] >= 2 for s in St[3:])                  # FP32 solves refined in FP64
    assert rel_err(F, mono["fields"])[2:].max() <= 1e-8
    if graph:
        Fe, Se = march(w, dt, n, gmres_params(**kw, use_graph=0, chunk=8))
        assert np.array_equal(F, Fe)
        assert St == Se


def test_parameter_errors_and_budget():
    need_gpu()
    w = W.config(1)
    dt = DT["config1"]["dt"]
    fs = D.FieldSolver(w.xyz, w.tets, w.part, w.n_sub).bind()
    fs.factor(dt)
    for bad in (gmres_params(restart=0),
                gmres_params(restart=D.DD_MAX_RESTART + 1), gmres_params(warm_start=3),
                D.make_params(solver=7)):
        with pytest.raises(D.DDError) as ei:
            fs.set_params(bad)
        assert ei.value.code == D.DD_ERR_ARG
    dofs = fs.dof_of_pairs(w.source_pairs)
    sv = torch.zeros(fs.n_dof, dtype=torch.float64, device="cuda")
    out = torch.empty_like(sv)
    d2g = w.d2G(dt, 30)
    for graph in (0, 1):
        fs.set_params(gmres_params(tol=1e-12, max_it=3, use_graph=graph))
        fs.set_state(torch.zeros_like(sv), torch.zeros_like(sv), 0)
        sv.zero_()
        sv[dofs] = float(d2g[25])
        st = fs.step(sv, out, raise_on_error=False)
        assert st["status"] == D.DD_ERR_NO_CONVERGENCE and st["iters"] == 3
        assert torch.isfinite(out).all()
        bad = sv.clone()
        bad[dofs[0]] = float("nan")
        fs.set_params(gmres_params(tol=1e-10, use_graph=graph))
        st = fs.step(bad, out, raise_on_error=False)
        assert st["rc"] == D.DD_ERR_NONFINITE
    # the handle stays usable
    fs.set_params(gmres_params(tol=1e-10))
    fs.set_state(torch.zeros_like(sv), torch.zeros_like(sv), 0)
    st = fs.step(sv, out)
    assert st["status"] == 0
    fs.close()


def test_fullsize_cavity48():
    """48^3 cavity, 512 subdomains, graph mode: GMRES(20) tol 1e-6 in FP64 (the paper's
    setting) and FP32 GMRES under FP64 refinement to 1e-10 (the bench's mixed
    configuration).  Step residual <= its bound and Gauss law <= 1e3 x that
    bound, both evaluated by the oracle's assembled matrices."""
    need_gpu()
    w = W.config(4)
    dt = DT["config4"]["dt"]
    n = 20
    space = fem.EdgeSpace(w.xyz, w.tets, w.eps, w.mu)
    T, S = space.assemble()
    A, B = newmark.newmark_matrices(T, S, dt)
    D0 = space.gradient_matrix()
    src = np.zeros(space.n)
    src[space.dof_of_pairs(w.source_pairs)] = 1.0
    d2g = w.d2G(dt, n)
    runs = [(gmres_params(tol=1e-6, use_graph=1, chunk=4), 1e-6),
            (gmres_params(precision=D.DD_MIXED, tol=1e-5, refine_tol=1e-10, max_refine=6, use_graph=1, chunk=2), 1e-9)]
    for prm, bound in runs:
        F, St = march(w, dt, n, prm)
        assert all(s[2] == 0 for s in St)
        f = [np.zeros(space.n), np.zeros(space.n)] + list(F)
        worst = gauss = 0.0
        for k in range(n):
            r = A @ f[k + 2] - B @ f[k + 1] + A @ f[k] + d2g[k] * src
            scale = np.linalg.norm(B @ f[k + 1]) + np.linalg.norm(A @ f[k]) + np.linalg.norm(d2g[k] * src)
            worst = max(worst, np.linalg.norm(r) / scale)
            Te = T @ f[k + 2]
            gauss = max(gauss, np.abs(D0.T @ Te).max() / max(np.abs(Te).max(), 1e-300))
        assert worst <= bound, (prm.precision, worst)
        assert gauss <= 1e3 * bound, (prm.precision, gauss)
