"""GPU parity of the MFETI-DP1 field solve against the CPU FP64 oracle.

Every test here runs the CUDA path through the C ABI (paper_2204_13254_gb300.dd)
and compares with the oracle (monolithic sparse-direct Newmark march and the
CPU DD solver) on the same seeded inputs.

Tolerances: FP64 relative L2 field error <= 1e-10 per step; DD_MIXED (FP32
application + FP64 refinement) <= 1e-8.
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


def oracle_run(w, dt, n, keep=True):
    space = fem.EdgeSpace(w.xyz, w.tets, w.eps, w.mu)
    T, S = space.assemble()
    src = np.zeros(space.n)
    src[space.dof_of_pairs(w.source_pairs)] = 1.0
    P = space.probe_operator(w.probes) if len(w.probes) else None
    out = newmark.run(T, S, dt, src, w.d2G(dt, n), n, P=P, keep=keep)
    return space, T, S, src, out


def gpu_run(w, dt, n, params, keep=True, probes=True, after_factor=None):
    fs = D.FieldSolver(w.xyz, w.tets, w.part, w.n_sub, w.eps, w.mu, params,
                       probes=w.probes if probes and len(w.probes) else None).bind()
    fs.factor(dt)
    if after_factor:
        after_factor(fs)
    dofs = fs.dof_of_pairs(w.source_pairs)
    src = torch.zeros(fs.n_dof, dtype=torch.float64, device="cuda")
    d2g = w.d2G(dt, n)
    fields, probe_vals, stats = [], [], []
    e_out = torch.empty(fs.n_dof, dtype=torch.float64, device="cuda")
    for k in range(n):
        src.zero_()
        src[dofs] = float(d2g[k])
        st = fs.step(src, e_out)
        stats.append(st)
        if keep:
            fields.append(e_out.cpu().numpy().copy())
        if probes and fs.n_probe:
            probe_vals.append(fs.probe().cpu().numpy())
    return fs, np.array(fields), np.array(probe_vals), stats


def rel_err(a, b):
    return np.linalg.norm(a - b, axis=-1) / np.maximum(np.linalg.norm(b, axis=-1), 1e-300)


def test_cavity_fp64_matches_oracle_200_steps():
    need_gpu()
    w = W.config(1)
    dt = DT["config1"]["dt"]
    n = 200
    space, T, S, src, ref = oracle_run(w, dt, n)
    fs, f, pv, stats = gpu_run(w, dt, n, D.make_params(tol=1e-13))
    err = rel_err(f, ref["fields"])
    assert err[2:].max() <= 1e-10, err.max()
    assert all(s["status"] == 0 for s in stats)
    assert np.abs(pv - ref["probes"]).max() <= 1e-10 * np.abs(ref["probes"]).max()
    # discrete Gauss law on the GPU fields (line current closes on the PEC walls: q = 0)
    D0 = space.gradient_matrix()
    gauss = max(np.abs(D0.T @ (T @ f[k])).max() for k in range(0, n, 10))
    # with DD the interface nodes carry the interface-CG residual (tol 1e-13): bound 1e-10 relative
    assert gauss <= 1e-10 * np.abs(T @ f[-1]).max()
    # energy invariant once the source is off (t > t0 + 10 sigma)
    En = np.array([newmark.energy(T, S, dt, f[k + 1], f[k]) for k in range(81, n - 1)])
    assert np.abs(En / En[0] - 1).max() < 1e-9
    fs.close()


def test_cavity_matches_oracle_dd_iterations():
    """Same torn system as the CPU DD oracle: per-step fields agree and the
    interface CG (same Jacobi preconditioner, warm start, tolerance) takes
    about the same number of iterations."""
    need_gpu()
    w = W.config(1)
    dt = DT["config1"]["dt"]
    n = 12
    space = fem.EdgeSpace(w.xyz, w.tets)
    m = odd.DDMaps(space, w.part, w.n_sub)
    src = np.zeros(space.n)
    src[space.dof_of_pairs(w.source_pairs)] = 1.0
    ref = odd.run(space, m, dt, src, w.d2G(dt, n), n, tol=1e-12, keep=True)
    fs, f, _, stats = gpu_run(w, dt, n, D.make_params(tol=1e-12), probes=False)
    err = rel_err(f, ref["fields"])
    assert err[2:].max() <= 1e-9
    gi = np.array([s["iters"] for s in stats])
    assert np.all(np.abs(gi[2:] - ref["iters"][2:]) <= 3), (gi, ref["iters"])
    fs.close()


def test_ragged_rcb_jittered_fp64():
    need_gpu()
    nx, ny, nz = 8, 6, 6
    L = (1.2, 1.0, 1.0)
    xyz, tets = W.kuhn_box(nx, ny, nz, *L)
    xyz, rng = W.jitter_nodes(xyz, L[0] / nx, L, 0.2, seed=5)
    part = W.rcb_partition(W.tet_centroids(xyz, tets), 7, rng.uniform(0.6, 1.4, size=7))
    w = W.Workload("ragged", xyz, tets, part, 7, rng.uniform(1, 4, size=len(tets)), 1.0, 40,
                   W.z_line_node_pairs(nx, ny, nz, 4, 3), probes=np.array([[0.5, 0.45, 0.52]]))
    space = fem.EdgeSpace(xyz, tets, w.eps)
    T, S = space.assemble()
    dt = 2.0 * newmark.cfl_dt(T, S)
    n = 40
    _, _, _, _, ref = oracle_run(w, dt, n)
    fs, f, pv, _ = gpu_run(w, dt, n, D.make_params(tol=1e-13))
    assert rel_err(f, ref["fields"])[2:].max() <= 1e-10
    assert np.abs(pv - ref["probes"]).max() <= 1e-10 * np.abs(ref["probes"]).max()
    fs.close()


def test_schur_operator_matches_oracle():
    need_gpu()
    w = W.cavity(6, 3)
    dt = 0.05
    space = fem.EdgeSpace(w.xyz, w.tets)
    m = odd.DDMaps(space, w.part, w.n_sub)
    solver = odd.DDSolver(space, m, dt)
    fs = D.FieldSolver(w.xyz, w.tets, w.part, w.n_sub).bind()
    fs.factor(dt)
    rng = np.random.default_rng(0)
    for _ in range(3):
        lam = rng.standard_normal(m.n_lambda)
        got = fs.schur_apply(torch.tensor(lam, device="cuda")).cpu().numpy()
        ref = solver.schur_apply(lam)
        assert np.linalg.norm(got - ref) <= 1e-12 * np.linalg.norm(ref)
    fs.close()


def test_mixed_precision_within_1e8():
    need_gpu()
    w = W.config(1)
    dt = DT["config1"]["dt"]
    n = 200
    _, _, _, _, ref = oracle_run(w, dt, n)
    prm = D.make_params(precision=D.DD_MIXED, tol=1e-6, refine_tol=1e-12, max_refine=6)
    fs, f, _, stats = gpu_run(w, dt, n, prm, probes=False)
    err = rel_err(f, ref["fields"])
    assert err[2:].max() <= 1e-8, err.max()
    assert all(s["status"] == 0 for s in stats)
    assert max(s["refinements"] for s in stats) >= 1
    fs.close()


def test_checkpoint_resume_bitwise_and_deterministic():
    need_gpu()
    w = W.config(1)
    dt = DT["config1"]["dt"]
    prm = D.make_params(tol=1e-12)
    fs, f, _, _ = gpu_run(w, dt, 30, prm, probes=False)
    fs2, f2, _, _ = gpu_run(w, dt, 30, prm, probes=False)
    assert np.array_equal(f, f2)                     # deterministic reductions
    # resume from step 15 of a second solver: identical remaining trajectory
    fs3 = D.FieldSolver(w.xyz, w.tets, w.part, w.n_sub, params=D.make_params(tol=1e-12, warm_start=0)).bind()
    fs3.factor(dt)
    fs4 = D.FieldSolver(w.xyz, w.tets, w.part, w.n_sub, params=D.make_params(tol=1e-12, warm_start=0)).bind()
    fs4.factor(dt)
    dofs = fs3.dof_of_pairs(w.source_pairs)
    d2g = w.d2G(dt, 30)
    src = torch.zeros(fs3.n_dof, dtype=torch.float64, device="cuda")
    out3 = torch.empty_like(src)
    traj = []
    for k in range(30):
        src.zero_(); src[dofs] = float(d2g[k])
        fs3.step(src, out3)
        traj.append(out3.cpu().numpy().copy())
        if k == 14:
            a, b, step = fs3.get_state()
            fs4.set_state(a, b, step)
    out4 = torch.empty_like(src)
    for k in range(15, 30):
        src.zero_(); src[dofs] = float(d2g[k])
        fs4.step(src, out4)
    assert np.array_equal(out4.cpu().numpy(), traj[-1])
    for x in (fs, fs2, fs3, fs4):
        x.close()


def test_error_status_without_fault():
    need_gpu()
    w = W.config(1)
    dt = DT["config1"]["dt"]
    fs = D.FieldSolver(w.xyz, w.tets, w.part, w.n_sub, params=D.make_params(tol=1e-14, max_it=1, chunk=1)).bind()
    with pytest.raises(D.DDError) as e:
        fs.step(None)                                   # not factored yet
    assert e.value.code == D.DD_ERR_STATE
    fs.factor(dt)
    dofs = fs.dof_of_pairs(w.source_pairs)
    src = torch.zeros(fs.n_dof, dtype=torch.float64, device="cuda")
    src[dofs] = 1e-3
    st = fs.step(src, raise_on_error=False)
    assert st["rc"] == D.DD_ERR_NO_CONVERGENCE and st["iters"] == 1
    src[dofs[0]] = float("nan")
    st = fs.step(src, raise_on_error=False)
    assert st["rc"] == D.DD_ERR_NONFINITE
    # the context is still usable
    fs.factor(dt)
    src.zero_()
    fs.set_params(D.make_params(tol=1e-12))
    assert fs.step(src)["status"] == 0
    fs.close()


WARM2 = [(D.DD_FP64, D.DD_SOLVER_SCHUR_CG, D.DD_SCHEME_DP1, 0), (D.DD_MIXED, D.DD_SOLVER_SCHUR_CG, D.DD_SCHEME_DP1, 0),
         (D.DD_FP64, D.DD_SOLVER_COUPLED_GMRES, D.DD_SCHEME_DP1, 0),
         (D.DD_MIXED, D.DD_SOLVER_COUPLED_GMRES, D.DD_SCHEME_DP1, 1),
         (D.DD_MIXED, D.DD_SOLVER_COUPLED_GMRES, D.DD_SCHEME_DP2, 0)]


@pytest.mark.parametrize("prec,solver,scheme,graph", WARM2)
def test_extrapolated_warm_start_matches_oracle(prec, solver, scheme, graph):
    """warm_start 2 (the solve of a step starts from 2 x^{n-1} - x^{n-2}: lambda for
    the CG, [lambda; x_c] -- DP2 [lambda1; lambda2; x_c] -- for the coupled GMRES)
    changes only the start of the interface solve."""
    need_gpu()
    w = W.config(1)
    dt = DT["config1"]["dt"]
    n = 200
    _, _, _, _, ref = oracle_run(w, dt, n)
    fp64 = prec == D.DD_FP64
    prm = D.make_params(precision=prec, tol=1e-13 if fp64 else (1e-6 if solver == D.DD_SOLVER_SCHUR_CG else 1e-5),
                        refine_tol=1e-12, max_refine=8, warm_start=2, solver=solver, scheme=scheme,
                        max_it=3000, use_graph=graph, chunk=2)
    fs, f, _, stats = gpu_run(w, dt, n, prm, probes=False)
    err = rel_err(f, ref["fields"])
    assert err[2:].max() <= (1e-10 if prec == D.DD_FP64 else 1e-8), err.max()
    fs.close()


PACKED_KINDS = ("local", "recover", "iface_rows", "coupled")


@pytest.mark.parametrize("solver", [D.DD_SOLVER_SCHUR_CG, D.DD_SOLVER_COUPLED_GMRES])
def test_packed_symmetric_fp32_tiles(solver):
    """DD_MIXED with the packed lower-triangular FP32 tiles (sym_fp32 = 1) and with
    the dense FP32 copy (0), on a jittered RCB split whose group sizes are not
    multiples of the tile edge: within 1e-8 of the monolithic fields, with about
    the same iteration counts, and the packed path deterministic -- for both
    kernel forms (CTA-synchronous, warp-specialised) over cluster sizes 1..8,
    ring depths 2..4 and L2-kept subdomain counts (clusters of 8 leave some CTAs
    of these small subdomains without tiles), and for the persistent queues."""
    need_gpu()
    nx, ny, nz = 10, 8, 8
    L = (1.2, 1.0, 1.0)
    xyz, tets = W.kuhn_box(nx, ny, nz, *L)
    xyz, rng = W.jitter_nodes(xyz, L[0] / nx, L, 0.2, seed=9)
    part = W.rcb_partition(W.tet_centroids(xyz, tets), 6, rng.uniform(0.6, 1.4, size=6))
    w = W.Workload("ragged", xyz, tets, part, 6, rng.uniform(1, 4, size=len(tets)), 1.0, 30,
                   W.z_line_node_pairs(nx, ny, nz, 5, 4))
    space = fem.EdgeSpace(xyz, tets, w.eps)
    T, S = space.assemble()
    dt = 2.0 * newmark.cfl_dt(T, S)
    n = 30
    _, _, _, _, ref = oracle_run(w, dt, n)

    def pin(cl, st, keep, ws):
        def f(fs):
            for kind in PACKED_KINDS:
                D.dd_set_sym_config(fs.h, kind, cl, st, keep, ws)
            cfg = D.dd_get_sym_config(fs.h)
            assert all(cfg[k] == (cl, st, keep, ws) for k in PACKED_KINDS), cfg
        return f

    cases = [("dense", 0, None), ("packed", 1, None), ("packed", 1, None),
             ("ws 2x3 keep 2", 1, pin(2, 3, 2, 1)), ("ws 1x2", 1, pin(1, 2, 0, 1)),
             ("ws 8x4 keep 6", 1, pin(8, 4, 6, 1)), ("ws 8x4 keep 6", 1, pin(8, 4, 6, 1)),
             ("sync 8x4 keep 3", 1, pin(8, 4, 3, 0)), ("queues 1x6 keep 2", 1, pin(1, 6, 2, 5)),
             ("queues 1x6 keep 2", 1, pin(1, 6, 2, 5)), ("queues 2x4", 1, pin(2, 4, 0, 5))]
    runs = {}
    for name, sym, hook in cases:
        prm = D.make_params(precision=D.DD_MIXED, tol=1e-5, refine_tol=1e-12, max_refine=6, solver=solver,
                            sym_fp32=sym)
        fs, f, _, stats = gpu_run(w, dt, n, prm, probes=False, after_factor=hook)
        fs.close()
        assert all(s["status"] == 0 for s in stats), name
        assert rel_err(f, ref["fields"])[2:].max() <= 1e-8, (name, rel_err(f, ref["fields"]).max())
        its = np.array([s["iters"] for s in stats])
        if name in runs:
            assert np.array_equal(runs[name][0], f), name          # deterministic
        else:
            runs[name] = (f, its)
    dense = runs["dense"][1]
    for name, (f, its) in runs.items():
        # the first steps (tiny right-hand sides) are the most rounding-sensitive
        assert np.all(np.abs(its[2:] - dense[2:]) <= 3), (name, its, dense)
        assert abs(its.sum() - dense.sum()) <= 0.05 * dense.sum(), (name, its, dense)


def test_sym_config_rejects_bad_values():
    need_gpu()
    w = W.config(1)
    fs = D.FieldSolver(w.xyz, w.tets, w.part, w.n_sub, w.eps, w.mu,
                       D.make_params(precision=D.DD_MIXED, tol=1e-5)).bind()
    fs.factor(DT["config1"]["dt"])
    for args in [("corner_rows", 1, 2, 0, 0), ("coarse", 1, 2, 0, 0), ("local", 3, 2, 0, 0), ("local", 1, 5, 0, 0), ("local", 1, 1, 0, 0),
                 ("local", 1, 2, w.n_sub + 1, 0), ("local", 1, 2, 0, 4), ("local", 1, 2, 0, -1)]:
        with pytest.raises(RuntimeError):
            D.dd_set_sym_config(fs.h, *args)
    D.dd_set_sym_config(fs.h, "coupled", 2, 4, 1, 1)
    assert D.dd_get_sym_config(fs.h)["coupled"] == (2, 4, 1, 1)
    fs.close()
