"""The other consumers of the field solve -- the PIC cycle and the discrete
adjoint -- under the coupled interface solvers (MFETI-DP1 coupled GMRES in FP64
and mixed precision, MFETI-DP2), against the same oracles as with the Schur CG;
and the jittered RCB workload at full size in the bench's mixed configuration."""
import json
import os

import numpy as np
import pytest
import scipy.sparse.linalg as spla

torch = pytest.importorskip("torch")

from oracle import adjoint as oadj
from oracle import fem, newmark
from oracle import pic as opic
from paper_2204_13254_gb300 import adjoint as A
from paper_2204_13254_gb300 import dd as D
from paper_2204_13254_gb300 import workloads as W

pytestmark = pytest.mark.gpu
GOLD = os.path.join(os.path.dirname(__file__), "golden")
G = D.DD_SOLVER_COUPLED_GMRES
VARIANTS = {
    "dp1_gmres_fp64": (D.make_params(tol=1e-13, solver=G, max_it=3000), 1e-9),
    "dp1_gmres_mixed": (D.make_params(precision=D.DD_MIXED, tol=1e-5, refine_tol=1e-13, max_refine=8, solver=G), 1e-8),
    "dp2_fp64": (D.make_params(tol=1e-13, solver=G, scheme=D.DD_SCHEME_DP2, max_it=3000), 1e-9),
    "dp2_mixed": (D.make_params(precision=D.DD_MIXED, tol=1e-5, refine_tol=1e-13, max_refine=8, solver=G,
                                scheme=D.DD_SCHEME_DP2), 1e-8),
}


def need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


@pytest.mark.parametrize("name", list(VARIANTS))
def test_pic_cycle(name):
    """Same beam and mesh as the Schur-CG PIC parity test; the oracle solves each
    step by one sparse LU of the monolithic matrix."""
    need_gpu()
    prm, bound = VARIANTS[name]
    w = W.box(4, 4, 8, 2, 2, 2, L=(1.0, 1.0, 2.0))
    space = fem.EdgeSpace(w.xyz, w.tets)
    T, S = space.assemble()
    dt = 2.0 * newmark.cfl_dt(T, S)
    n_steps = 60
    x, v, t, q, qm = W.beam(w, 40, 0.5 * n_steps * dt, speed=0.3, sigma=0.1, q=-0.05, qm=-1.0, seed=1, clip=0.4)
    Am, Bm = newmark.newmark_matrices(T, S, dt)
    lu = spla.splu(Am)
    beam = opic.Beam(opic.Mesh(space), x, v, t, q, qm)
    ref = opic.run(space, lambda en, enm1, d2g: lu.solve(Bm @ en - Am @ enm1 - d2g), beam, dt, n_steps)
    fs = D.FieldSolver(w.xyz, w.tets, w.part, w.n_sub, params=prm).set_beam(x, v, t, q, qm).bind()
    fs.factor(dt)
    worst = 0.0
    for k in range(n_steps):
        fs.pic_step()
        e_n, _, _ = fs.get_state()
        e = e_n.cpu().numpy()
        worst = max(worst, np.linalg.norm(e - ref["fields"][k]) / max(np.linalg.norm(ref["fields"][k]), 1e-300))
    px, st, Gc, b = fs.pic_state()
    st = st.cpu().numpy()
    assert np.array_equal(st, beam.status)
    assert worst <= bound, worst
    D0 = space.gradient_matrix()
    r = D0.T @ (T @ e + Gc.cpu().numpy())
    assert np.abs(r).max() <= 10 * bound * np.abs(D0.T @ Gc.cpu().numpy()).max()
    fs.close()


@pytest.mark.parametrize("name", ["dp1_gmres_fp64", "dp2_fp64", "dp1_gmres_mixed"])
def test_adjoint_gradient(name):
    """Gradient of the probe objective through the coupled solvers = the oracle's adjoint."""
    need_gpu()
    prm, bound = VARIANTS[name]
    steps = 24
    w = W.box(4, 4, 4, 2, 2, 2, steps=steps, probes=W.PROBES_ADJOINT)
    eps = np.random.default_rng(3).uniform(1.0, 4.0, size=len(w.tets))
    space = fem.EdgeSpace(w.xyz, w.tets, eps)
    T, S = space.assemble()
    dt = 2.0 * newmark.cfl_dt(T, S)
    prob = dict(xyz=w.xyz, tets=w.tets, part=w.part, n_sub=w.n_sub, probes=w.probes,
                source_pairs=w.source_pairs, d2g=w.d2G(dt, steps), dt=dt)
    src = np.zeros(space.n)
    src[space.dof_of_pairs(w.source_pairs)] = 1.0
    P = space.probe_operator(w.probes)
    J0, g0, ga0, _ = oadj.gradients(space, dt, src, prob["d2g"], steps, P)
    e = torch.tensor(eps, dtype=torch.float64, device="cuda", requires_grad=True)
    a = torch.tensor(1.0, dtype=torch.float64, requires_grad=True)
    J = A.probe_objective(e, a, prob, steps, 7, params=prm)
    J.backward()
    assert abs(float(J.detach()) - J0) <= 10 * bound * J0
    g = e.grad.cpu().numpy()
    assert np.linalg.norm(g - g0) <= 100 * bound * np.linalg.norm(g0)
    assert abs(float(a.grad) - ga0) <= 100 * bound * abs(ga0)


def test_config3_jittered_rcb300_mixed_gmres():
    """Config 3 (2x1x1 box, 64x32x32 jittered cubes, 300 RCB subdomains, 15,082 corners):
    the bench's mixed configuration in graph mode with tuned tiles; step residual <= 1e-9
    and the Gauss law, both with the oracle's assembled matrices."""
    need_gpu()
    w = W.config(3)
    dt = json.load(open(os.path.join(GOLD, "cfl_dt.json")))["config3"]["dt"]
    n = 10
    space = fem.EdgeSpace(w.xyz, w.tets, w.eps, w.mu)
    T, S = space.assemble()
    Am, Bm = newmark.newmark_matrices(T, S, dt)
    D0 = space.gradient_matrix()
    src = np.zeros(space.n)
    src[space.dof_of_pairs(w.source_pairs)] = 1.0
    d2g = w.d2G(dt, n)
    prm = D.make_params(precision=D.DD_MIXED, tol=1e-5, refine_tol=1e-10, max_refine=6, use_graph=1, chunk=2,
                        solver=G)
    fs = D.FieldSolver(w.xyz, w.tets, w.part, w.n_sub, w.eps, w.mu, prm).bind()
    fs.factor(dt)
    D.dd_autotune(fs.h, None)
    dofs = fs.dof_of_pairs(w.source_pairs)
    sv = torch.zeros(fs.n_dof, dtype=torch.float64, device="cuda")
    out = torch.empty_like(sv)
    f = [np.zeros(space.n), np.zeros(space.n)]
    worst = gauss = 0.0
    for k in range(n):
        sv.zero_()
        sv[dofs] = float(d2g[k])
        assert fs.step(sv, out)["status"] == 0
        f.append(out.cpu().numpy().copy())
        r = Am @ f[-1] - Bm @ f[-2] + Am @ f[-3] + d2g[k] * src
        scale = np.linalg.norm(Bm @ f[-2]) + np.linalg.norm(Am @ f[-3]) + np.linalg.norm(d2g[k] * src)
        worst = max(worst, np.linalg.norm(r) / scale)
        Te = T @ f[-1]
        gauss = max(gauss, np.abs(D0.T @ Te).max() / max(np.abs(Te).max(), 1e-300))
    fs.close()
    assert worst <= 1e-9, worst
    assert gauss <= 1e-6, gauss
