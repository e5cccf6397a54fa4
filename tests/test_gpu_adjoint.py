"""GPU discrete adjoint (dd_adjoint_step behind torch.autograd) against the CPU
FP64 oracle adjoint, central finite differences and the closed form dJ/da = 2J/a."""
import json
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import adjoint as oadj
from oracle import fem, newmark
from paper_2204_13254_gb300 import adjoint as A
from paper_2204_13254_gb300 import dd as D
from paper_2204_13254_gb300 import workloads as W

pytestmark = pytest.mark.gpu
GOLD = os.path.join(os.path.dirname(__file__), "golden")


def need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def small_problem(steps=30, seed=3, n=4, k=2):
    w = W.box(n, n, n, k, k, k, steps=steps, probes=W.PROBES_ADJOINT)
    eps = np.random.default_rng(seed).uniform(1.0, 4.0, size=len(w.tets))
    space = fem.EdgeSpace(w.xyz, w.tets, eps)
    T, S = space.assemble()
    dt = 2.0 * newmark.cfl_dt(T, S)
    prob = dict(xyz=w.xyz, tets=w.tets, part=w.part, n_sub=w.n_sub, probes=w.probes,
                source_pairs=w.source_pairs, d2g=w.d2G(dt, steps), dt=dt)
    return w, eps, space, dt, prob


def gpu_grad(eps, amp, prob, steps, checkpoint=100):
    e = torch.tensor(eps, dtype=torch.float64, device="cuda", requires_grad=True)
    a = torch.tensor(amp, dtype=torch.float64, requires_grad=True)
    J = A.probe_objective(e, a, prob, steps, checkpoint)
    J.backward()
    return float(J.detach()), e.grad.cpu().numpy(), float(a.grad)


def test_adjoint_matches_oracle_adjoint():
    need_gpu()
    steps = 30
    w, eps, space, dt, prob = small_problem(steps)
    src = np.zeros(space.n)
    src[space.dof_of_pairs(w.source_pairs)] = 1.0
    P = space.probe_operator(w.probes)
    J0, g0, ga0, _ = oadj.gradients(space, dt, src, prob["d2g"], steps, P)
    J, g, ga = gpu_grad(eps, 1.0, prob, steps, checkpoint=7)
    assert abs(J - J0) <= 1e-11 * J0
    assert np.linalg.norm(g - g0) <= 1e-9 * np.linalg.norm(g0)
    assert abs(ga - ga0) <= 1e-9 * abs(ga0)


def test_checkpoint_size_invariance_and_amplitude_closed_form():
    need_gpu()
    steps = 24
    w, eps, space, dt, prob = small_problem(steps, seed=4)
    J1, g1, a1 = gpu_grad(eps, 0.7, prob, steps, checkpoint=5)
    J2, g2, a2 = gpu_grad(eps, 0.7, prob, steps, checkpoint=100)
    assert abs(J1 - J2) <= 1e-12 * J1
    assert np.linalg.norm(g1 - g2) <= 1e-10 * np.linalg.norm(g2)
    assert abs(a1 - 2.0 * J1 / 0.7) <= 1e-9 * abs(a1)


def test_adjoint_central_differences_20_elements():
    """One handle serves the gradient and all 40 perturbed evaluations (dd_set_eps + refactor)."""
    need_gpu()
    steps = 30
    w, eps, space, dt, prob = small_problem(steps, seed=11)
    pm = A.ProbeMarch(prob)
    try:
        J, g, _ = gpu_grad(eps, 1.0, pm, steps)
        rng = np.random.default_rng(11)
        h = 1e-6
        one = torch.tensor(1.0, dtype=torch.float64)
        with torch.no_grad():
            for K in rng.choice(len(eps), size=20, replace=False):
                ep, em = eps.copy(), eps.copy()
                ep[K] += h
                em[K] -= h
                Jp = float(A.probe_objective(torch.tensor(ep, device="cuda"), one, pm, steps))
                Jm = float(A.probe_objective(torch.tensor(em, device="cuda"), one, pm, steps))
                fd = (Jp - Jm) / (2 * h)
                assert abs(fd - g[K]) <= 1e-5 * np.abs(g).max() + 1e-5 * abs(fd), (K, fd, g[K])
        # back at the unperturbed eps the same handle reproduces J
        J2 = float(A.probe_objective(torch.tensor(eps, device="cuda"), one, pm, steps))
        assert abs(J2 - J) <= 1e-13 * J
    finally:
        pm.close()


def test_set_eps_equals_setup_with_eps_bitwise():
    """dd_set_eps re-assembles the local mass on the device in the host's order:
    a handle set up with eps = 1 and then given eps marches bitwise like a handle
    set up with eps (FP64, eager)."""
    need_gpu()
    steps = 8
    w, eps, space, dt, prob = small_problem(steps, seed=5)
    runs = []
    for via_device in (False, True):
        fs = D.FieldSolver(w.xyz, w.tets, w.part, w.n_sub, eps=None if via_device else eps,
                           params=D.make_params(tol=1e-13)).bind()
        if via_device:
            D.dd_set_eps(fs.h, torch.tensor(eps, device="cuda"))
        fs.factor(dt)
        pat = torch.zeros(fs.n_dof, dtype=torch.float64, device="cuda")
        pat[torch.as_tensor(fs.dof_of_pairs(w.source_pairs), device="cuda")] = 1.0
        out = torch.empty_like(pat)
        for k in range(steps):
            D.dd_step_scaled(fs.h, pat, prob["d2g"][k], out)
        runs.append(out.cpu().numpy())
        fs.close()
    assert np.array_equal(runs[0], runs[1])
    assert np.linalg.norm(runs[0]) > 0


def test_adjoint_full_size_mesh_fd():
    """Config-5 mesh (32^3 cubes, 256 subdomains, eps ~ U[1,4] seed 11, 4 probes), 300 steps
    with checkpoints every 100 (three recomputed segments): directional finite difference
    along a random eps perturbation and dJ/da = 2J/a, one handle for all evaluations."""
    need_gpu()
    w = W.config(5)
    dt = json.load(open(os.path.join(GOLD, "cfl_dt.json")))["config5"]["dt"]
    steps = 300
    prob = dict(xyz=w.xyz, tets=w.tets, part=w.part, n_sub=w.n_sub, probes=w.probes,
                source_pairs=w.source_pairs, d2g=w.d2G(dt, steps), dt=dt)
    pm = A.ProbeMarch(prob, params=D.make_params(tol=1e-12))
    try:
        J, g, ga = gpu_grad(w.eps, 1.0, pm, steps, checkpoint=100)
        assert J > 0
        assert abs(ga - 2.0 * J) <= 1e-8 * abs(ga)
        v = np.random.default_rng(2).standard_normal(len(w.eps))
        h = 1e-6
        one = torch.tensor(1.0, dtype=torch.float64)
        with torch.no_grad():
            Jp = float(A.probe_objective(torch.tensor(w.eps + h * v, device="cuda"), one, pm, steps))
            Jm = float(A.probe_objective(torch.tensor(w.eps - h * v, device="cuda"), one, pm, steps))
    finally:
        pm.close()
    fd = (Jp - Jm) / (2 * h)
    assert abs(fd - g @ v) <= 1e-4 * abs(fd), (fd, g @ v)
