"""GPU PIC cycle (dd_pic_step) against the CPU oracle PIC, and Gauss' law at
round-off with the DD field solve (Sec. II, II-A; the paper's Fig. dgls claim)."""
import json
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import scipy.sparse.linalg as spla

from oracle import fem, newmark
from oracle import pic as opic
from paper_2204_13254_gb300 import dd as D
from paper_2204_13254_gb300 import workloads as W

pytestmark = pytest.mark.gpu
GOLD = os.path.join(os.path.dirname(__file__), "golden")


def need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def test_pic_matches_oracle_small():
    need_gpu()
    w = W.box(4, 4, 8, 2, 2, 2, L=(1.0, 1.0, 2.0))
    space = fem.EdgeSpace(w.xyz, w.tets)
    T, S = space.assemble()
    dt = 2.0 * newmark.cfl_dt(T, S)
    n_steps = 60
    x, v, t, q, qm = W.beam(w, 40, 0.5 * n_steps * dt, speed=0.3, sigma=0.1, q=-0.05, qm=-1.0, seed=1, clip=0.4)
    # oracle: monolithic solve
    A, B = newmark.newmark_matrices(T, S, dt)
    lu = spla.splu(A)
    beam = opic.Beam(opic.Mesh(space), x, v, t, q, qm)
    ref = opic.run(space, lambda en, enm1, d2g: lu.solve(B @ en - A @ enm1 - d2g), beam, dt, n_steps)
    # GPU: MFETI-DP1 field solve, CUDA-graph steps
    for prm in (D.make_params(tol=1e-13), D.make_params(tol=1e-13, use_graph=1, chunk=2)):
        fs = D.FieldSolver(w.xyz, w.tets, w.part, w.n_sub, params=prm).set_beam(x, v, t, q, qm).bind()
        fs.factor(dt)
        worst_e = 0.0
        for k in range(n_steps):
            fs.pic_step()
            e_n, _, _ = fs.get_state()
            e = e_n.cpu().numpy()
            worst_e = max(worst_e, np.linalg.norm(e - ref["fields"][k]) / max(np.linalg.norm(ref["fields"][k]), 1e-300))
        px, st, G, b = fs.pic_state()
        st = st.cpu().numpy()
        assert np.array_equal(st, beam.status)
        alive = st > 0
        assert np.abs(px.cpu().numpy()[alive] - beam.x[alive]).max() < 1e-10
        assert np.linalg.norm(G.cpu().numpy() - ref["G"][-1]) <= 1e-10 * np.linalg.norm(ref["G"][-1])
        assert np.linalg.norm(b.cpu().numpy() - ref["b"]) <= 1e-9 * np.linalg.norm(ref["b"])
        assert worst_e <= 1e-9
        # Gauss' law on the GPU fields: D0^T (T e + G) = 0 at interior nodes
        D0 = space.gradient_matrix()
        r = D0.T @ (T @ e + G.cpu().numpy())
        assert np.abs(r).max() <= 1e-10 * np.abs(D0.T @ G.cpu().numpy()).max()
        fs.close()


def test_config2_beam_full_size_gauss_law():
    """Config 2: 1x1x2 PEC box, 16x16x32 cubes, 128 subdomains, 1e5 macro-particles at 0.1c
    (sigma 0.05, injection times U[0, 2000 dt), seed 0); 300 PIC steps in the bench's graph mode."""
    need_gpu()
    w = W.config(2)
    dt = json.load(open(os.path.join(GOLD, "cfl_dt.json")))["config2"]["dt"]
    x, v, t, q, qm = W.beam(w, 100000, 2000 * dt, seed=0)
    fs = D.FieldSolver(w.xyz, w.tets, w.part, w.n_sub, params=D.make_params(tol=1e-12, use_graph=1, chunk=2))
    fs.set_beam(x, v, t, q, qm).bind()
    fs.factor(dt)
    for k in range(300):
        st = fs.pic_step(stats=(k % 50 == 49))
    e_n, _, _ = fs.get_state()
    px, status, G, b = fs.pic_state()
    status = status.cpu().numpy()
    assert (status == 1).sum() > 1000           # particles in flight
    space = fem.EdgeSpace(w.xyz, w.tets)
    T, _ = space.assemble()
    D0 = space.gradient_matrix()
    Gn = G.cpu().numpy()
    r = D0.T @ (T @ e_n.cpu().numpy() + Gn)
    assert np.abs(r).max() <= 1e-9 * np.abs(D0.T @ Gn).max()
    fs.close()
