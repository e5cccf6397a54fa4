"""Pins of the oracle's PIC coupling (no GPU): charge-conserving Whitney current
deposition, field interpolation, discrete curl, Boris push and Gauss' law
through a full PIC march (Sec. II, II-A)."""
import numpy as np

from oracle import fem, newmark
from oracle import pic
from paper_2204_13254_gb300 import workloads as W


def mesh_of(n=4, L=(1.0, 1.0, 1.0)):
    w = W.box(n, n, n, 1, 1, 1, L=L)
    space = fem.EdgeSpace(w.xyz, w.tets)
    return w, space, pic.Mesh(space)


def test_deposit_conserves_charge_per_segment():
    w, space, mesh = mesh_of(4)
    D0 = space.gradient_matrix()
    interior = ~fem.boundary_node_mask(space.tets, len(space.xyz))
    rng = np.random.default_rng(0)
    for _ in range(10):
        p0 = rng.uniform(0.15, 0.85, 3)
        p1 = rng.uniform(0.15, 0.85, 3)
        t0 = pic.Beam.locate_on_wall(type("B", (), {"mesh": mesh})(), p0)
        dep = np.zeros(space.n)
        t1, pe, alive = pic.deposit_path(mesh, t0, p0, p1, 0.7, dep)
        assert alive and np.allclose(pe, p1)
        rho = np.zeros(len(space.xyz))
        np.add.at(rho, space.tets[t1], 0.7 * mesh.lam(t1, p1))
        np.add.at(rho, space.tets[t0], -0.7 * mesh.lam(t0, p0))
        assert np.abs(D0.T @ dep - rho[interior]).max() < 1e-14
        assert np.all(mesh.lam(t1, p1) >= -1e-12)


def test_constant_field_line_integral_and_interpolation():
    w, space, mesh = mesh_of(6)
    E0 = np.array([0.3, -1.1, 0.7])
    e = np.array([E0 @ (space.xyz[b] - space.xyz[a]) for a, b in space.edges[space.interior_edges]])
    p0, p1 = np.array([0.3, 0.35, 0.31]), np.array([0.66, 0.62, 0.7])
    t0 = pic.Beam.locate_on_wall(type("B", (), {"mesh": mesh})(), p0)
    dep = np.zeros(space.n)
    t1, _, _ = pic.deposit_path(mesh, t0, p0, p1, 1.3, dep)
    assert abs(e @ dep - 1.3 * E0 @ (p1 - p0)) < 1e-13
    assert np.allclose(mesh.E_at(t1, p1, e), E0, atol=1e-13)
    # constant B: face fluxes b_f = B0 . (b-a)x(c-a)/2 for the sorted triple (a,b,c)
    B0 = np.array([-0.4, 0.9, 0.25])
    X = space.xyz
    fa, fb, fc = X[mesh.faces[:, 0]], X[mesh.faces[:, 1]], X[mesh.faces[:, 2]]
    bflux = 0.5 * np.cross(fb - fa, fc - fa) @ B0
    assert np.allclose(mesh.B_at(t1, p1, bflux), B0, atol=1e-13)


def test_discrete_curl_of_gradient_vanishes():
    w, space, mesh = mesh_of(4)
    D0 = space.gradient_matrix().toarray()
    for k in range(0, D0.shape[1], 3):
        assert np.abs(mesh.curl(D0[:, k])).max() < 1e-15


def test_boris_rotation_angle_and_energy():
    qm, dt, B = -1.0, 0.1, np.array([0.0, 0.0, 2.0])
    v = np.array([0.05, 0.0, 0.01])
    v1 = pic.boris(v, np.zeros(3), B, qm, dt)
    ang = np.arctan2(v1[1], v1[0]) - np.arctan2(v[1], v[0])
    assert abs(abs(ang) - 2 * np.arctan(abs(qm) * 2.0 * dt / 2)) < 1e-14
    assert abs(np.linalg.norm(v1) - np.linalg.norm(v)) < 1e-16
    assert v1[2] == v[2]


def test_pic_march_keeps_gauss_law():
    """Small beam through a PEC box with the monolithic Newmark solve: D0^T (T e^n + G^n) = 0."""
    w = W.box(4, 4, 8, 1, 1, 1, L=(1.0, 1.0, 2.0))
    space = fem.EdgeSpace(w.xyz, w.tets)
    T, S = space.assemble()
    dt = 2.0 * newmark.cfl_dt(T, S)
    A, B = newmark.newmark_matrices(T, S, dt)
    import scipy.sparse.linalg as spla
    lu = spla.splu(A)
    mesh = pic.Mesh(space)
    rng = np.random.default_rng(1)
    n_p, n_steps = 40, 60
    xy = 0.5 + np.clip(rng.normal(0, 0.1, size=(n_p, 2)), -0.4, 0.4)
    x_inj = np.column_stack([xy, np.zeros(n_p)])
    v_inj = np.tile([0.0, 0.0, 0.3], (n_p, 1))
    beam = pic.Beam(mesh, x_inj, v_inj, rng.uniform(0, 0.5 * n_steps * dt, n_p), q=-0.05, qm=-1.0)
    out = pic.run(space, lambda en, enm1, d2g: lu.solve(B @ en - A @ enm1 - d2g), beam, dt, n_steps)
    D0 = space.gradient_matrix()
    worst = 0.0
    for e, G in zip(out["fields"], out["G"]):
        r = D0.T @ (T @ e + G)
        worst = max(worst, np.abs(r).max() / max(np.abs(D0.T @ G).max(), 1e-300))
    assert worst < 1e-11          # round-off of 60 sparse solves
    assert (beam.status == pic.ALIVE).sum() > 0 and np.abs(out["fields"][-1]).max() > 0
