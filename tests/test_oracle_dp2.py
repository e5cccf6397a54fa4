"""Pins of the oracle's MFETI-DP2 (Sec. III-B, edge-only reading; no GPU).

* The tangential face mass M_T: exact on constant tangential fields (Whitney
  forms reproduce constants, so e^T M_T e = |F_t|^2 area), equal to an
  independent quadrature of the explicit 2-D Whitney functions (edge-midpoint
  rule, exact for their quadratic products), symmetric positive definite.
* Interface faces of a k^3 block split of an n^3 Kuhn cube: 6 n^2 (k - 1).
* M_T on the multiplier edges is block diagonal by subdomain pair.
* The coupled operator's diagonal is [1; 1; diag(K~cc)] (the preconditioner).
* DP2 = the monolithic sparse-direct march for several Robin coefficients, on a
  block split and on a ragged RCB split of a jittered mesh; at convergence the
  two sides' interface traces agree and lambda^(1) + lambda^(2) = 2 alpha M_T x.
"""
import json
import os

import numpy as np
import pytest

from oracle import dd, fem, newmark
from paper_2204_13254_gb300 import workloads as W

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def test_face_mass_constant_fields_and_quadrature():
    rng = np.random.default_rng(0)
    P = rng.standard_normal((20, 3, 3))
    M = fem.face_tangential_mass(P)
    fe = [(0, 1), (1, 2), (0, 2)]
    for k in range(20):
        p = P[k]
        nrm = np.cross(p[1] - p[0], p[2] - p[0])
        area = 0.5 * np.linalg.norm(nrm)
        n = nrm / np.linalg.norm(nrm)
        F = rng.standard_normal(3)
        e = np.array([F @ (p[b] - p[a]) for a, b in fe])
        Ft = F - (F @ n) * n
        assert abs(e @ M[k] @ e - Ft @ Ft * area) <= 1e-12 * (Ft @ Ft * area)
        # explicit 2-D Whitney functions at the edge midpoints: barycentric (1/2,1/2,0) etc.
        A = np.stack([p[1] - p[0], p[2] - p[0]], axis=1)            # 3x2
        G = A.T @ A
        grads = np.linalg.solve(G, A.T).T                            # surface gradients of l1, l2 (rows)
        g = np.stack([-grads[:, 0] - grads[:, 1], grads[:, 0], grads[:, 1]])
        mids = [np.array([0.5, 0.5, 0.0]), np.array([0.0, 0.5, 0.5]), np.array([0.5, 0.0, 0.5])]
        Q = np.zeros((3, 3))
        for lam in mids:
            Wv = np.array([lam[a] * g[b] - lam[b] * g[a] for a, b in fe])
            Q += (area / 3.0) * Wv @ Wv.T
        assert np.allclose(Q, M[k], rtol=1e-12, atol=1e-14 * np.abs(M[k]).max())
        assert np.allclose(M[k], M[k].T) and np.linalg.eigvalsh(M[k]).min() > 0


@pytest.mark.parametrize("n,k", [(4, 2), (6, 3)])
def test_interface_face_count(n, k):
    w = W.cavity(n, k)
    faces, pairs = fem.interface_faces(w.tets, w.part)
    assert len(faces) == 6 * n * n * (k - 1)
    assert np.all(pairs[:, 0] < pairs[:, 1])


def dp2_case(w, dt, alpha=None):
    space = fem.EdgeSpace(w.xyz, w.tets, w.eps, w.mu)
    m = dd.DDMaps(space, w.part, w.n_sub)
    return space, m, dd.DP2Solver(space, m, dt, w.part, alpha)


def test_interface_mass_blocks_and_operator_diagonal():
    w = W.cavity(4, 2)
    dt = 0.1
    space, m, s = dp2_case(w, dt)
    M = s.M.tocoo()
    assert np.abs(s.M - s.M.T).max() <= 1e-15
    same = (m.mult_sub[M.row] == m.mult_sub[M.col]).all(axis=1)
    assert same.all()                                               # block diagonal by pair
    assert np.linalg.eigvalsh(s.M.toarray()).min() > 0
    nu = 2 * m.n_lambda + m.n_corner
    diag = np.array([s.coupled_apply(np.eye(nu)[i])[i] for i in range(nu)])
    ref = np.concatenate([np.ones(2 * m.n_lambda), s.diag_c])
    assert np.allclose(diag, ref, rtol=1e-12, atol=1e-12)


def march_err(w, dt, n_steps, alpha, tol=1e-12):
    space = fem.EdgeSpace(w.xyz, w.tets, w.eps, w.mu)
    T, S = space.assemble()
    src = np.zeros(space.n)
    src[space.dof_of_pairs(w.source_pairs)] = 1.0
    d2g = w.d2G(dt, n_steps)
    mono = newmark.run(T, S, dt, src, d2g, n_steps, keep=True)
    m = dd.DDMaps(space, w.part, w.n_sub)
    r = dd.run_dp2(space, m, w.part, dt, src, d2g, n_steps, tol=tol, keep=True, alpha=alpha)
    err = np.linalg.norm(r["fields"] - mono["fields"], axis=1) / np.maximum(np.linalg.norm(mono["fields"], axis=1), 1e-300)
    return err, r


@pytest.mark.parametrize("scale", [1.0, 0.2, 10.0])
def test_dp2_equals_monolithic_cavity(scale):
    w = W.config(1)
    dt = json.load(open(os.path.join(GOLD, "cfl_dt.json")))["config1"]["dt"]
    err, r = march_err(w, dt, 12, scale * 0.5 * dt)
    assert err[3:].max() < 1e-10, err.max()


def test_dp2_equals_monolithic_ragged_rcb():
    nx, ny, nz = 6, 4, 4
    L = (1.5, 1.0, 1.0)
    xyz, tets = W.kuhn_box(nx, ny, nz, *L)
    xyz, rng = W.jitter_nodes(xyz, L[0] / nx, L, 0.2, seed=3)
    part = W.rcb_partition(W.tet_centroids(xyz, tets), 5, rng.uniform(0.6, 1.4, size=5))
    w = W.Workload(name="ragged", xyz=xyz, tets=tets, part=part, n_sub=5, eps=rng.uniform(1, 4, len(tets)), mu=1.0,
                   steps=10, source_pairs=W.z_line_node_pairs(nx, ny, nz, 3, 2), dims=(nx, ny, nz), L=L)
    space = fem.EdgeSpace(xyz, tets, w.eps)
    T, S = space.assemble()
    dt = 2 * newmark.cfl_dt(T, S)
    err, _ = march_err(w, dt, 10, None)
    assert err[3:].max() < 1e-10, err.max()


def test_transmission_conditions_at_convergence():
    w = W.cavity(4, 2)
    dt = 0.1
    space, m, s = dp2_case(w, dt)
    rng = np.random.default_rng(1)
    b = s.newmark_rhs(rng.standard_normal(space.n), rng.standard_normal(space.n), np.zeros(space.n))
    x, u, it, res = s.solve(b, tol=1e-13, warm=False)
    lam1, lam2, _ = s.split(u)
    t1, t2 = s.traces([xs[:m.nr[k]] for k, xs in enumerate(x)])
    assert np.linalg.norm(t1 - t2) <= 1e-10 * np.linalg.norm(t1)
    assert np.linalg.norm(lam1 + lam2 - 2 * s.alpha * (s.M @ t1)) <= 1e-10 * np.linalg.norm(lam1 + lam2)
    A, B = newmark.newmark_matrices(*space.assemble(), dt)
    import scipy.sparse.linalg as spla
    rhs_global = np.zeros(space.n)
    for k in range(m.n_sub):
        np.add.at(rhs_global, m.local[k], b[k])
    ref = spla.spsolve(A.tocsc(), rhs_global)
    assert np.linalg.norm(s.gather_global(x) - ref) <= 1e-10 * np.linalg.norm(ref)
