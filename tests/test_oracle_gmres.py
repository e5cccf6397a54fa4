"""Pins of the oracle's restarted GMRES and of the coupled MFETI-DP1 system (no GPU).

GMRES is pinned by its definition, checked by brute force: the k-th iterate of
a cycle minimises ||b - M x|| over x0 + D^-1 K_k(M D^-1, r0), computed here
from an orthonormalised Krylov matrix and a least-squares solve, cycle by
cycle for the restarted method; its residual estimate equals the true
residual of that iterate.

The coupled operator of Eqs. F1lr + F1uc is pinned by what the algebra fixes:
its off-diagonal blocks are F_rc and -F_rc^T, its diagonal blocks symmetric,
eliminating x_c from it gives the Schur operator of Eq. f1schur, and the
coupled solve reproduces the monolithic sparse-direct Newmark fields.
"""
import json
import os

import numpy as np
import pytest

from oracle import dd, fem, newmark
from oracle.gmres import gmres
from paper_2204_13254_gb300 import workloads as W

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def positive_real_system(n=40, seed=0):
    rng = np.random.default_rng(seed)
    K = rng.standard_normal((n, n))
    M = 3.0 * np.eye(n) + 0.4 * (K - K.T) + 0.1 * rng.standard_normal((n, n))
    b = rng.standard_normal(n)
    x0 = rng.standard_normal(n)
    dinv = rng.uniform(0.5, 2.0, n)
    return M, b, x0, dinv


def brute_force_cycle(M, b, x, dinv, k):
    """argmin ||b - M y|| over y in x + D^-1 K_k(M D^-1, b - M x)."""
    Ap = M * dinv[None, :]
    r0 = b - M @ x
    cols = [r0]
    for _ in range(k - 1):
        cols.append(Ap @ cols[-1])
    Q, _ = np.linalg.qr(np.stack(cols, axis=1))
    c, *_ = np.linalg.lstsq(Ap @ Q, r0, rcond=None)
    return x + dinv * (Q @ c)


def test_gmres_iterates_minimise_the_residual():
    M, b, x0, dinv = positive_real_system()
    for k in range(1, 9):
        x, it, res, hist = gmres(lambda v: M @ v, b, x0, dinv, tol=0.0, restart=20, max_it=k)
        assert it == k
        ref = brute_force_cycle(M, b, x0, dinv, k)
        assert np.linalg.norm(x - ref) <= 1e-10 * np.linalg.norm(ref)


def test_restarted_gmres_cycles():
    M, b, x0, dinv = positive_real_system(seed=1)
    x, it, res, hist = gmres(lambda v: M @ v, b, x0, dinv, tol=0.0, restart=4, max_it=10)
    assert it == 10
    ref = x0
    for k in (4, 4, 2):
        ref = brute_force_cycle(M, b, ref, dinv, k)
    assert np.linalg.norm(x - ref) <= 1e-10 * np.linalg.norm(ref)


def test_residual_estimate_is_the_true_residual():
    M, b, x0, dinv = positive_real_system(seed=2)
    _, _, _, hist = gmres(lambda v: M @ v, b, x0, dinv, tol=0.0, restart=6, max_it=15)
    for k in range(1, 16):
        xk, _, _, _ = gmres(lambda v: M @ v, b, x0, dinv, tol=0.0, restart=6, max_it=k)
        true = np.linalg.norm(b - M @ xk) / np.linalg.norm(b)
        assert abs(hist[k - 1] - true) <= 1e-9 * true + 1e-15
    assert all(hist[i + 1] <= hist[i] * (1 + 1e-12) for i in range(len(hist) - 1) if (i + 1) % 6)   # monotone in a cycle


def test_gmres_converges_to_the_solution():
    M, b, x0, dinv = positive_real_system(seed=3)
    x, it, res, _ = gmres(lambda v: M @ v, b, x0, dinv, tol=1e-12, restart=5, max_it=500)
    assert res <= 1e-12 and it < 500
    assert np.linalg.norm(b - M @ x) <= 2e-12 * np.linalg.norm(b)


def test_zero_rhs_and_exact_start():
    M, b, x0, dinv = positive_real_system(seed=4)
    x, it, res, _ = gmres(lambda v: M @ v, np.zeros(len(b)), np.zeros(len(b)), dinv, tol=1e-6)
    assert it == 0 and np.all(x == 0)
    xs = np.linalg.solve(M, b)
    x, it, res, _ = gmres(lambda v: M @ v, b, xs, dinv, tol=1e-6)
    assert it == 0


def test_lucky_breakdown_is_exact():
    """A 3-dimensional Krylov space (M with 3 distinct eigenvalues, D = I): exact after 3 steps."""
    rng = np.random.default_rng(5)
    Q, _ = np.linalg.qr(rng.standard_normal((12, 12)))
    M = Q @ np.diag(np.repeat([1.0, 2.0, 5.0], 4)) @ Q.T
    b = rng.standard_normal(12)
    x, it, res, _ = gmres(lambda v: M @ v, b, np.zeros(12), np.ones(12), tol=1e-13, restart=20, max_it=50)
    assert it == 3
    assert np.linalg.norm(M @ x - b) <= 1e-12 * np.linalg.norm(b)


def coupled_case():
    w = W.cavity(4, 2)
    space = fem.EdgeSpace(w.xyz, w.tets)
    T, S = space.assemble()
    dt = 2 * newmark.cfl_dt(T, S)
    m = dd.DDMaps(space, w.part, w.n_sub)
    return w, space, T, S, dt, m, dd.DDSolver(space, m, dt)


def test_coupled_operator_structure_and_schur_elimination():
    w, space, T, S, dt, m, solver = coupled_case()
    nl, nc = m.n_lambda, m.n_corner
    assert nl > 0 and nc > 0
    E = np.eye(nl + nc)
    C = np.stack([solver.coupled_apply(E[i]) for i in range(nl + nc)], axis=1)
    Crr, Crc, Ccr, Ccc = C[:nl, :nl], C[:nl, nl:], C[nl:, :nl], C[nl:, nl:]
    scale = np.abs(C).max()
    assert np.abs(Crc + Ccr.T).max() <= 1e-13 * scale            # [F_rc ; -F_rc^T]
    assert np.abs(Crr - Crr.T).max() <= 1e-13 * scale
    assert np.abs(Ccc - Ccc.T).max() <= 1e-13 * scale
    assert np.linalg.eigvalsh(0.5 * (C + C.T)).min() > 0           # positive real: GMRES(m) converges
    K = np.stack([solver.schur_apply(np.eye(nl)[i]) for i in range(nl)], axis=1)
    Kc = Crr - Crc @ np.linalg.solve(Ccc, Ccr)                     # eliminate x_c
    assert np.abs(Kc - K).max() <= 1e-11 * np.abs(K).max()
    # the preconditioner is the diagonal of the coupled matrix
    assert np.allclose(np.concatenate([solver.diag, solver.diag_c]), np.diag(C), rtol=1e-12, atol=0)


def test_coupled_solve_matches_schur_solve_and_monolithic():
    w, space, T, S, dt, m, solver = coupled_case()
    rng = np.random.default_rng(7)
    e_n, e_nm1 = rng.standard_normal(space.n), rng.standard_normal(space.n)
    src = np.zeros(space.n)
    src[space.dof_of_pairs(w.source_pairs)] = 0.3
    A, B = newmark.newmark_matrices(T, S, dt)
    import scipy.sparse.linalg as spla
    x_mono = spla.spsolve(A.tocsc(), B @ e_n - A @ e_nm1 - src)
    b = solver.newmark_rhs(e_n, e_nm1, src)
    xg, lam_g, xc_g, it_g, res_g = solver.solve(b, tol=1e-12, warm=False, solver="gmres", restart=20)
    assert res_g <= 1e-12
    xs, lam_s, xc_s, it_s, _ = solver.solve(b, tol=1e-13, warm=False)
    assert np.linalg.norm(lam_g - lam_s) <= 1e-9 * np.linalg.norm(lam_s)
    assert np.linalg.norm(xc_g - xc_s) <= 1e-9 * np.linalg.norm(xc_s)
    e = solver.gather_global(xg)
    assert np.linalg.norm(e - x_mono) <= 1e-10 * np.linalg.norm(x_mono)


def test_coupled_march_equals_monolithic():
    w = W.config(1)
    dt = json.load(open(os.path.join(GOLD, "cfl_dt.json")))["config1"]["dt"]
    space = fem.EdgeSpace(w.xyz, w.tets, w.eps, w.mu)
    T, S = space.assemble()
    src = np.zeros(space.n)
    src[space.dof_of_pairs(w.source_pairs)] = 1.0
    n_steps = 15
    d2g = w.d2G(dt, n_steps)
    mono = newmark.run(T, S, dt, src, d2g, n_steps, keep=True)
    m = dd.DDMaps(space, w.part, w.n_sub)
    r = dd.run(space, m, dt, src, d2g, n_steps, tol=1e-12, keep=True, solver="gmres", restart=20)
    err = np.linalg.norm(r["fields"] - mono["fields"], axis=1) / np.maximum(np.linalg.norm(mono["fields"], axis=1), 1e-300)
    assert err[3:].max() < 1e-9
    assert r["iters"].max() < 200
