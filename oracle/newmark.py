"""Implicit Newmark-beta time march, monolithic (oracle; test infrastructure only).

Paper Sec. II-B ("Temporal Discretization", Eq. maxnmb) discretises the
semi-discrete system with Newmark-beta, gamma = 1/2, beta = 1/4, which is
unconditionally stable.  In the edge-only wave-equation reading used here
(the paper notes in Sec. I that its conservation machinery carries over to the
wave equation, and its Sec. VI wants edge-only unknowns), the semi-discrete
system is

    T e'' + S e = -g''(t),      g_i(t) = <W_i, G(t)>,  G = int_0^t J,

and Newmark gamma=1/2, beta=1/4 with the source taken as the second difference
of the integrated current (Sec. II-A: G is used so that the current evolves
consistently with Gauss' law for any time marching) gives the recurrence

    A e^{n+1} = B e^n - A e^{n-1} - (g^{n+1} - 2 g^n + g^{n-1}),
    A = T + (dt^2/4) S,   B = 2T - (dt^2/2) S,

started from e^{-1} = e^0 = 0.  ``run`` solves it with one sparse direct
factorisation of A, reused every step (the paper's "monolithic" solve).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla


def newmark_matrices(T, S, dt):
    A = (T + (dt * dt / 4.0) * S).tocsc()
    B = (2.0 * T - (dt * dt / 2.0) * S).tocsr()
    return A, B


def run(T, S, dt, src, d2g, n_steps, P=None, keep=False, dense=False):
    """March the recurrence n_steps from rest.

    src   -- [n] spatial source pattern (g(t) = src * G(t)).
    d2g   -- [>= n_steps] second differences G^{n+1} - 2G^n + G^{n-1}, one per step.
    P     -- optional probe operator; probe values after every step are returned.
    keep  -- return every field e^1..e^{n_steps} as a [n_steps, n] array.
    dense -- solve with a dense LU (numpy) instead of the sparse factorisation.
    Returns dict with e_n (last), e_nm1 (second last), probes, fields.
    """
    A, B = newmark_matrices(T, S, dt)
    n = A.shape[0]
    if dense:
        Ad = A.toarray()
        solve = lambda b: np.linalg.solve(Ad, b)
    else:
        lu = spla.splu(A)
        solve = lu.solve
    e_nm1 = np.zeros(n)
    e_n = np.zeros(n)
    probes, fields = [], []
    for k in range(n_steps):
        rhs = B @ e_n - A @ e_nm1 - d2g[k] * src
        e_np1 = solve(rhs)
        e_nm1, e_n = e_n, e_np1
        if P is not None:
            probes.append(P @ e_n)
        if keep:
            fields.append(e_n.copy())
    out = dict(e_n=e_n, e_nm1=e_nm1)
    if P is not None:
        out["probes"] = np.array(probes)
    if keep:
        out["fields"] = np.array(fields)
    return out


def step_residual(T, S, dt, e_np1, e_n, e_nm1, d2g_vec):
    """Residual of the recurrence, A e^{n+1} - B e^n + A e^{n-1} + d2g, and the scale ||B e^n|| + ||A e^{n-1}|| + ||d2g||."""
    A, B = newmark_matrices(T, S, dt)
    r = A @ e_np1 - B @ e_n + A @ e_nm1 + d2g_vec
    scale = np.linalg.norm(B @ e_n) + np.linalg.norm(A @ e_nm1) + np.linalg.norm(d2g_vec)
    return r, scale


def energy(T, S, dt, e_np1, e_n):
    """Discrete energy W^{n+1/2} = (de)^T T (de) / dt^2 + (se)^T S (se) / 4,
    de = e^{n+1} - e^n, se = e^{n+1} + e^n; conserved exactly by the
    source-free recurrence (it is the recurrence's own quadratic invariant)."""
    de = e_np1 - e_n
    se = e_np1 + e_n
    return de @ (T @ de) / dt ** 2 + se @ (S @ se) / 4.0


def gauss_residual(D0, T, e, q=None):
    """r = D0^T T e (+ q): discrete Gauss law on interior nodes."""
    r = D0.T @ (T @ e)
    return r if q is None else r + q


def cfl_dt(T, S, tol=1e-9):
    """Explicit (central-difference, consistent-mass) stability limit 2/sqrt(lambda_max(T^-1 S)).

    lambda_max by ARPACK (Lanczos) on the symmetric-definite pencil (S, T); T^-1
    is applied by conjugate gradients (T is a well-conditioned mass matrix), so
    no sparse factorisation is needed at large sizes.
    """
    Tc = T.tocsr()
    d = Tc.diagonal()
    M = spla.LinearOperator(T.shape, matvec=lambda v: v / d, dtype=np.float64)

    def tinv(v):
        x, info = spla.cg(Tc, v, rtol=1e-13, atol=0.0, maxiter=2000, M=M)
        assert info == 0
        return x
    Minv = spla.LinearOperator(T.shape, matvec=tinv, dtype=np.float64)
    lam = spla.eigsh(S, k=1, M=Tc, Minv=Minv, which="LA", tol=tol, ncv=32, return_eigenvectors=False)
    return 2.0 / np.sqrt(float(lam[0]))
