"""Discrete adjoint of the Newmark march (oracle; test infrastructure only).

Not in the paper; derived here from the recurrence of Sec. II-B (edge-only
reading).  Forward, for k = 0..N-1 with e^{-1} = e^0 = 0:

    R^k = A e^{k+1} - B e^k + A e^{k-1} + a * d2g^k = 0,
    A = T(eps) + (dt^2/4) S,  B = 2 T(eps) - (dt^2/2) S,  T(eps) = sum_K eps_K T_K,

where a scales the source and d2g^k is the second difference of the unit tested
integrated current.  The objective is J = sum_{k=1..N} sum_p |E(r_p; e^k)|^2 =
sum_k e^k^T P^T P e^k.  With multipliers mu^{k+1} for R^k the stationarity
conditions give, backward for k = N..1 (mu^{N+1} = mu^{N+2} = 0),

    A mu^k = B mu^{k+1} - A mu^{k+2} + 2 P^T P e^k,

and the gradients

    dJ/deps_K = - sum_{k=0..N-1} mu^{k+1}^T T_K (e^{k+1} - 2 e^k + e^{k-1}),
    dJ/da     = - sum_{k=0..N-1} mu^{k+1}^T d2g^k.

dt is held fixed (not differentiated).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse.linalg as spla

from . import newmark


def forward_fields(T, S, dt, src, d2g, n_steps, amp=1.0):
    """All fields e^{-1}, e^0, ..., e^N as an [N+2, n] array (e^{-1} = e^0 = 0)."""
    A, B = newmark.newmark_matrices(T, S, dt)
    lu = spla.splu(A)
    n = A.shape[0]
    E = np.zeros((n_steps + 2, n))
    for k in range(n_steps):
        E[k + 2] = lu.solve(B @ E[k + 1] - A @ E[k] - amp * d2g[k] * src)
    return E


def objective(P, E):
    """J = sum_{k>=1} |P e^k|^2 over the fields e^1..e^N (rows 2.. of E)."""
    V = E[2:] @ P.T
    return float(np.sum(V * V))


def gradients(space, dt, src, d2g, n_steps, P, amp=1.0):
    """(J, dJ/deps [n_tets], dJ/da, E) for the probe objective, by the discrete adjoint."""
    T, S = space.assemble()
    A, B = newmark.newmark_matrices(T, S, dt)
    lu = spla.splu(A)
    E = forward_fields(T, S, dt, src, d2g, n_steps, amp)
    J = objective(P, E)
    n = A.shape[0]
    PtP = (P.T @ P).tocsr()
    mu_k1 = np.zeros(n)      # mu^{k+1}
    mu_k2 = np.zeros(n)      # mu^{k+2}
    g_eps = np.zeros(len(space.tets))
    g_amp = 0.0
    dofs = space.tet_dof
    for k in range(n_steps, 0, -1):
        mu_k = lu.solve(B @ mu_k1 - A @ mu_k2 + 2.0 * (PtP @ E[k + 1]))
        # mu^k multiplies R^{k-1}: fields e^k, e^{k-1}, e^{k-2} are rows k+1, k, k-1
        d2e = E[k + 1] - 2.0 * E[k] + E[k - 1]
        mloc = np.where(dofs >= 0, mu_k[np.maximum(dofs, 0)], 0.0)
        vloc = np.where(dofs >= 0, d2e[np.maximum(dofs, 0)], 0.0)
        g_eps -= np.einsum("kp,kpq,kq->k", mloc, space.That, vloc)
        g_amp -= mu_k @ (d2g[k - 1] * src)
        mu_k2, mu_k1 = mu_k1, mu_k
    return J, g_eps, g_amp, E
