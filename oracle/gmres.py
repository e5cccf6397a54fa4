"""Restarted GMRES(m) with a right diagonal preconditioner (oracle; test infrastructure only).

Sec. IV (discussion of Fig. fetiIter): the coupled MFETI-DP1 equations are solved
with GMRES restarted after 20 iterations, tolerance 1e-6 and a diagonal
preconditioner.  Readings used here (the paper names neither):

* Right preconditioning, M D^-1 u = b, x = D^-1 u, so that the quantity that is
  driven below tol * ||b|| is the true residual ||b - M x|| (in exact
  arithmetic); the Givens-updated least-squares residual |g_{j+1}| is the
  convergence test, checked after every Arnoldi step.
* Arnoldi with modified Gram-Schmidt; H is reduced to triangular form by Givens
  rotations as it is built (the textbook algorithm, Saad, "Iterative Methods
  for Sparse Linear Systems", Alg. 6.9 with right preconditioning, Alg. 9.5).
* A cycle ends after m steps, on convergence, on a zero subdiagonal (the
  Krylov space is invariant: the least-squares solution is exact) or when the
  iteration budget is spent; the iterate is then updated and, unless done,
  the method restarts from the new true residual.
"""
from __future__ import annotations

import numpy as np


def givens(a, b):
    """(c, s) with [c s; -s c] [a; b] = [hypot(a, b); 0]."""
    r = np.hypot(a, b)
    if r == 0.0:
        return 1.0, 0.0
    return a / r, b / r


def gmres(apply, b, x0, dinv, tol, restart=20, max_it=1000):
    """Solve apply(x) = b.  Returns (x, iterations, relative residual estimate, history).

    history[k] is |g_{j+1}| / ||b|| after the k-th Arnoldi step (the residual norm
    of the k-th iterate, not yet formed)."""
    m = int(restart)
    bnorm = float(np.linalg.norm(b))
    x = np.array(x0, dtype=np.float64, copy=True)
    it, hist = 0, []
    while True:
        r = b - apply(x)
        beta = float(np.linalg.norm(r))
        if beta <= tol * bnorm or it >= max_it:
            return x, it, (beta / bnorm if bnorm > 0 else 0.0), hist
        V = np.zeros((m + 1, len(b)))
        V[0] = r / beta
        H = np.zeros((m + 1, m))
        cs, sn = np.zeros(m), np.zeros(m)
        g = np.zeros(m + 1)
        g[0] = beta
        k, converged = 0, False
        for j in range(m):
            w = apply(dinv * V[j])
            for i in range(j + 1):
                H[i, j] = w @ V[i]
                w = w - H[i, j] * V[i]
            hsub = float(np.linalg.norm(w))
            H[j + 1, j] = hsub
            for i in range(j):
                a, c = H[i, j], H[i + 1, j]
                H[i, j], H[i + 1, j] = cs[i] * a + sn[i] * c, -sn[i] * a + cs[i] * c
            cs[j], sn[j] = givens(H[j, j], H[j + 1, j])
            H[j, j] = cs[j] * H[j, j] + sn[j] * H[j + 1, j]
            H[j + 1, j] = 0.0
            g[j + 1] = -sn[j] * g[j]
            g[j] = cs[j] * g[j]
            it += 1
            k = j + 1
            hist.append(abs(g[j + 1]) / bnorm)
            converged = abs(g[j + 1]) <= tol * bnorm
            if converged or it >= max_it or hsub == 0.0:
                break
            V[j + 1] = w / hsub
        y = np.zeros(k)
        for i in range(k - 1, -1, -1):
            y[i] = (g[i] - H[i, i + 1:k] @ y[i + 1:]) / H[i, i]
        x = x + dinv * (V[:k].T @ y)
        if converged or it >= max_it:
            return x, it, hist[-1], hist
