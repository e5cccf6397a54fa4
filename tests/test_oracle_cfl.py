"""Pins of the oracle's explicit stability limit ``newmark.cfl_dt`` (no GPU).

Every workload steps at dt = 2 x the explicit limit of the central-difference
(leapfrog) march with the consistent mass matrix, dt_CFL = 2 / sqrt(lambda_max)
with lambda_max the largest eigenvalue of the pencil (S, T) (the reading of the
time step for Sec. II-B's unconditionally stable Newmark scheme).  The oracle
finds lambda_max with ARPACK and an inner CG; it is checked here against

  * a dense generalised symmetric eigensolve of (S, T) (LAPACK), on the 8^3
    cavity and on a small jittered mesh with a random permittivity per tet, and
  * the property that defines the limit: the leapfrog march
    T (e^{n+1} - 2 e^n + e^{n-1}) = -dt^2 S e^n stays bounded at 0.98 dt_CFL
    and blows up at 1.02 dt_CFL.

A wrong factor (1/sqrt instead of 2/sqrt), the wrong pencil (S alone, a lumped
T, or T^-1 applied on the wrong side) or an ARPACK tolerance miss fails one of
these.  tests/golden/cfl_dt.json, the stored time steps, is checked to be the
oracle's own result for the configurations small enough to recompute here.
"""
import json
import os

import numpy as np
import pytest
import scipy.linalg as sla
import scipy.sparse.linalg as spla

from oracle import fem, newmark
from paper_2204_13254_gb300 import workloads as W

GOLD = os.path.join(os.path.dirname(__file__), "golden", "cfl_dt.json")


def _jittered_eps_mesh():
    """5 x 4 x 3 Kuhn box on [0, 1.25] x [0, 1] x [0, 0.75], interior nodes jittered by
    +-20 % of h (seed 3), eps ~ U[1, 4] per tet (seed 5)."""
    L = (1.25, 1.0, 0.75)
    xyz, tets = W.kuhn_box(5, 4, 3, *L)
    xyz, _ = W.jitter_nodes(xyz, 0.25, L, 0.2, seed=3)
    eps = np.random.default_rng(5).uniform(1.0, 4.0, size=len(tets))
    return fem.EdgeSpace(xyz, tets, eps, 1.0)


def _cavity8():
    w = W.config(1)
    return fem.EdgeSpace(w.xyz, w.tets, w.eps, w.mu)


@pytest.fixture(scope="module", params=["cavity8", "jitter_eps"])
def pencil(request):
    space = _cavity8() if request.param == "cavity8" else _jittered_eps_mesh()
    T, S = space.assemble()
    return request.param, T, S


def test_cfl_dt_matches_dense_generalised_eigensolve(pencil):
    name, T, S = pencil
    lam = sla.eigh(S.toarray(), T.toarray(), eigvals_only=True, driver="gvd")
    lam_max = float(lam[-1])
    dt_dense = 2.0 / np.sqrt(lam_max)
    dt = newmark.cfl_dt(T, S)
    assert abs(dt - dt_dense) <= 1e-8 * dt_dense, (name, dt, dt_dense)


def _leapfrog_growth(T, S, dt, n_steps=2000, seed=1):
    """Largest ||e^n||_T / ||e^0||_T of the leapfrog march from a random start
    (e^{-1} = e^0), stopping early once it exceeds 1e12."""
    lu = spla.splu(T.tocsc())
    rng = np.random.default_rng(seed)
    e0 = rng.standard_normal(T.shape[0])
    e_nm1, e_n = e0.copy(), e0.copy()
    n0 = np.sqrt(e0 @ (T @ e0))
    worst = 1.0
    for _ in range(n_steps):
        e_np1 = 2.0 * e_n - e_nm1 - dt * dt * lu.solve(S @ e_n)
        e_nm1, e_n = e_n, e_np1
        g = np.sqrt(e_n @ (T @ e_n)) / n0
        worst = max(worst, g)
        if worst > 1e12:
            break
    return worst


def test_leapfrog_stable_below_and_unstable_above_cfl(pencil):
    name, T, S = pencil
    dt = newmark.cfl_dt(T, S)
    below = _leapfrog_growth(T, S, 0.98 * dt)
    above = _leapfrog_growth(T, S, 1.02 * dt)
    # Below the limit every mode oscillates with unit amplification; the T-norm
    # of e^n (not the conserved discrete energy) can swing by a bounded factor.
    assert below < 50.0, (name, below)
    # Above it the top mode is amplified by ~1.5 per step.
    assert above > 1e12, (name, above)


def test_golden_dt_is_the_oracle_limit():
    table = json.load(open(GOLD))
    space = _cavity8()
    T, S = space.assemble()
    dt = newmark.cfl_dt(T, S)
    assert abs(table["config1"]["dt_cfl"] - dt) <= 1e-10 * dt
    assert table["config1"]["dt"] == 2.0 * table["config1"]["dt_cfl"]
    for key, row in table.items():
        assert row["dt"] == 2.0 * row["dt_cfl"], key
        assert row["n_dof"] > 0
