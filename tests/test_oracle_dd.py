"""Pins of the oracle's MFETI-DP1 decomposition (no GPU).

Checks against closed forms and against the monolithic solve (Sec. III-A;
the paper's claim in Sec. V-A that the DD fields agree with the monolithic ones
to near machine precision):
* multiplier and corner counts of a k^3 block split of an n^3 Kuhn cube;
* each multiplier joins exactly two subdomains with opposite signs;
* sum_s R_s^T A_s R_s = A (subassembly);
* the Schur operator of Eq. f1schur is symmetric positive definite;
* DD fields equal the monolithic sparse-direct fields step by step, on a
  regular block split and on a ragged RCB split of a jittered mesh.
"""
import json
import os

import numpy as np
import pytest
import scipy.sparse as sp

from oracle import dd, fem, newmark
from paper_2204_13254_gb300 import workloads as W

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def n_lambda_closed(n, k):
    # per interior cut plane (k-1 per axis, 3 axes): the plane's edges (2n(n+1) axis + n^2 diagonal),
    # minus the 4n on the box wall, minus the 2(k-1)n lying on crossings with the other cut planes
    return 3 * (k - 1) * ((2 * n * (n + 1) + n * n) - 4 * n - 2 * (k - 1) * n)


def n_corner_closed(n, k):
    # (k-1)^2 crossing lines per axis direction, n edges each
    return 3 * (k - 1) ** 2 * n


@pytest.mark.parametrize("n,k", [(4, 2), (8, 2), (6, 3), (12, 3), (8, 4)])
def test_map_counts_closed_form(n, k):
    w = W.cavity(n, k)
    space = fem.EdgeSpace(w.xyz, w.tets)
    m = dd.DDMaps(space, w.part, w.n_sub)
    assert m.n_lambda == n_lambda_closed(n, k)
    assert m.n_corner == n_corner_closed(n, k)
    # every interior dof is owned by one subdomain; r/c split consistent
    assert np.all(m.owner >= 0)
    assert sum(len(l) for l in m.local) == int(m.mult.sum())
    if (n, k) == (8, 2):
        assert np.all(m.nI + m.nG == 436) and np.all(m.nC == 12)


def test_signed_boolean_rows():
    w = W.cavity(6, 3)
    space = fem.EdgeSpace(w.xyz, w.tets)
    m = dd.DDMaps(space, w.part, w.n_sub)
    s1, s2 = m.mult_sub[:, 0], m.mult_sub[:, 1]
    assert np.all(s1 < s2)
    for side in range(2):
        s = m.mult_sub[:, side]
        li = m.mult_loc[:, side]
        assert np.all(li >= m.nI[s]) and np.all(li < m.nr[s])       # an interface (r) slot
        got = np.array([m.local[ss][l] for ss, l in zip(s, li)])
        assert np.array_equal(got, m.mult_dof)                     # same global edge on both sides
    # each (subdomain, interface slot) carries exactly one multiplier
    keys = np.concatenate([m.mult_sub[:, 0] * 100000 + m.mult_loc[:, 0], m.mult_sub[:, 1] * 100000 + m.mult_loc[:, 1]])
    assert len(np.unique(keys)) == 2 * m.n_lambda == int(m.nG.sum())


def test_subassembly_sums_to_global():
    w = W.cavity(6, 3)
    space = fem.EdgeSpace(w.xyz, w.tets)
    T, S = space.assemble()
    m = dd.DDMaps(space, w.part, w.n_sub)
    acc_T = sp.csr_matrix(T.shape)
    acc_S = sp.csr_matrix(S.shape)
    for s in range(m.n_sub):
        loc = m.local[s]
        dm = -np.ones(space.n, dtype=np.int64); dm[loc] = np.arange(len(loc))
        Ts, Ss = space.assemble(m.tets_of[s], dm, len(loc))
        R = sp.csr_matrix((np.ones(len(loc)), (np.arange(len(loc)), loc)), shape=(len(loc), space.n))
        acc_T = acc_T + R.T @ Ts @ R
        acc_S = acc_S + R.T @ Ss @ R
    assert abs(acc_T - T).max() <= 1e-15 * abs(T).max()
    assert abs(acc_S - S).max() <= 1e-14 * abs(S).max()


def test_schur_operator_spd():
    w = W.cavity(4, 2)
    space = fem.EdgeSpace(w.xyz, w.tets)
    T, S = space.assemble()
    dt = 2 * newmark.cfl_dt(T, S)
    m = dd.DDMaps(space, w.part, w.n_sub)
    solver = dd.DDSolver(space, m, dt)
    K = np.stack([solver.schur_apply(np.eye(m.n_lambda)[i]) for i in range(m.n_lambda)], axis=1)
    assert np.abs(K - K.T).max() <= 1e-13 * np.abs(K).max()
    assert np.linalg.eigvalsh(K).min() > 0


def _compare_dd_mono(w, dt, n_steps, tol=1e-14):
    space = fem.EdgeSpace(w.xyz, w.tets, w.eps, w.mu)
    T, S = space.assemble()
    src = np.zeros(space.n)
    src[space.dof_of_pairs(w.source_pairs)] = 1.0
    d2g = w.d2G(dt, n_steps)
    mono = newmark.run(T, S, dt, src, d2g, n_steps, keep=True)
    m = dd.DDMaps(space, w.part, w.n_sub)
    ddr = dd.run(space, m, dt, src, d2g, n_steps, tol=tol, keep=True)
    err = np.linalg.norm(ddr["fields"] - mono["fields"], axis=1) / np.maximum(np.linalg.norm(mono["fields"], axis=1), 1e-300)
    return err, ddr


def test_dd_equals_monolithic_cavity():
    w = W.config(1)
    dt = json.load(open(os.path.join(GOLD, "cfl_dt.json")))["config1"]["dt"]
    err, ddr = _compare_dd_mono(w, dt, 25)
    assert err[3:].max() < 1e-12
    assert ddr["iters"].max() < 100


def test_dd_equals_monolithic_ragged_rcb():
    nx, ny, nz = 6, 4, 4
    L = (1.5, 1.0, 1.0)
    xyz, tets = W.kuhn_box(nx, ny, nz, *L)
    xyz, rng = W.jitter_nodes(xyz, L[0] / nx, L, 0.2, seed=3)
    part = W.rcb_partition(W.tet_centroids(xyz, tets), 5, rng.uniform(0.6, 1.4, size=5))
    w = W.Workload(name="ragged", xyz=xyz, tets=tets, part=part, n_sub=5, eps=None, mu=1.0, steps=12,
                   source_pairs=W.z_line_node_pairs(nx, ny, nz, 3, 2), dims=(nx, ny, nz), L=L)
    space = fem.EdgeSpace(xyz, tets)
    m = dd.DDMaps(space, part, 5)
    assert m.n_corner > 0 and len(set(m.nr.tolist())) > 1       # uneven subdomains with corners
    T, S = space.assemble()
    dt = 2 * newmark.cfl_dt(T, S)
    err, _ = _compare_dd_mono(w, dt, 12)
    assert err[3:].max() < 1e-12
