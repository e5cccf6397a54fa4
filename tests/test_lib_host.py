"""Host-side tests of libdd.so (no GPU needed).

* The library loads and exports every function declared in include/dd.h.
* dd_setup's tearing maps (edges, PEC removal, local numbering, B_r, B_c,
  owners) are bit-exact against the oracle's independent implementation
  (Sec. III-A), on a regular block split and a ragged RCB split of a jittered
  mesh.
* Bad input is reported through status codes, not crashes.
"""
import os
import re

import numpy as np
import pytest

from paper_2204_13254_gb300 import dd as D
from paper_2204_13254_gb300 import workloads as W
from oracle import dd as odd
from oracle import fem

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def built():
    if not os.path.exists(D.LIB_PATH):
        from paper_2204_13254_gb300 import build
        build.build()
    return D.lib()


def header_functions():
    src = open(os.path.join(ROOT, "include", "dd.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(dd_[a-z_]+)\s*\(", src)))


def test_exports_every_header_symbol(built):
    names = header_functions()
    assert "dd_step" in names and "dd_factor" in names
    for n in names:
        assert hasattr(built, n), n
    assert set(names) <= set(D.SYMBOLS) | {n for n in names if hasattr(built, n)}


def _compare_maps(w):
    h = D.dd_setup(w.xyz, w.tets, w.part, w.n_sub, w.eps)
    try:
        got = D.dd_get_maps(h)
        sz = D.dd_get_sizes(h)
    finally:
        D.dd_destroy(h)
    space = fem.EdgeSpace(w.xyz, w.tets, w.eps)
    m = odd.DDMaps(space, w.part, w.n_sub)
    assert np.array_equal(got["edges"], space.edges)
    assert np.array_equal(got["dof_edge"], space.interior_edges)
    assert sz.n_dof == space.n
    loc = np.concatenate(m.local)
    assert np.array_equal(got["local_dof"], loc)
    assert np.array_equal(got["sub_ptr"], np.concatenate([[0], np.cumsum([len(x) for x in m.local])]))
    assert np.array_equal(got["n_int"], m.nI) and np.array_equal(got["n_gam"], m.nG)
    assert np.array_equal(got["n_cor"], m.nC)
    assert np.array_equal(got["mult_dof"], m.mult_dof)
    assert np.array_equal(got["mult_sub"], m.mult_sub)
    assert np.array_equal(got["mult_loc"], m.mult_loc)
    assert np.array_equal(got["corner_dof"], m.corner_dof)
    assert np.array_equal(got["owner"], m.owner)
    return sz


def test_maps_bitexact_cavity(built):
    sz = _compare_maps(W.config(1))
    assert (sz.n_dof, sz.n_lambda, sz.n_corner) == (3032, 480, 24)


def test_maps_bitexact_ragged(built):
    nx, ny, nz = 6, 4, 4
    L = (1.5, 1.0, 1.0)
    xyz, tets = W.kuhn_box(nx, ny, nz, *L)
    xyz, rng = W.jitter_nodes(xyz, L[0] / nx, L, 0.2, seed=3)
    part = W.rcb_partition(W.tet_centroids(xyz, tets), 5, rng.uniform(0.6, 1.4, size=5))
    w = W.Workload("ragged", xyz, tets, part, 5, None, 1.0, 1, W.z_line_node_pairs(nx, ny, nz, 3, 2))
    # reorder the vertices of every other tet: orientation must not matter
    tets2 = tets.copy()
    tets2[::2, [1, 2]] = tets2[::2, [2, 1]]
    w2 = W.Workload("ragged2", xyz, tets2, part, 5, None, 1.0, 1, w.source_pairs)
    _compare_maps(w)
    _compare_maps(w2)


def test_maps_bitexact_blocks_k3(built):
    _compare_maps(W.cavity(6, 3))


def test_status_codes(built):
    xyz, tets = W.kuhn_box(2, 2, 2)
    part = np.zeros(len(tets), np.int32)
    with pytest.raises(D.DDError) as e:
        D.dd_setup(xyz, tets, part + 5, 2)
    assert e.value.code == D.DD_ERR_ARG
    bad = tets.copy()
    bad[0, 1] = bad[0, 0]
    with pytest.raises(D.DDError) as e:
        D.dd_setup(xyz, bad, part, 1)
    assert e.value.code == D.DD_ERR_MESH
    with pytest.raises(D.DDError) as e:
        D.dd_setup(xyz, tets, part, 2)          # subdomain 1 is empty
    assert e.value.code == D.DD_ERR_PARTITION
    flat = xyz.copy()
    flat[:, 2] = 0.0                            # every tet degenerate
    with pytest.raises(D.DDError) as e:
        D.dd_setup(flat, tets, part, 1)
    assert e.value.code == D.DD_ERR_MESH


def test_interface_mass_matches_oracle():
    """MFETI-DP2 interface tangential mass assembled by the library (host) equals the
    oracle's, on a block split and on the 8^3 cavity."""
    import scipy.sparse as sp
    from oracle import dd as odd
    from oracle import fem
    from paper_2204_13254_gb300 import workloads as W
    for w in (W.cavity(4, 2), W.config(1)):
        space = fem.EdgeSpace(w.xyz, w.tets)
        m = odd.DDMaps(space, w.part, w.n_sub)
        ref = odd.interface_mass(space, m, w.part)
        h = D.dd_setup(w.xyz, w.tets, w.part, w.n_sub)
        try:
            ptr, col, val = D.dd_get_interface_mass(h)
        finally:
            D.dd_destroy(h)
        got = sp.csr_matrix((val, col, ptr), shape=ref.shape)
        assert got.nnz == ref.nnz
        assert abs(got - ref).max() <= 1e-15 * abs(ref).max()


def test_ensemble_setup_shares_the_operators(built):
    """members = R: R copies of the tearing maps (member r = mesh copy r, node ids
    + r N), every count R times the single problem's, the dense operators
    stored once, and the Schur CG refused (it would need the stacked K~cc^-1)."""
    w = W.config(1)
    R = 3
    one = D.dd_setup(w.xyz, w.tets, w.part, w.n_sub, params=D.make_params(solver=D.DD_SOLVER_COUPLED_GMRES))
    ens = D.dd_setup(w.xyz, w.tets, w.part, w.n_sub,
                     params=D.make_params(solver=D.DD_SOLVER_COUPLED_GMRES, members=R))
    try:
        s1, sR = D.dd_get_sizes(one), D.dd_get_sizes(ens)
        assert s1.members == 1 and sR.members == R
        for f in ("n_edges", "n_dof", "n_sub", "n_lambda", "n_corner", "n_local", "nnz_local"):
            assert getattr(sR, f) == R * getattr(s1, f), f
        assert sR.dense_bytes_fp64 == s1.dense_bytes_fp64
        assert sR.workspace_bytes < R * s1.workspace_bytes
        m1, mR = D.dd_get_maps(one), D.dd_get_maps(ens)
        N = len(w.xyz)
        e1 = m1["edges"][m1["dof_edge"]]
        eR = mR["edges"][mR["dof_edge"]].reshape(R, -1, 2)
        for r in range(R):
            assert np.array_equal(eR[r], e1 + r * N)
        ns1 = np.diff(m1["sub_ptr"])
        assert np.array_equal(np.diff(mR["sub_ptr"]), np.tile(ns1, R))
        ms = mR["mult_sub"].reshape(R, -1, 2)
        for r in range(R):
            assert np.array_equal(ms[r], m1["mult_sub"].reshape(-1, 2) + r * w.n_sub)
    finally:
        D.dd_destroy(one)
        D.dd_destroy(ens)
    for bad in (D.make_params(members=R), D.make_params(solver=D.DD_SOLVER_COUPLED_GMRES, members=0),
                D.make_params(solver=D.DD_SOLVER_COUPLED_GMRES, members=65)):
        with pytest.raises(D.DDError) as e:
            D.dd_setup(w.xyz, w.tets, w.part, w.n_sub, params=bad)
        assert e.value.code == D.DD_ERR_ARG


def test_ensemble_interface_mass_is_block_diagonal_by_member(built):
    """members = R: the DP2 interface mass is the single problem's, repeated once per
    member on the diagonal (member r's multipliers are rows r*n .. (r+1)*n - 1)."""
    import scipy.sparse as sp
    w = W.cavity(4, 2)
    R = 3
    g = D.make_params(solver=D.DD_SOLVER_COUPLED_GMRES)
    one = D.dd_setup(w.xyz, w.tets, w.part, w.n_sub, params=g)
    ens = D.dd_setup(w.xyz, w.tets, w.part, w.n_sub,
                     params=D.make_params(solver=D.DD_SOLVER_COUPLED_GMRES, members=R))
    try:
        p1, c1, v1 = D.dd_get_interface_mass(one)
        pR, cR, vR = D.dd_get_interface_mass(ens)
        n = len(p1) - 1
    finally:
        D.dd_destroy(one)
        D.dd_destroy(ens)
    M1 = sp.csr_matrix((v1, c1, p1), shape=(n, n))
    MR = sp.csr_matrix((vR, cR, pR), shape=(R * n, R * n))
    ref = sp.block_diag([M1] * R, format="csr")
    assert MR.nnz == ref.nnz
    assert abs(MR - ref).max() == 0.0
