"""Pins of the oracle's Whitney edge-element layer against mathematics (no GPU).

Each test checks the oracle against something other than itself: closed-form
mesh counts, pointwise quadrature of the Whitney functions, the Whitney
tangential-moment property, Stokes' theorem for the curl, the discrete de Rham
property S D0 = 0, the dimension of the gradient null space and the analytic
resonances of the PEC unit cube (Sec. II-B, Whitney 1-forms).
"""
import numpy as np
import pytest

from oracle import fem
from paper_2204_13254_gb300 import workloads as W

RNG = np.random.default_rng(1234)


def random_tet():
    while True:
        X = RNG.normal(size=(4, 3))
        D = np.array([X[1] - X[0], X[2] - X[0], X[3] - X[0]])
        v = np.linalg.det(D) / 6
        if abs(v) > 0.05:
            if v < 0:
                X[[1, 2]] = X[[2, 1]]
            return X


# degree-2 exact 4-point rule on the reference tet (barycentric coordinates)
_A, _B = 0.5854101966249685, 0.1381966011250105
QUAD2 = np.array([[_A, _B, _B, _B], [_B, _A, _B, _B], [_B, _B, _A, _B], [_B, _B, _B, _A]])


@pytest.mark.parametrize("n", [1, 2, 3, 8])
def test_kuhn_mesh_counts(n):
    xyz, tets = W.kuhn_box(n, n, n)
    X = xyz[tets]
    D = np.stack([X[:, 1] - X[:, 0], X[:, 2] - X[:, 0], X[:, 3] - X[:, 0]], axis=1)
    vol = np.linalg.det(D) / 6
    assert np.all(vol > 0)
    assert abs(vol.sum() - 1.0) < 1e-12
    edges, _, _ = fem.mesh_edges(tets)
    total = 3 * n * (n + 1) ** 2 + 3 * n * n * (n + 1) + n ** 3     # axis + face-diagonal + body-diagonal edges
    assert len(edges) == total
    # surface triangulation of the cube is a sphere: F = 12 n^2 triangles, E = 3F/2
    bf = fem.boundary_faces(tets)
    assert len(bf) == 12 * n * n
    pec = fem.pec_edge_mask(tets, edges)
    assert pec.sum() == 18 * n * n
    if n == 8:
        assert len(edges) - pec.sum() == 3032


def test_element_matrices_vs_quadrature():
    for _ in range(20):
        X = random_tet()
        T, S, vol = fem.element_matrices(X)
        g, _ = fem.barycentric_gradients(X)
        Tq = np.zeros((6, 6))
        for lam in QUAD2:
            Wv = fem.whitney_at(X, lam)
            Tq += vol / 4 * Wv @ Wv.T
        assert np.allclose(T, Tq, rtol=0, atol=1e-13 * np.abs(T).max())
        # curl of W_ab by central differences of the pointwise field (W is affine)
        h = 1e-3
        x0 = X.mean(axis=0)

        def Wx(x):
            D = np.array([X[1] - X[0], X[2] - X[0], X[3] - X[0]])
            l123 = np.linalg.solve(D.T, x - X[0])
            return fem.whitney_at(X, np.concatenate([[1 - l123.sum()], l123]))
        J = np.zeros((6, 3, 3))   # J[e, i, j] = d W_i / d x_j
        for j in range(3):
            dx = np.zeros(3); dx[j] = h
            J[:, :, j] = (Wx(x0 + dx) - Wx(x0 - dx)) / (2 * h)
        curl = np.stack([J[:, 2, 1] - J[:, 1, 2], J[:, 0, 2] - J[:, 2, 0], J[:, 1, 0] - J[:, 0, 1]], axis=1)
        Sq = vol * curl @ curl.T
        assert np.allclose(S, Sq, rtol=0, atol=1e-8 * np.abs(S).max())


def test_element_spd_and_rank():
    X = random_tet()
    T, S, _ = fem.element_matrices(X)
    assert np.linalg.eigvalsh(T).min() > 0
    ev = np.linalg.eigvalsh(S)
    assert ev.min() > -1e-12 * ev.max()
    assert np.sum(ev > 1e-10 * ev.max()) == 3          # curls of the 6 Whitney forms span R^3


def test_whitney_tangential_moments():
    """int_{edge f} W_e . dl = delta_ef (the Whitney degrees of freedom)."""
    X = random_tet()
    gl, gw = np.polynomial.legendre.leggauss(4)
    for f, (c, d) in enumerate(fem.LOCAL_EDGES):
        t = X[d] - X[c]
        acc = np.zeros(6)
        for s, w in zip(gl, gw):
            u = 0.5 * (s + 1)
            lam = np.zeros(4); lam[c] = 1 - u; lam[d] = u
            acc += 0.5 * w * fem.whitney_at(X, lam) @ t
        expect = np.zeros(6); expect[f] = 1.0
        assert np.allclose(acc, expect, atol=1e-13)


def test_curl_stokes_on_faces():
    """Flux of curl W_ab through face (a,b,c) equals the circulation of W_ab around it (= 1)."""
    X = random_tet()
    g, _ = fem.barycentric_gradients(X)
    for (a, b) in fem.LOCAL_EDGES:
        curl = 2 * np.cross(g[a], g[b])
        for c in range(4):
            if c in (a, b):
                continue
            area_vec = 0.5 * np.cross(X[b] - X[a], X[c] - X[a])   # oriented a->b->c
            assert abs(curl @ area_vec - 1.0) < 1e-12


def test_discrete_de_rham_and_null_space():
    w = W.config(1)
    space = fem.EdgeSpace(w.xyz, w.tets)
    T, S = space.assemble()
    D0 = space.gradient_matrix()
    assert D0.shape == (3032, 343)
    assert abs(S @ D0).max() <= 1e-13 * abs(S).max()
    ev = np.linalg.eigvalsh(S.toarray())
    assert np.sum(np.abs(ev) < 1e-9 * ev.max()) == 343       # = interior nodes, 7^3
    assert np.linalg.eigvalsh(T.toarray()).min() > 0


def test_cavity_resonances():
    """PEC unit cube: omega = pi sqrt(m^2+n^2+p^2); lowest (1,1,0) triplet, then (1,1,1) pair."""
    import scipy.linalg as sla
    w = W.config(1)
    space = fem.EdgeSpace(w.xyz, w.tets)
    T, S = space.assemble()
    lam = sla.eigh(S.toarray(), T.toarray(), eigvals_only=True)
    nz = np.sort(lam[lam > 1e-8 * lam.max()])
    om = np.sqrt(nz[:5])
    assert np.all(np.abs(om[:3] / (np.pi * np.sqrt(2)) - 1) < 0.03)
    assert np.all(np.abs(om[3:5] / (np.pi * np.sqrt(3)) - 1) < 0.03)


def test_assembly_symmetry_and_probe():
    w = W.cavity(4, 2)
    space = fem.EdgeSpace(w.xyz, w.tets)
    T, S = space.assemble()
    assert abs(T - T.T).max() < 1e-15 and abs(S - S.T).max() < 1e-15
    # a constant field E = (0,0,1) is represented exactly by its edge moments
    e = np.array([(space.xyz[b] - space.xyz[a])[2] for a, b in space.edges[space.interior_edges]])
    P = space.probe_operator(np.array([[0.3, 0.4, 0.55], [0.6, 0.7, 0.4]]))
    assert np.allclose(P @ e, [0, 0, 1, 0, 0, 1], atol=1e-13)
