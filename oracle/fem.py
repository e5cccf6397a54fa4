"""Whitney edge elements on tetrahedra (oracle; test infrastructure only).

Paper Sec. II-B: the electric field is expanded in Whitney 1-forms W^(1),
E = sum_i e_i W_i, which are tangentially continuous.  For the edge (a,b) of a
tet with barycentric coordinates lambda,

    W_ab = lambda_a grad(lambda_b) - lambda_b grad(lambda_a),
    curl W_ab = 2 grad(lambda_a) x grad(lambda_b).

With the edge-only wave-equation reading, the matrices are the mass
T_ij = <W_i, eps W_j> and the curl-curl S_ij = <curl W_i, mu^-1 curl W_j>,
integrated exactly with  int_K lambda_a lambda_b = |K| (1 + delta_ab) / 20.

Global edges are the distinct node pairs (low id, high id), sorted, and oriented
from the lower to the higher node id.  PEC walls (tangential E = 0) remove every
edge that lies in a boundary triangle.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

# local edge k of a tet joins local vertices LOCAL_EDGES[k]
LOCAL_EDGES = [(0, 1), (0, 2), (0, 3), (1, 2), (1, 3), (2, 3)]
LOCAL_FACES = [(1, 2, 3), (0, 2, 3), (0, 1, 3), (0, 1, 2)]


def mesh_edges(tets):
    """Global edge list and tet->edge incidence.

    Returns (edges [E,2] int64 sorted lexicographically with edges[:,0] < edges[:,1],
             tet_edge [T,6] global edge id of each local edge,
             tet_sign [T,6] +1 if the local edge (a,b), a<b in local order, runs from
             the lower to the higher global node id, else -1).
    """
    tets = np.asarray(tets, dtype=np.int64)
    a = tets[:, [p for p, _ in LOCAL_EDGES]]
    b = tets[:, [q for _, q in LOCAL_EDGES]]
    lo = np.minimum(a, b)
    hi = np.maximum(a, b)
    n = int(tets.max()) + 1
    key = lo * n + hi
    ukey, inv = np.unique(key.ravel(), return_inverse=True)
    edges = np.stack([ukey // n, ukey % n], axis=1)
    tet_edge = inv.reshape(-1, 6)
    tet_sign = np.where(a < b, 1, -1)
    return edges, tet_edge, tet_sign


def boundary_faces(tets):
    """Triangles that belong to exactly one tet (sorted node triples)."""
    tets = np.asarray(tets, dtype=np.int64)
    f = np.concatenate([np.sort(tets[:, list(fc)], axis=1) for fc in LOCAL_FACES], axis=0)
    uf, cnt = np.unique(f, axis=0, return_counts=True)
    return uf[cnt == 1]


def pec_edge_mask(tets, edges):
    """True for edges lying in a boundary triangle (removed by the PEC condition)."""
    bf = boundary_faces(tets)
    n = int(np.max(tets)) + 1
    pairs = np.concatenate([bf[:, [0, 1]], bf[:, [0, 2]], bf[:, [1, 2]]], axis=0)
    bkeys = np.unique(pairs[:, 0] * n + pairs[:, 1])
    ekeys = edges[:, 0] * n + edges[:, 1]
    return np.isin(ekeys, bkeys)


def boundary_node_mask(tets, n_nodes):
    bf = boundary_faces(tets)
    m = np.zeros(n_nodes, dtype=bool)
    m[bf.ravel()] = True
    return m


def barycentric_gradients(X):
    """Gradients [...,4,3] of the barycentric functions and volumes of tets X [...,4,3]."""
    X = np.asarray(X, dtype=np.float64)
    D = np.stack([X[..., 1, :] - X[..., 0, :], X[..., 2, :] - X[..., 0, :], X[..., 3, :] - X[..., 0, :]], axis=-2)
    vol = np.linalg.det(D) / 6.0
    Dinv = np.linalg.inv(D)           # lambda_{1..3}(x) = (x - x0) @ Dinv
    g = np.zeros(X.shape[:-2] + (4, 3))
    g[..., 1:, :] = np.swapaxes(Dinv, -1, -2)
    g[..., 0, :] = -g[..., 1:, :].sum(axis=-2)
    return g, vol


def element_matrices(X):
    """Unit-coefficient Whitney mass and curl-curl 6x6 matrices of tets X [...,4,3].

    Local orientation: local edge (a,b) runs from local vertex a to b (a < b).
    Returns (T_hat, S_hat, vol) with T = eps*T_hat and S = S_hat/mu, where
    T_hat[p,q] = int W_p . W_q and S_hat[p,q] = int curl W_p . curl W_q.
    """
    g, vol = barycentric_gradients(X)
    # M[a,c] = int lambda_a lambda_c = vol (1 + delta_ac) / 20
    M = (np.ones((4, 4)) + np.eye(4)) / 20.0
    M = vol[..., None, None] * M
    GG = g @ np.swapaxes(g, -1, -2)
    ea = np.array([a for a, _ in LOCAL_EDGES])
    eb = np.array([b for _, b in LOCAL_EDGES])
    A, C = np.meshgrid(ea, ea, indexing="ij")
    B, D = np.meshgrid(eb, eb, indexing="ij")
    # W_ab . W_cd = l_a l_c gb.gd - l_a l_d gb.gc - l_b l_c ga.gd + l_b l_d ga.gc
    T = (M[..., A, C] * GG[..., B, D] - M[..., A, D] * GG[..., B, C]
         - M[..., B, C] * GG[..., A, D] + M[..., B, D] * GG[..., A, C])
    curl = 2.0 * np.cross(g[..., ea, :], g[..., eb, :])
    S = vol[..., None, None] * (curl @ np.swapaxes(curl, -1, -2))
    return T, S, vol


def face_tangential_mass(P):
    """Tangential Whitney mass 3x3 of triangles P [...,3,3] (node rows sorted by global id).

    Edges in the order (0,1), (1,2), (0,2), each oriented from its lower to its
    higher node.  The tangential trace of the 3-D Whitney function of an edge of
    the face is the 2-D Whitney function l_a g_b - l_b g_a of the triangle (g:
    surface gradients of its barycentrics), so
    M[p,q] = int_face (n x W_p).(n x W_q) = int_face W_p,t . W_q,t, integrated
    exactly with int l_a l_c = area (1 + delta_ac) / 12.
    """
    P = np.asarray(P, dtype=np.float64)
    E1 = P[..., 1, :] - P[..., 0, :]
    E2 = P[..., 2, :] - P[..., 0, :]
    G = np.stack([np.stack([(E1 * E1).sum(-1), (E1 * E2).sum(-1)], -1),
                  np.stack([(E1 * E2).sum(-1), (E2 * E2).sum(-1)], -1)], -2)
    Gi = np.linalg.inv(G)
    g = np.zeros(P.shape[:-2] + (3, 3))
    g[..., 1, :] = Gi[..., 0, 0, None] * E1 + Gi[..., 0, 1, None] * E2
    g[..., 2, :] = Gi[..., 1, 0, None] * E1 + Gi[..., 1, 1, None] * E2
    g[..., 0, :] = -g[..., 1, :] - g[..., 2, :]
    area = 0.5 * np.linalg.norm(np.cross(E1, E2), axis=-1)
    Ml = area[..., None, None] * (np.ones((3, 3)) + np.eye(3)) / 12.0
    GG = g @ np.swapaxes(g, -1, -2)
    fe = [(0, 1), (1, 2), (0, 2)]
    M = np.zeros(P.shape[:-2] + (3, 3))
    for p_, (a, b) in enumerate(fe):
        for q_, (c, d) in enumerate(fe):
            M[..., p_, q_] = (Ml[..., a, c] * GG[..., b, d] - Ml[..., a, d] * GG[..., b, c]
                              - Ml[..., b, c] * GG[..., a, d] + Ml[..., b, d] * GG[..., a, c])
    return M


def interface_faces(tets, part):
    """Triangles shared by two tets of different subdomains: (sorted node triples [F,3],
    subdomain pairs [F,2] with the lower id first)."""
    tets = np.asarray(tets, dtype=np.int64)
    part = np.asarray(part, dtype=np.int64)
    T = len(tets)
    f = np.concatenate([np.sort(tets[:, list(fc)], axis=1) for fc in LOCAL_FACES], axis=0)
    owner = np.tile(np.arange(T), 4)
    uf, inv, cnt = np.unique(f, axis=0, return_inverse=True, return_counts=True)
    first = -np.ones(len(uf), dtype=np.int64)
    second = -np.ones(len(uf), dtype=np.int64)
    for r, u in enumerate(inv):
        if first[u] < 0:
            first[u] = owner[r]
        else:
            second[u] = owner[r]
    shared = (cnt == 2)
    sa, sb = part[first[shared]], part[second[shared]]
    keep = sa != sb
    faces = uf[shared][keep]
    pairs = np.stack([np.minimum(sa, sb)[keep], np.maximum(sa, sb)[keep]], axis=1)
    return faces, pairs


def whitney_at(X, lam):
    """Values [6,3] of the six local Whitney functions at barycentric point lam [4]."""
    g, _ = barycentric_gradients(X)
    return np.array([lam[a] * g[b] - lam[b] * g[a] for a, b in LOCAL_EDGES])


class EdgeSpace:
    """Interior (non-PEC) Whitney edge space of a tetrahedral mesh."""

    def __init__(self, xyz, tets, eps=None, mu=1.0):
        self.xyz = np.asarray(xyz, dtype=np.float64)
        self.tets = np.asarray(tets, dtype=np.int64)
        nt = len(self.tets)
        self.eps = np.ones(nt) if eps is None else np.asarray(eps, dtype=np.float64)
        self.mu = float(mu)
        self.edges, self.tet_edge, self.tet_sign = mesh_edges(self.tets)
        pec = pec_edge_mask(self.tets, self.edges)
        self.interior_edges = np.flatnonzero(~pec)          # global edge ids kept
        self.edge_to_dof = -np.ones(len(self.edges), dtype=np.int64)
        self.edge_to_dof[self.interior_edges] = np.arange(len(self.interior_edges))
        self.n = len(self.interior_edges)
        self.tet_dof = self.edge_to_dof[self.tet_edge]      # -1 where PEC
        Th, Sh, vol = element_matrices(self.xyz[self.tets])
        ss = self.tet_sign[:, :, None] * self.tet_sign[:, None, :]
        self.That = Th * ss
        self.Shat = Sh * ss
        self.vol = vol

    def element_T(self, k):
        return self.eps[k] * self.That[k]

    def element_S(self, k):
        return self.Shat[k] / self.mu

    def assemble(self, tet_ids=None, dof_map=None, n_dof=None):
        """Assemble (T, S) as CSR over the selected tets.

        ``dof_map`` maps interior-dof id -> row id (default identity); entries
        mapping to -1 are dropped.
        """
        if tet_ids is None:
            tet_ids = np.arange(len(self.tets))
        if dof_map is None:
            dof_map = np.arange(self.n)
            n_dof = self.n
        tet_ids = np.asarray(tet_ids, dtype=np.int64)
        d = self.tet_dof[tet_ids]
        loc = np.where(d >= 0, dof_map[np.where(d >= 0, d, 0)], -1)       # [K,6]
        Tk = self.eps[tet_ids, None, None] * self.That[tet_ids]
        Sk = self.Shat[tet_ids] / self.mu
        r = np.broadcast_to(loc[:, :, None], Tk.shape)
        c = np.broadcast_to(loc[:, None, :], Tk.shape)
        ok = (r >= 0) & (c >= 0)
        T = sp.csr_matrix((Tk[ok], (r[ok], c[ok])), shape=(n_dof, n_dof))
        S = sp.csr_matrix((Sk[ok], (r[ok], c[ok])), shape=(n_dof, n_dof))
        T.sum_duplicates()
        S.sum_duplicates()
        return T, S

    def gradient_matrix(self):
        """Discrete gradient D0 [n_edges_interior, n_nodes_interior] (signed incidence).

        grad(phi_a) = sum_e D0[e,a] W_e for the nodal hat function phi_a of an
        interior node a (D0[e,a] = -1 if e starts at a, +1 if it ends at a).
        """
        bmask = boundary_node_mask(self.tets, len(self.xyz))
        interior_nodes = np.flatnonzero(~bmask)
        nmap = -np.ones(len(self.xyz), dtype=np.int64)
        nmap[interior_nodes] = np.arange(len(interior_nodes))
        rows, cols, vals = [], [], []
        for dof, ge in enumerate(self.interior_edges):
            a, b = self.edges[ge]
            if nmap[a] >= 0:
                rows.append(dof); cols.append(nmap[a]); vals.append(-1.0)
            if nmap[b] >= 0:
                rows.append(dof); cols.append(nmap[b]); vals.append(1.0)
        return sp.csr_matrix((vals, (rows, cols)), shape=(self.n, len(interior_nodes)))

    def dof_of_pairs(self, pairs):
        """Interior-dof ids of node pairs (lo, hi); raises if a pair is not an interior edge."""
        n = int(self.tets.max()) + 1
        keys = self.edges[:, 0] * n + self.edges[:, 1]
        pk = np.asarray(pairs)[:, 0] * n + np.asarray(pairs)[:, 1]
        pos = np.searchsorted(keys, pk)
        assert np.all(keys[pos] == pk), "source pair is not a mesh edge"
        d = self.edge_to_dof[pos]
        assert np.all(d >= 0), "source edge lies on the PEC wall"
        return d

    def locate(self, p):
        """Lowest-id tet containing point p (barycentrics >= -1e-12) and its barycentrics."""
        X = self.xyz[self.tets]
        D = np.stack([X[:, 1] - X[:, 0], X[:, 2] - X[:, 0], X[:, 3] - X[:, 0]], axis=1)
        l123 = np.linalg.solve(np.swapaxes(D, 1, 2), (np.asarray(p) - X[:, 0])[:, :, None])[:, :, 0]
        lam = np.concatenate([1.0 - l123.sum(axis=1, keepdims=True), l123], axis=1)
        inside = np.flatnonzero(np.all(lam >= -1e-12, axis=1))
        assert len(inside) > 0, "probe outside mesh"
        k = int(inside[0])
        return k, lam[k]

    def probe_operator(self, points):
        """Sparse P [3*n_points, n] with E(points) = P e (E = sum_i e_i W_i)."""
        rows, cols, vals = [], [], []
        for pi, p in enumerate(np.asarray(points, dtype=np.float64)):
            k, lam = self.locate(p)
            W = whitney_at(self.xyz[self.tets[k]], lam) * self.tet_sign[k][:, None]
            for le in range(6):
                d = self.tet_dof[k, le]
                if d < 0:
                    continue
                for c in range(3):
                    rows.append(3 * pi + c); cols.append(d); vals.append(W[le, c])
        P = sp.csr_matrix((vals, (rows, cols)), shape=(3 * len(points), self.n))
        P.sum_duplicates()
        return P
