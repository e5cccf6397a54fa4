"""Seeded synthetic inputs for the Maxwell DD time step.

This module generates the *inputs* of the method and nothing else: tetrahedral
meshes, subdomain labels, per-tet permittivities, the excitation current and
probe points.  It holds none of the method's arithmetic (no Whitney elements, no
assembly, no solves), so both the CUDA path and the CPU oracle may be fed from it.

Workloads (all in normalised units, c = eps0 = mu0 = 1):

* ``kuhn_box`` -- a box of nx*ny*nz cubes, each split into the six Kuhn
  tetrahedra that share the cube's (0,0,0)->(1,1,1) body diagonal.  Every cube
  is split the same way, so face diagonals agree across neighbouring cubes and
  the mesh is conforming.  Nodes are numbered lexicographically (i fastest).
  This stands in for the paper's METIS-split box and cavity meshes (Sec. V),
  which are not available.
* ``block_partition`` -- kx*ky*kz equal blocks of cubes (subdomain id x-fastest).
* ``jitter_nodes`` / ``rcb_partition`` -- the uneven-subdomain workload:
  interior nodes perturbed by up to +-20% of h, and recursive coordinate
  bisection with random target weights, so subdomain sizes vary.
* ``gaussian_pulse_G`` -- time integral G(t) of a Gaussian current pulse
  I(t) = exp(-(t-t0)^2 / (2 sigma^2)) switched on at t = 0 (the integrated
  current of Sec. II-A that enters the right-hand side).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

# ----------------------------------------------------------------------------
# Meshes
# ----------------------------------------------------------------------------

# The six Kuhn tetrahedra of the unit cube: monotone lattice paths from corner
# (0,0,0) to (1,1,1), one per permutation of the axes.  Each entry lists the
# axis order; the tet is (v000, v000+e_a, v000+e_a+e_b, v111).
_KUHN_PERMS = [(0, 1, 2), (0, 2, 1), (1, 0, 2), (1, 2, 0), (2, 0, 1), (2, 1, 0)]


def _perm_parity(p):
    inv = 0
    for i in range(3):
        for j in range(i + 1, 3):
            if p[i] > p[j]:
                inv += 1
    return inv % 2


def kuhn_box(nx: int, ny: int, nz: int, Lx: float = 1.0, Ly: float = 1.0, Lz: float = 1.0):
    """Structured Kuhn tetrahedral mesh of [0,Lx]x[0,Ly]x[0,Lz].

    Returns ``xyz`` float64 [N,3] and ``tets`` int32 [6*nx*ny*nz, 4] with
    positive orientation.  Tets are ordered cube by cube (cube index i fastest),
    six per cube in the order of ``_KUHN_PERMS``.
    """
    ii, jj, kk = np.meshgrid(np.arange(nx + 1), np.arange(ny + 1), np.arange(nz + 1), indexing="ij")
    # lexicographic, i fastest: id = i + (nx+1)*(j + (ny+1)*k)
    xyz = np.zeros(((nx + 1) * (ny + 1) * (nz + 1), 3))
    nid = ii + (nx + 1) * (jj + (ny + 1) * kk)
    xyz[nid.ravel(), 0] = ii.ravel() * (Lx / nx)
    xyz[nid.ravel(), 1] = jj.ravel() * (Ly / ny)
    xyz[nid.ravel(), 2] = kk.ravel() * (Lz / nz)

    def node(i, j, k):
        return i + (nx + 1) * (j + (ny + 1) * k)

    ci, cj, ck = np.meshgrid(np.arange(nx), np.arange(ny), np.arange(nz), indexing="ij")
    # cube order: i fastest
    ci = ci.transpose(2, 1, 0).ravel()
    cj = cj.transpose(2, 1, 0).ravel()
    ck = ck.transpose(2, 1, 0).ravel()
    tets = np.zeros((ci.size, 6, 4), dtype=np.int64)
    for t, p in enumerate(_KUHN_PERMS):
        off = np.zeros(3, dtype=np.int64)
        verts = [node(ci, cj, ck)]
        for a in p:
            off = off.copy()
            off[a] += 1
            verts.append(node(ci + off[0], cj + off[1], ck + off[2]))
        v = np.stack(verts, axis=1)
        if _perm_parity(p) == 1:  # odd permutation -> negative volume; swap two vertices
            v[:, [1, 2]] = v[:, [2, 1]]
        tets[:, t, :] = v
    return xyz, tets.reshape(-1, 4).astype(np.int32)


def box_boundary_nodes(xyz: np.ndarray, L=(1.0, 1.0, 1.0), tol: float = 1e-12):
    """Boolean mask of nodes on the faces of the box [0,L]."""
    m = np.zeros(len(xyz), dtype=bool)
    for a in range(3):
        m |= np.abs(xyz[:, a]) < tol
        m |= np.abs(xyz[:, a] - L[a]) < tol
    return m


def jitter_nodes(xyz: np.ndarray, h: float, L, frac: float = 0.2, seed: int = 7):
    """Perturb nodes by U[-frac*h, frac*h] per coordinate (seeded).

    Interior nodes move in all three directions; nodes on a box face move only
    tangentially to every face they lie on, so the box stays a box.
    """
    rng = np.random.default_rng(seed)
    d = rng.uniform(-frac * h, frac * h, size=xyz.shape)
    out = xyz.copy()
    for a in range(3):
        on_face = (np.abs(xyz[:, a]) < 1e-12) | (np.abs(xyz[:, a] - L[a]) < 1e-12)
        d[on_face, a] = 0.0
    out += d
    return out, rng


def block_partition(nx, ny, nz, kx, ky, kz):
    """Subdomain label per tet for a kx*ky*kz block split of a Kuhn box.

    Requires nx % kx == ny % ky == nz % kz == 0.  Subdomain id is
    bx + kx*(by + ky*bz).
    """
    assert nx % kx == 0 and ny % ky == 0 and nz % kz == 0
    ci, cj, ck = np.meshgrid(np.arange(nx), np.arange(ny), np.arange(nz), indexing="ij")
    ci = ci.transpose(2, 1, 0).ravel()
    cj = cj.transpose(2, 1, 0).ravel()
    ck = ck.transpose(2, 1, 0).ravel()
    b = (ci // (nx // kx)) + kx * ((cj // (ny // ky)) + ky * (ck // (nz // kz)))
    return np.repeat(b, 6).astype(np.int32)


def tet_centroids(xyz, tets):
    return xyz[tets].mean(axis=1)


def rcb_partition(centroids: np.ndarray, n_parts: int, weights: np.ndarray):
    """Recursive coordinate bisection of tets into ``n_parts`` subdomains.

    A set of tets destined for k parts is split into floor(k/2) and ceil(k/2)
    parts along the axis of largest centroid extent, at the point where the
    cumulative target weight of the first half is reached.  Ties in the
    coordinate are broken by tet id.  ``weights[k]`` is the relative target size
    of part k (part ids are assigned in depth-first order).
    """
    part = np.empty(len(centroids), dtype=np.int32)

    def rec(ids, p0, k):
        if k == 1:
            part[ids] = p0
            return
        c = centroids[ids]
        ext = c.max(axis=0) - c.min(axis=0)
        ax = int(np.argmax(ext))
        order = np.lexsort((ids, c[:, ax]))
        ids = ids[order]
        k1 = k // 2
        w1 = weights[p0:p0 + k1].sum()
        w = weights[p0:p0 + k].sum()
        n1 = int(round(len(ids) * w1 / w))
        n1 = min(max(n1, 1), len(ids) - 1)
        rec(ids[:n1], p0, k1)
        rec(ids[n1:], p0 + k1, k - k1)

    rec(np.arange(len(centroids)), 0, n_parts)
    return part


# ----------------------------------------------------------------------------
# Excitation and probes
# ----------------------------------------------------------------------------

def gaussian_pulse_G(t, t0: float, sigma: float):
    """G(t) = int_0^t I(s) ds for I(s) = exp(-(s-t0)^2/(2 sigma^2)), I = 0 for s < 0."""
    t = np.asarray(t, dtype=np.float64)
    s2 = sigma * math.sqrt(2.0)
    erf = np.vectorize(math.erf)
    g = sigma * math.sqrt(math.pi / 2.0) * (erf((t - t0) / s2) + math.erf(t0 / s2))
    return np.where(t > 0.0, g, 0.0)


def z_line_node_pairs(nx, ny, nz, i, j):
    """Node pairs (lower id, upper id) of the z-directed grid line through (i,j)."""
    def node(i_, j_, k_):
        return i_ + (nx + 1) * (j_ + (ny + 1) * k_)
    return np.array([[node(i, j, k), node(i, j, k + 1)] for k in range(nz)], dtype=np.int64)


@dataclass
class Workload:
    """One synthetic field-solve workload."""
    name: str
    xyz: np.ndarray
    tets: np.ndarray
    part: np.ndarray
    n_sub: int
    eps: np.ndarray | None
    mu: float
    steps: int
    source_pairs: np.ndarray          # [n_src, 2] node ids (low, high), current flows low->high
    t0_over_dt: float = 20.0
    sigma_over_dt: float = 6.0
    probes: np.ndarray = field(default_factory=lambda: np.zeros((0, 3)))
    dims: tuple = (1, 1, 1)
    L: tuple = (1.0, 1.0, 1.0)

    def G_at_steps(self, dt: float, n_steps: int):
        """Integrated source current G(t_m) for m = -1..n_steps (length n_steps+2)."""
        t = dt * np.arange(-1, n_steps + 1, dtype=np.float64)
        return gaussian_pulse_G(t, self.t0_over_dt * dt, self.sigma_over_dt * dt)

    def d2G(self, dt: float, n_steps: int):
        """Second differences G^{n+1} - 2 G^n + G^{n-1}, n = 0..n_steps-1 (one per step)."""
        g = self.G_at_steps(dt, n_steps)
        return g[2:] - 2.0 * g[1:-1] + g[:-2]


def cavity(n: int, k: int, steps: int = 200, probes=None) -> Workload:
    """Unit PEC cube, n^3 Kuhn cubes, k^3 block subdomains, z-line pulse at x=y=1/2."""
    assert n % 2 == 0
    xyz, tets = kuhn_box(n, n, n)
    part = block_partition(n, n, n, k, k, k)
    if probes is None:
        probes = np.array([[0.30, 0.40, 0.55]])
    return Workload(name=f"cavity{n}_k{k}", xyz=xyz, tets=tets, part=part, n_sub=k ** 3, eps=None,
                    mu=1.0, steps=steps, source_pairs=z_line_node_pairs(n, n, n, n // 2, n // 2),
                    probes=np.asarray(probes, dtype=np.float64), dims=(n, n, n))


def box(nx, ny, nz, kx, ky, kz, L=(1.0, 1.0, 1.0), steps=200, probes=None, eps=None, src_ij=None) -> Workload:
    """General Kuhn box with block subdomains and a z-line source through node column src_ij."""
    xyz, tets = kuhn_box(nx, ny, nz, *L)
    part = block_partition(nx, ny, nz, kx, ky, kz)
    if src_ij is None:
        src_ij = (nx // 2, ny // 2)
    if probes is None:
        probes = np.array([[0.30 * L[0], 0.40 * L[1], 0.55 * L[2]]])
    return Workload(name=f"box{nx}x{ny}x{nz}_k{kx}x{ky}x{kz}", xyz=xyz, tets=tets, part=part,
                    n_sub=kx * ky * kz, eps=eps, mu=1.0, steps=steps,
                    source_pairs=z_line_node_pairs(nx, ny, nz, *src_ij),
                    probes=np.asarray(probes, dtype=np.float64), dims=(nx, ny, nz), L=tuple(L))


def beam(w: Workload, n_particles: int, t_max: float, speed: float = 0.1, sigma: float = 0.05, q: float = -1e-6,
         qm: float = -1.0, seed: int = 0, clip: float = 0.45):
    """Electron-like beam entering through the z = 0 wall on the axis x = y = L/2.

    Transverse offsets ~ N(0, sigma^2) clipped to +-clip, velocity (0, 0, speed),
    injection times ~ U[0, t_max) (seeded).  Returns (x_inj, v_inj, t_inj, q, qm).
    """
    rng = np.random.default_rng(seed)
    off = np.clip(rng.normal(0.0, sigma, size=(n_particles, 2)), -clip, clip)
    x = np.column_stack([w.L[0] / 2 + off[:, 0], w.L[1] / 2 + off[:, 1], np.zeros(n_particles)])
    v = np.tile([0.0, 0.0, speed], (n_particles, 1))
    t = rng.uniform(0.0, t_max, size=n_particles)
    return x, v, t, q, qm


PROBES_ADJOINT = np.array([[0.2, 0.3, 0.4], [0.7, 0.6, 0.3], [0.4, 0.8, 0.7], [0.6, 0.25, 0.8]])


def config(idx: int) -> Workload:
    """The five field-solve workloads (1-based index).

    1: unit PEC cavity, 8^3 cubes, 2x2x2 subdomains, 200 steps.
    2: 1x1x2 box, 16x16x32 cubes, 4x4x8 subdomains, 2000 steps (beam-shaped box;
       the field-solve stage is driven here by the z-line pulse).
    3: jittered 2x1x1 box, 64x32x32 cubes (+-20% h node jitter, seed 7), 300
       RCB subdomains with +-40% target weights, 500 steps.
    4: unit cavity, 48^3 cubes, 8x8x8 subdomains, 1000 steps.
    5: unit cavity, 32^3 cubes, 8x8x4 subdomains, eps ~ U[1,4] (seed 11), 4 probes, 1500 steps.
    """
    if idx == 1:
        return cavity(8, 2, steps=200)
    if idx == 2:
        return box(16, 16, 32, 4, 4, 8, L=(1.0, 1.0, 2.0), steps=2000)
    if idx == 3:
        nx, ny, nz = 64, 32, 32
        L = (2.0, 1.0, 1.0)
        xyz, tets = kuhn_box(nx, ny, nz, *L)
        h = L[0] / nx
        xyz, rng = jitter_nodes(xyz, h, L, 0.2, seed=7)
        w = rng.uniform(0.6, 1.4, size=300)
        part = rcb_partition(tet_centroids(xyz, tets), 300, w)
        return Workload(name="jitter64x32x32_rcb300", xyz=xyz, tets=tets, part=part, n_sub=300, eps=None,
                        mu=1.0, steps=500, source_pairs=z_line_node_pairs(nx, ny, nz, 32, 16),
                        probes=np.array([[0.61, 0.40, 0.55]]), dims=(nx, ny, nz), L=L)
    if idx == 4:
        return cavity(48, 8, steps=1000)
    if idx == 5:
        rng = np.random.default_rng(11)
        w = box(32, 32, 32, 8, 8, 4, steps=1500, probes=PROBES_ADJOINT)
        w.eps = rng.uniform(1.0, 4.0, size=len(w.tets))
        w.name = "cavity32_k8x8x4_eps"
        return w
    raise ValueError(idx)
