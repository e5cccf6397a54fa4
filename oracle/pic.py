"""Particle-in-cell coupling around the field solve (oracle; test infrastructure only).

Paper Sec. II (PIC cycle: gather the particles onto the mesh, solve for the
fields, interpolate the fields at the particles, push) and Sec. II-A (the
charge is a 0-form, the current a 1-form, and the integrated current G enters
the right-hand side so that Gauss' law holds for any time marching).

* Current deposition: a particle of charge q moving on a straight segment
  from p0 to p1 inside a tet adds q * int_{p0}^{p1} W_e . dl to g_e for every
  edge e of the tet; for the Whitney form of edge (a,b) this line integral is
  lambda_a(p0) lambda_b(p1) - lambda_b(p0) lambda_a(p1).  Segments are cut at
  the faces they cross.  Because sum_e D0[e,a] W_e = grad(phi_a), the deposit
  changes D0^T g by exactly the change of the particle's 0-form charge
  q phi_a(x): charge conservation holds per particle.
* Magnetic flux: the paper's second unknown B lives on faces (Whitney 2-forms,
  Sec. II-B).  With edge unknowns only, B follows from Faraday's law, applied
  with the trapezoidal (gamma = 1/2) rule of the Newmark march:
  b^{n+1} = b^n - dt/2 * C (e^{n+1} + e^n), C the face-edge incidence (the
  discrete curl).  B(x) = sum_f b_f W2_f(x), W2_abc = 2 (l_a grad l_b x grad l_c
  + l_b grad l_c x grad l_a + l_c grad l_a x grad l_b).
* Push: the Boris scheme (leapfrog; positions at t_n, velocities at t_{n-1/2}),
  non-relativistic, with E and B at x^n.  The paper uses Adams-Bashforth; the
  Boris push is the reading used here.
* Injection: a particle appears at its injection time t_i on the wall z = 0
  (so no charge appears inside the domain) and moves without a push for the
  rest of that step.  A particle whose path reaches a wall stops there (its
  charge stays on the wall nodes).
"""
from __future__ import annotations

import numpy as np

from .fem import LOCAL_EDGES, LOCAL_FACES, barycentric_gradients

ALIVE, WAITING, DEAD = 1, 0, 2


class Mesh:
    """Faces, tet adjacency, discrete curl and the per-tet data a particle needs."""

    def __init__(self, space):
        self.space = space
        tets = space.tets
        T = len(tets)
        f = np.concatenate([np.sort(tets[:, list(fc)], axis=1) for fc in LOCAL_FACES], axis=0)   # [4T,3], face k of tet t at row k*T+t
        self.faces, inv = np.unique(f, axis=0, return_inverse=True)
        self.tet_face = inv.reshape(4, T).T                                  # [T,4] global face opposite local vertex k
        owners = [[] for _ in range(len(self.faces))]
        for k in range(4):
            for t in range(T):
                owners[self.tet_face[t, k]].append(t)
        self.neighbor = -np.ones((T, 4), dtype=np.int64)
        for t in range(T):
            for k in range(4):
                o = owners[self.tet_face[t, k]]
                if len(o) == 2:
                    self.neighbor[t, k] = o[0] if o[1] == t else o[1]
        self.g, self.vol = barycentric_gradients(space.xyz[tets])           # [T,4,3]
        self.x0 = space.xyz[tets[:, 0]]
        # discrete curl on all faces: (C e)_f = e_ab + e_bc - e_ac for the sorted triple (a,b,c)
        n = int(tets.max()) + 1
        ek = space.edges[:, 0] * n + space.edges[:, 1]
        def dof(a, b):
            pos = np.searchsorted(ek, a * n + b)
            return space.edge_to_dof[pos]
        self.face_edge_dof = np.stack([dof(self.faces[:, 0], self.faces[:, 1]), dof(self.faces[:, 1], self.faces[:, 2]),
                                       dof(self.faces[:, 0], self.faces[:, 2])], axis=1)
        self.face_edge_sign = np.array([1.0, 1.0, -1.0])

    def curl(self, e):
        d = self.face_edge_dof
        v = np.where(d >= 0, e[np.maximum(d, 0)], 0.0)
        return v @ self.face_edge_sign

    def lam(self, t, x):
        l123 = self.g[t, 1:] @ (x - self.x0[t])
        return np.concatenate([[1.0 - l123.sum()], l123])

    def E_at(self, t, x, e):
        lam = self.lam(t, x)
        g = self.g[t]
        out = np.zeros(3)
        for k, (a, b) in enumerate(LOCAL_EDGES):
            d = self.space.tet_dof[t, k]
            if d >= 0:
                out += e[d] * self.space.tet_sign[t, k] * (lam[a] * g[b] - lam[b] * g[a])
        return out

    def B_at(self, t, x, bflux):
        lam = self.lam(t, x)
        g = self.g[t]
        nodes = self.space.tets[t]
        out = np.zeros(3)
        for k in range(4):
            fid = self.tet_face[t, k]
            a, b, c = [int(np.flatnonzero(nodes == v)[0]) for v in self.faces[fid]]
            W2 = 2.0 * (lam[a] * np.cross(g[b], g[c]) + lam[b] * np.cross(g[c], g[a]) + lam[c] * np.cross(g[a], g[b]))
            out += bflux[fid] * W2
        return out


def deposit_path(mesh, t, p0, p1, q, g_out, max_cross=64):
    """Move from p0 (inside tet t) toward p1, adding q * int W_e.dl to g_out.

    Returns (tet, end point, alive): alive is False when the path hit a wall."""
    space = mesh.space
    for _ in range(max_cross):
        l0 = mesh.lam(t, p0)
        l1 = mesh.lam(t, p1)
        s_exit, k_exit = 1.0, -1
        for k in range(4):
            if l1[k] < 0.0 and l1[k] < l0[k]:
                s = max(l0[k], 0.0) / (l0[k] - l1[k])
                if s < s_exit:
                    s_exit, k_exit = s, k
        pe = p1 if k_exit < 0 else p0 + s_exit * (p1 - p0)
        le = l1 if k_exit < 0 else l0 + s_exit * (l1 - l0)
        for k, (a, b) in enumerate(LOCAL_EDGES):
            d = space.tet_dof[t, k]
            if d >= 0:
                g_out[d] += q * space.tet_sign[t, k] * (l0[a] * le[b] - l0[b] * le[a])
        if k_exit < 0:
            return t, p1, True
        nb = mesh.neighbor[t, k_exit]
        if nb < 0:
            return t, pe, False
        t, p0 = nb, pe
    raise RuntimeError("particle crossed too many tets in one step")


def boris(v, E, B, qm, dt):
    vm = v + 0.5 * qm * dt * E
    tv = 0.5 * qm * dt * B
    vp = vm + np.cross(vm, tv)
    s = 2.0 * tv / (1.0 + tv @ tv)
    return vm + np.cross(vp, s) + 0.5 * qm * dt * E


class Beam:
    """Particle state: injection data, position, velocity, tet, status."""

    def __init__(self, mesh, x_inj, v_inj, t_inj, q, qm):
        self.mesh = mesh
        self.x = np.array(x_inj, dtype=np.float64)
        self.v = np.array(v_inj, dtype=np.float64)
        self.t_inj = np.asarray(t_inj, dtype=np.float64)
        self.q, self.qm = float(q), float(qm)
        self.status = np.full(len(self.x), WAITING)
        self.tet = np.array([self.locate_on_wall(p) for p in self.x])

    def locate_on_wall(self, p):
        g, x0 = self.mesh.g, self.mesh.x0
        l123 = np.einsum("tij,tj->ti", g[:, 1:], p - x0)
        lam = np.concatenate([1.0 - l123.sum(axis=1, keepdims=True), l123], axis=1)
        ins = np.flatnonzero(np.all(lam >= -1e-12, axis=1))
        assert len(ins), "injection point outside the mesh"
        return int(ins[0])

    def step(self, t_n, dt, e, bflux):
        """Advance every particle from t_n to t_n + dt; returns the deposit over the step."""
        dep = np.zeros(self.mesh.space.n)
        t1 = t_n + dt
        for i in range(len(self.x)):
            if self.status[i] == DEAD:
                continue
            if self.status[i] == WAITING:
                if self.t_inj[i] > t1:
                    continue
                # inject at t_inj on the wall, move for the rest of the step without a push
                tau = t1 - max(self.t_inj[i], t_n)
                self.status[i] = ALIVE
            else:
                tt = self.tet[i]
                self.v[i] = boris(self.v[i], self.mesh.E_at(tt, self.x[i], e), self.mesh.B_at(tt, self.x[i], bflux),
                                  self.qm, dt)
                tau = dt
            p1 = self.x[i] + tau * self.v[i]
            t, pe, alive = deposit_path(self.mesh, self.tet[i], self.x[i], p1, self.q, dep)
            self.tet[i], self.x[i] = t, pe
            if not alive:
                self.status[i] = DEAD
        return dep

    def charge_at_nodes(self, n_nodes):
        """0-form charge q phi_a(x) of the particles in flight, per mesh node."""
        rho = np.zeros(n_nodes)
        for i in np.flatnonzero(self.status == ALIVE):
            lam = self.mesh.lam(self.tet[i], self.x[i])
            np.add.at(rho, self.mesh.space.tets[self.tet[i]], self.q * lam)
        return rho


def run(space, dd_solve_step, beam, dt, n_steps, keep=True):
    """PIC march: push/deposit with (e^n, b^n), field step with d2g = dep^{n+1/2} - dep^{n-1/2},
    Faraday update of b.  dd_solve_step(e_n, e_nm1, d2g) -> e^{n+1}."""
    mesh = beam.mesh
    n = space.n
    e_nm1, e_n = np.zeros(n), np.zeros(n)
    b = np.zeros(len(mesh.faces))
    dep_prev = np.zeros(n)
    G = np.zeros(n)
    out = dict(fields=[], G=[], x=[])
    for k in range(n_steps):
        dep = beam.step(k * dt, dt, e_n, b)
        G = G + dep
        e_np1 = dd_solve_step(e_n, e_nm1, dep - dep_prev)
        b = b - 0.5 * dt * (mesh.curl(e_np1) + mesh.curl(e_n))
        dep_prev = dep
        e_nm1, e_n = e_n, e_np1
        if keep:
            out["fields"].append(e_n.copy())
            out["G"].append(G.copy())
            out["x"].append(beam.x.copy())
    out["b"] = b
    return out
