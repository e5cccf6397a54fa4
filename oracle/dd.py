"""MFETI-DP1 domain decomposition of the Newmark step (oracle; test infrastructure only).

Paper Sec. III-A.  The mesh is torn into N_v non-overlapping subdomains (the
subdomain of a tet is given).  Readings of the paper used here:

* Unknowns are the interior (non-PEC) edges.  The multiplicity m(e) of an edge
  is the number of distinct subdomains among the tets that contain it.
  m = 1: interior of a subdomain; m = 2: interface edge with one Lagrange
  multiplier (the signed Boolean B_r of Sec. III-A is +1 in the lower subdomain
  id and -1 in the higher); m >= 3: a "corner" (the junction of more than two
  volumes), kept primal and assembled with the unsigned Boolean B_c.
* Local edge order in a subdomain: [interior, interface (r), corner], each
  group sorted by global edge id; multipliers and corners are numbered in
  global edge order.
* Eqs. rF1, F1lr, F1uc and f1schur with the evident misprints corrected:
  x_r = A_rr^-1 (L_r - A_rc B_c x_c - B_r^T lambda)     (rF1, no inverse on A_rc)
  F_rr = sum B_r A_rr^-1 B_r^T                             (K_rr, inverse restored)
  F_rc = sum B_r A_rr^-1 A_rc B_c                          (second "K_rr" is K_rc)
  K~cc = sum B_c^T (A_cc - A_cr A_rr^-1 A_rc) B_c          (K_cc, no stray inverses)
  d_r  = sum B_r A_rr^-1 L_r,  f~_c = sum B_c^T (L_c - A_cr A_rr^-1 L_r)
  (F_rr + F_rc K~cc^-1 F_rc^T) lambda = d_r - F_rc K~cc^-1 f~_c       (f1schur)
  x_c = K~cc^-1 (f~_c + F_rc^T lambda)                                (F1uc)
* The interface Krylov solver of Sec. III-C (GMRES with a diagonal
  preconditioner) is taken as CG, the Schur system being symmetric positive
  definite, with the Jacobi preconditioner diag(F_rr); it stops when
  ||r_k|| <= tol ||rhs||.
* The coupled variant (end of Sec. III-A; Fig. fetiIter) solves Eqs. F1lr and
  F1uc together for u = [lambda; x_c]:
      [ F_rr     F_rc ] [lambda]   [d_r ]
      [ -F_rc^T  K~cc ] [x_c   ] = [f~_c]
  with restarted GMRES (oracle.gmres) and the diagonal preconditioner
  diag(F_rr) (+) diag(K~cc).  The matrix is not symmetric; its symmetric part
  is blockdiag(F_rr, K~cc), positive definite, so GMRES(m) converges.  The warm
  start is the previous step's [lambda; x_c].
* The local right-hand side L^(i) is the subassembled Newmark right side
  B^(i) e^n - A^(i) e^{n-1} on the (consistent) local copies of the fields,
  plus the source on the lowest-id subdomain that owns the edge.  The global
  field is read from the lowest-id subdomain that owns each edge.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp

from .gmres import gmres


class DDMaps:
    """Tearing maps of Sec. III-A for a labelled tet mesh."""

    def __init__(self, space, part, n_sub):
        part = np.asarray(part, dtype=np.int64)
        self.n_sub = int(n_sub)
        d = space.tet_dof
        pairs = np.stack([d.ravel(), np.repeat(part, 6)], axis=1)
        pairs = pairs[pairs[:, 0] >= 0]
        pairs = np.unique(pairs, axis=0)                 # (dof, sub) sorted by dof then sub
        n = space.n
        self.mult = np.bincount(pairs[:, 0], minlength=n)
        self.owner = np.full(n, -1, dtype=np.int64)      # lowest subdomain containing the dof
        first = np.ones(len(pairs), dtype=bool)
        first[1:] = pairs[1:, 0] != pairs[:-1, 0]
        self.owner[pairs[first, 0]] = pairs[first, 1]
        self.local = []        # per subdomain: global dof ids in local order [I, G, C]
        self.nI = np.zeros(self.n_sub, dtype=np.int64)
        self.nG = np.zeros(self.n_sub, dtype=np.int64)
        self.nC = np.zeros(self.n_sub, dtype=np.int64)
        for s in range(self.n_sub):
            dofs = pairs[pairs[:, 1] == s, 0]
            m = self.mult[dofs]
            I, G, C = dofs[m == 1], dofs[m == 2], dofs[m >= 3]
            self.nI[s], self.nG[s], self.nC[s] = len(I), len(G), len(C)
            self.local.append(np.concatenate([I, G, C]))
        self.nr = self.nI + self.nG
        # multipliers: edges of multiplicity 2, in global order
        self.mult_dof = np.flatnonzero(self.mult == 2)
        self.mult_sub = np.zeros((len(self.mult_dof), 2), dtype=np.int64)
        self.mult_loc = np.zeros((len(self.mult_dof), 2), dtype=np.int64)
        pos = {}
        for s in range(self.n_sub):
            for li, g in enumerate(self.local[s]):
                pos[(s, g)] = li
        subs_of = {}
        for g, s in pairs:
            subs_of.setdefault(g, []).append(s)
        for k, g in enumerate(self.mult_dof):
            s1, s2 = sorted(subs_of[g])
            self.mult_sub[k] = (s1, s2)
            self.mult_loc[k] = (pos[(s1, g)], pos[(s2, g)])
        # corners
        self.corner_dof = np.flatnonzero(self.mult >= 3)
        cidx = -np.ones(n, dtype=np.int64)
        cidx[self.corner_dof] = np.arange(len(self.corner_dof))
        self.corner_of_local = [cidx[self.local[s][self.nr[s]:]] for s in range(self.n_sub)]
        self.tets_of = [np.flatnonzero(part == s) for s in range(self.n_sub)]

    @property
    def n_lambda(self):
        return len(self.mult_dof)

    @property
    def n_corner(self):
        return len(self.corner_dof)


class DDSolver:
    """CPU MFETI-DP1 solve of A x = b with A = T + (dt^2/4) S, subassembled per subdomain."""

    def __init__(self, space, maps: DDMaps, dt):
        self.space, self.maps, self.dt = space, maps, float(dt)
        self.A, self.B, self.chol = [], [], []
        self.Acc_tilde = np.zeros((maps.n_corner, maps.n_corner))
        for s in range(maps.n_sub):
            loc = maps.local[s]
            dof_map = -np.ones(space.n, dtype=np.int64)
            dof_map[loc] = np.arange(len(loc))
            Ts, Ss = space.assemble(maps.tets_of[s], dof_map, len(loc))
            As = (Ts + (dt * dt / 4.0) * Ss).toarray()
            Bs = (2.0 * Ts - (dt * dt / 2.0) * Ss).toarray()
            self.A.append(As)
            self.B.append(Bs)
            nr = maps.nr[s]
            cf = sla.cho_factor(As[:nr, :nr], lower=True)
            self.chol.append(cf)
            Arc = As[:nr, nr:]
            Sc = As[nr:, nr:] - Arc.T @ sla.cho_solve(cf, Arc)
            ci = maps.corner_of_local[s]
            self.Acc_tilde[np.ix_(ci, ci)] += Sc
        self.Kcc = sla.cho_factor(self.Acc_tilde, lower=True) if maps.n_corner else None
        # Jacobi diagonal of F_rr: (A_rr^-1)_{ii} of the two subdomains of each multiplier
        self.diag = np.zeros(maps.n_lambda)
        for side in range(2):
            for k in range(maps.n_lambda):
                s, li = maps.mult_sub[k, side], maps.mult_loc[k, side]
                u = np.zeros(maps.nr[s]); u[li] = 1.0
                self.diag[k] += sla.cho_solve(self.chol[s], u)[li]
        self.diag_c = np.diag(self.Acc_tilde).copy()
        self.lam = np.zeros(maps.n_lambda)
        self.xc = np.zeros(maps.n_corner)

    # -- Boolean maps ---------------------------------------------------------
    def Br_T(self, lam, s):
        """(B_r^(s))^T lambda as a local r-vector."""
        m = self.maps
        z = np.zeros(m.nr[s])
        sel = m.mult_sub[:, 0] == s
        z[m.mult_loc[sel, 0]] += lam[sel]
        sel = m.mult_sub[:, 1] == s
        z[m.mult_loc[sel, 1]] -= lam[sel]
        return z

    def Br_sum(self, xr):
        """sum_s B_r^(s) x_r^(s): the jump x_{s1}[i1] - x_{s2}[i2] across every interface edge."""
        m = self.maps
        off = np.concatenate([[0], np.cumsum([len(v) for v in xr])])
        flat = np.concatenate(xr) if len(xr) else np.zeros(0)
        return (flat[off[m.mult_sub[:, 0]] + m.mult_loc[:, 0]]
                - flat[off[m.mult_sub[:, 1]] + m.mult_loc[:, 1]])

    def Bc_sum(self, xc):
        out = np.zeros(self.maps.n_corner)
        for s in range(self.maps.n_sub):
            np.add.at(out, self.maps.corner_of_local[s], xc[s])
        return out

    # -- operators of Eqs. F1lr / F1uc ------------------------------------------
    def Arr_solve(self, s, v):
        return sla.cho_solve(self.chol[s], v)

    def F_rr(self, lam):
        return self.Br_sum([self.Arr_solve(s, self.Br_T(lam, s)) for s in range(self.maps.n_sub)])

    def F_rc(self, xc):
        m = self.maps
        out = []
        for s in range(m.n_sub):
            nr = m.nr[s]
            out.append(self.Arr_solve(s, self.A[s][:nr, nr:] @ xc[m.corner_of_local[s]]))
        return self.Br_sum(out)

    def F_rcT(self, lam):
        m = self.maps
        out = []
        for s in range(m.n_sub):
            nr = m.nr[s]
            out.append(self.A[s][nr:, :nr] @ self.Arr_solve(s, self.Br_T(lam, s)))
        return self.Bc_sum(out)

    def Kcc_solve(self, v):
        return sla.cho_solve(self.Kcc, v) if self.Kcc is not None else v

    def schur_apply(self, lam):
        """(F_rr + F_rc K~cc^-1 F_rc^T) lambda   (Eq. f1schur)."""
        out = self.F_rr(lam)
        if self.maps.n_corner:
            out = out + self.F_rc(self.Kcc_solve(self.F_rcT(lam)))
        return out

    def coupled_apply(self, u):
        """[F_rr lambda + F_rc x_c ; -F_rc^T lambda + K~cc x_c]   (Eqs. F1lr, F1uc)."""
        nl = self.maps.n_lambda
        lam, xc = u[:nl], u[nl:]
        top = self.F_rr(lam) + self.F_rc(xc)
        bottom = self.Acc_tilde @ xc - self.F_rcT(lam)
        return np.concatenate([top, bottom])

    def recover(self, b_local, lam, x_c):
        """x_r = A_rr^-1 (b_r - A_rc B_c x_c - B_r^T lambda) per subdomain   (Eq. rF1)."""
        m = self.maps
        x = []
        for s in range(m.n_sub):
            nr = m.nr[s]
            xc_s = x_c[m.corner_of_local[s]]
            xr = self.Arr_solve(s, b_local[s][:nr] - self.A[s][:nr, nr:] @ xc_s - self.Br_T(lam, s))
            x.append(np.concatenate([xr, xc_s]))
        return x

    def rhs_parts(self, b_local):
        """d_r = sum B_r A_rr^-1 b_r and f~_c = sum B_c^T (b_c - A_cr A_rr^-1 b_r)."""
        m = self.maps
        y = []
        fc_parts = []
        for s in range(m.n_sub):
            nr = m.nr[s]
            ys = self.Arr_solve(s, b_local[s][:nr])
            y.append(ys)
            fc_parts.append(b_local[s][nr:] - self.A[s][nr:, :nr] @ ys)
        return self.Br_sum(y), self.Bc_sum(fc_parts)

    def solve_coupled(self, b_local, tol=1e-6, max_it=1000, warm=True, restart=20):
        """Coupled solve of Eqs. F1lr + F1uc by GMRES(restart) with the diagonal preconditioner.

        Returns (x_local list, lambda, x_c, iterations, relative residual estimate)."""
        m = self.maps
        d_r, f_c = self.rhs_parts(b_local)
        b = np.concatenate([d_r, f_c])
        x0 = np.concatenate([self.lam, self.xc]) if warm else np.zeros(len(b))
        dinv = np.concatenate([1.0 / self.diag, 1.0 / self.diag_c])
        it, res = 0, 0.0
        u = x0
        if len(b):
            u, it, res, _ = gmres(self.coupled_apply, b, x0, dinv, tol, restart, max_it)
        lam, x_c = u[:m.n_lambda].copy(), u[m.n_lambda:].copy()
        self.lam, self.xc = lam, x_c
        return self.recover(b_local, lam, x_c), lam, x_c, it, res

    # -- one solve ------------------------------------------------------------
    def solve(self, b_local, tol=1e-14, max_it=1000, warm=True, solver="cg", restart=20):
        """Solve the torn system for local right-hand sides b_local[s] (length n_s).

        solver "cg": Schur form (Eq. f1schur) with Jacobi CG; "gmres": coupled
        form (Eqs. F1lr + F1uc) with GMRES(restart).
        Returns (x_local list, lambda, x_c, iterations, final relative residual).
        """
        if solver == "gmres":
            return self.solve_coupled(b_local, tol, max_it, warm, restart)
        m = self.maps
        d_r, f_c = self.rhs_parts(b_local)
        rhs = d_r - (self.F_rc(self.Kcc_solve(f_c)) if m.n_corner else 0.0)
        lam = self.lam.copy() if warm else np.zeros(m.n_lambda)
        r = rhs - self.schur_apply(lam)
        nrm0 = np.linalg.norm(rhs)
        it = 0
        if nrm0 > 0 and np.linalg.norm(r) > tol * nrm0:
            z = r / self.diag
            p = z.copy()
            rz = r @ z
            while it < max_it:
                q = self.schur_apply(p)
                alpha = rz / (p @ q)
                lam += alpha * p
                r -= alpha * q
                it += 1
                if np.linalg.norm(r) <= tol * nrm0:
                    break
                z = r / self.diag
                rz_new = r @ z
                p = z + (rz_new / rz) * p
                rz = rz_new
        self.lam = lam
        x_c = self.Kcc_solve(f_c + self.F_rcT(lam)) if m.n_corner else np.zeros(0)
        self.xc = x_c
        x = self.recover(b_local, lam, x_c)
        res = np.linalg.norm(rhs - self.schur_apply(lam)) / nrm0 if nrm0 > 0 else 0.0
        return x, lam, x_c, it, res

    def gather_global(self, x_local):
        """Global field from the lowest-id subdomain owning each dof."""
        m = self.maps
        e = np.zeros(self.space.n)
        for s in range(m.n_sub - 1, -1, -1):      # lower ids overwrite higher ones
            e[m.local[s]] = x_local[s]
        return e

    def newmark_rhs(self, e_n, e_nm1, src_vec):
        """Local right-hand sides L^(s) = B^(s) e^n|_s - A^(s) e^{n-1}|_s - (source on owner)."""
        m = self.maps
        out = []
        for s in range(m.n_sub):
            loc = m.local[s]
            b = self.B[s] @ e_n[loc] - self.A[s] @ e_nm1[loc]
            own = m.owner[loc] == s
            b[own] -= src_vec[loc[own]]
            out.append(b)
        return out


def run(space, maps, dt, src, d2g, n_steps, tol=1e-14, P=None, keep=False, solver="cg", restart=20):
    """Newmark march with every step solved by the CPU MFETI-DP1 solver."""
    dd = DDSolver(space, maps, dt)
    e_nm1 = np.zeros(space.n)
    e_n = np.zeros(space.n)
    its, probes, fields = [], [], []
    for k in range(n_steps):
        b = dd.newmark_rhs(e_n, e_nm1, d2g[k] * src)
        x, lam, xc, it, res = dd.solve(b, tol=tol, solver=solver, restart=restart)
        e_np1 = dd.gather_global(x)
        e_nm1, e_n = e_n, e_np1
        its.append(it)
        if P is not None:
            probes.append(P @ e_n)
        if keep:
            fields.append(e_n.copy())
    out = dict(e_n=e_n, e_nm1=e_nm1, iters=np.array(its), solver=dd)
    if P is not None:
        out["probes"] = np.array(probes)
    if keep:
        out["fields"] = np.array(fields)
    return out


def interface_mass(space, maps, part):
    """Tangential Whitney mass M_T of the interface faces on the multiplier edges (sparse
    n_lambda x n_lambda).  An entry couples two multiplier edges of one interface face;
    both edges then join the same pair of subdomains, so M_T is block diagonal by pair."""
    from .fem import face_tangential_mass, interface_faces
    faces, _ = interface_faces(space.tets, part)
    n = int(space.tets.max()) + 1
    ekey = space.edges[:, 0] * n + space.edges[:, 1]
    def dof(a, b):
        return space.edge_to_dof[np.searchsorted(ekey, a * n + b)]
    fd = np.stack([dof(faces[:, 0], faces[:, 1]), dof(faces[:, 1], faces[:, 2]),
                   dof(faces[:, 0], faces[:, 2])], axis=1)                      # [F,3], -1 on the PEC wall
    midx = -np.ones(space.n, dtype=np.int64)
    midx[maps.mult_dof] = np.arange(maps.n_lambda)
    fm = np.where(fd >= 0, midx[np.maximum(fd, 0)], -1)
    Mf = face_tangential_mass(space.xyz[faces])
    r = np.broadcast_to(fm[:, :, None], Mf.shape)
    c = np.broadcast_to(fm[:, None, :], Mf.shape)
    ok = (r >= 0) & (c >= 0)
    M = sp.csr_matrix((Mf[ok], (r[ok], c[ok])), shape=(maps.n_lambda, maps.n_lambda))
    M.sum_duplicates()
    return M


class DP2Solver:
    """CPU MFETI-DP2 solve of A x = b (Sec. III-B), re-derived for the edge-only step system.

    Readings (the paper's DP2 is written for its mixed E/B system with face unknowns):
    * The Robin transmission condition Lambda = n x H - eta^-1 n x n x E becomes, in
      the Newmark step matrix A = T + dt^2/4 S, the interface term R^(s) = alpha M_T^(s)
      added to every local matrix on its interface (m = 2) edges, M_T the tangential
      Whitney mass of the interface faces; alpha = dt / (2 eta) with eta = 1 (the
      admittance term is a first time derivative; Newmark's gamma = 1/2 gives dt/2).
      Any alpha > 0 gives the monolithic solution at convergence.
    * One multiplier per interface edge and side: (A^(s) + R^(s)) x^(s) = b^(s) +
      lambda^(s) (unsigned, on the side's own interface edges), corners primal as in
      DP1.  Transmission (Eq. f2imp1): lambda^(1) + lambda^(2) = (R^(1) + R^(2)) x^(2)
      and = (R^(1) + R^(2)) x^(1), so that at convergence the traces agree and the
      interface rows of the subassembled system hold; R^(1) + R^(2) = 2 alpha M_T on
      the pair's edges.
    * Coupled system for u = [lambda^(s1); lambda^(s2); x_c] (s1 < s2 the multiplier's
      subdomains), solved by restarted GMRES with the diagonal preconditioner
      [1; 1; diag(K~cc)] (the lambda-lambda diagonal of the coupled matrix is 1).
    """

    def __init__(self, space, maps: DDMaps, dt, part, alpha=None):
        self.space, self.maps, self.dt = space, maps, float(dt)
        self.alpha = 0.5 * self.dt if alpha is None else float(alpha)
        self.M = interface_mass(space, maps, part)
        m = maps
        self.A, self.B, self.Ahat, self.chol = [], [], [], []
        self.Acc_tilde = np.zeros((m.n_corner, m.n_corner))
        Md = self.M.toarray() if m.n_lambda <= 20000 else None
        for s in range(m.n_sub):
            loc = m.local[s]
            dof_map = -np.ones(space.n, dtype=np.int64)
            dof_map[loc] = np.arange(len(loc))
            Ts, Ss = space.assemble(m.tets_of[s], dof_map, len(loc))
            As = (Ts + (dt * dt / 4.0) * Ss).toarray()
            self.A.append(As)
            self.B.append((2.0 * Ts - (dt * dt / 2.0) * Ss).toarray())
            # R^(s) = alpha M_T on the multipliers that involve s, at their local positions
            ks, ls = [], []
            for side in range(2):
                sel = np.flatnonzero(m.mult_sub[:, side] == s)
                ks.append(sel)
                ls.append(m.mult_loc[sel, side])
            k = np.concatenate(ks)
            l = np.concatenate(ls)
            Ah = As.copy()
            sub = Md[np.ix_(k, k)] if Md is not None else self.M[k][:, k].toarray()
            Ah[np.ix_(l, l)] += self.alpha * sub
            self.Ahat.append(Ah)
            nr = m.nr[s]
            cf = sla.cho_factor(Ah[:nr, :nr], lower=True)
            self.chol.append(cf)
            Arc = Ah[:nr, nr:]
            ci = m.corner_of_local[s]
            self.Acc_tilde[np.ix_(ci, ci)] += Ah[nr:, nr:] - Arc.T @ sla.cho_solve(cf, Arc)
        self.diag_c = np.diag(self.Acc_tilde).copy()
        self.u = np.zeros(2 * m.n_lambda + m.n_corner)

    # -- maps ----------------------------------------------------------------------
    def local_z(self, lam1, lam2, s):
        """lambda^(s) on the local r-vector of s (unsigned, the side's own multipliers)."""
        m = self.maps
        z = np.zeros(m.nr[s])
        sel = m.mult_sub[:, 0] == s
        z[m.mult_loc[sel, 0]] += lam1[sel]
        sel = m.mult_sub[:, 1] == s
        z[m.mult_loc[sel, 1]] += lam2[sel]
        return z

    def traces(self, xr):
        """(t1, t2): the interface values of the multiplier edges in s1 and in s2."""
        m = self.maps
        off = np.concatenate([[0], np.cumsum([len(v) for v in xr])])
        flat = np.concatenate(xr)
        return (flat[off[m.mult_sub[:, 0]] + m.mult_loc[:, 0]],
                flat[off[m.mult_sub[:, 1]] + m.mult_loc[:, 1]])

    def Bc_sum(self, xc):
        out = np.zeros(self.maps.n_corner)
        for s in range(self.maps.n_sub):
            np.add.at(out, self.maps.corner_of_local[s], xc[s])
        return out

    def split(self, u):
        nl = self.maps.n_lambda
        return u[:nl], u[nl:2 * nl], u[2 * nl:]

    # -- coupled operator (Eq. f2imp1 with Eq. F2un) ----------------------------------
    def coupled_apply(self, u):
        m = self.maps
        lam1, lam2, xc = self.split(u)
        xr, cpart = [], []
        for s in range(m.n_sub):
            nr = m.nr[s]
            z = self.local_z(lam1, lam2, s)
            x = sla.cho_solve(self.chol[s], z - self.Ahat[s][:nr, nr:] @ xc[m.corner_of_local[s]])
            xr.append(x)
            cpart.append(self.Ahat[s][nr:, :nr] @ sla.cho_solve(self.chol[s], z))
        t1, t2 = self.traces(xr)
        two_a_M = 2.0 * self.alpha * self.M
        y1 = lam1 + lam2 - two_a_M @ t2
        y2 = lam1 + lam2 - two_a_M @ t1
        yc = self.Acc_tilde @ xc + self.Bc_sum(cpart)      # lambda enters the local problems with +
        return np.concatenate([y1, y2, yc])

    def rhs(self, b_local):
        m = self.maps
        y0, fc = [], []
        for s in range(m.n_sub):
            nr = m.nr[s]
            y = sla.cho_solve(self.chol[s], b_local[s][:nr])
            y0.append(y)
            fc.append(b_local[s][nr:] - self.Ahat[s][nr:, :nr] @ y)
        t1, t2 = self.traces(y0)
        two_a_M = 2.0 * self.alpha * self.M
        return np.concatenate([two_a_M @ t2, two_a_M @ t1, self.Bc_sum(fc)]), y0

    def solve(self, b_local, tol=1e-12, max_it=2000, warm=True, restart=20):
        """Returns (x_local list, u = [lambda1; lambda2; x_c], iterations, residual estimate)."""
        m = self.maps
        b, y0 = self.rhs(b_local)
        dinv = np.concatenate([np.ones(2 * m.n_lambda), 1.0 / self.diag_c])
        x0 = self.u.copy() if warm else np.zeros(len(b))
        u, it, res = x0, 0, 0.0
        if len(b):
            u, it, res, _ = gmres(self.coupled_apply, b, x0, dinv, tol, restart, max_it)
        self.u = u.copy()
        lam1, lam2, xc = self.split(u)
        x = []
        for s in range(m.n_sub):
            nr = m.nr[s]
            xc_s = xc[m.corner_of_local[s]]
            z = self.local_z(lam1, lam2, s)
            xr = y0[s] + sla.cho_solve(self.chol[s], z - self.Ahat[s][:nr, nr:] @ xc_s)
            x.append(np.concatenate([xr, xc_s]))
        return x, u, it, res

    def gather_global(self, x_local):
        e = np.zeros(self.space.n)
        for s in range(self.maps.n_sub - 1, -1, -1):
            e[self.maps.local[s]] = x_local[s]
        return e

    def newmark_rhs(self, e_n, e_nm1, src_vec):
        """Subassembled L^(s) = B^(s) e^n - A^(s) e^{n-1} - (source on the owner), unmodified A."""
        m = self.maps
        out = []
        for s in range(m.n_sub):
            loc = m.local[s]
            b = self.B[s] @ e_n[loc] - self.A[s] @ e_nm1[loc]
            own = m.owner[loc] == s
            b[own] -= src_vec[loc[own]]
            out.append(b)
        return out


def run_dp2(space, maps, part, dt, src, d2g, n_steps, tol=1e-12, keep=False, restart=20, alpha=None):
    """Newmark march with every step solved by the CPU MFETI-DP2 solver."""
    dd = DP2Solver(space, maps, dt, part, alpha)
    e_nm1 = np.zeros(space.n)
    e_n = np.zeros(space.n)
    its, fields = [], []
    for k in range(n_steps):
        b = dd.newmark_rhs(e_n, e_nm1, d2g[k] * src)
        x, u, it, res = dd.solve(b, tol=tol, restart=restart)
        e_np1 = dd.gather_global(x)
        e_nm1, e_n = e_n, e_np1
        its.append(it)
        if keep:
            fields.append(e_n.copy())
    out = dict(e_n=e_n, iters=np.array(its), solver=dd)
    if keep:
        out["fields"] = np.array(fields)
    return out
