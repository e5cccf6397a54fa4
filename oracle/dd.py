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
