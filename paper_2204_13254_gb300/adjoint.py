"""Gradients of a probe objective through the DD time march (torch.autograd).

J(eps, a) = weight * sum_{k=1..N} sum_p |E(r_p; e^k)|^2, where e^k is the Newmark
march of the edge-element wave equation driven by the separable source
a * d2g_k * p (p: the tested current pattern of the source edges, d2g_k: the
second difference of the pulse's integrated current) and solved step by step by
MFETI-DP1 on the GPU.  Every operation on field data runs in the library:
dd_step_scaled advances the march with the source scaled on the device,
dd_probe_objective accumulates J in a device scalar, dd_probe_seed forms
dJ/de^k, and dd_adjoint_step_scaled runs one level of the discrete adjoint
(same factors) and accumulates dJ/deps per tet and dJ/da.  This module only
marshals pointers and host scalars.

Checkpointing: the forward pass keeps (e^k, e^{k-1}) every `checkpoint` steps;
the backward pass recomputes each segment's forward fields from its checkpoint
and sweeps the adjoint back through it, so device memory holds one segment.

A ProbeMarch keeps one handle (tearing, workspace) for a fixed mesh, partition,
dt and probe set; a new permittivity goes to the device (dd_set_eps) and is
followed by a refactorisation, so repeated evaluations (finite differences,
optimisation loops) reuse the handle.
"""
from __future__ import annotations

import numpy as np
import torch

from . import dd as D


class ProbeMarch:
    """One handle for repeated evaluations of J(eps, a) and its adjoint.

    problem: dict(xyz, tets, part, n_sub, mu, probes, source_pairs, d2g (per-step
    unit second differences), dt, weight=1.0)."""

    def __init__(self, problem, params=None, eps0=None):
        xyz, tets = problem["xyz"], problem["tets"]
        eps0 = np.ones(len(tets)) if eps0 is None else np.asarray(eps0, dtype=np.float64)
        self.fs = D.FieldSolver(xyz, tets, problem["part"], problem["n_sub"], eps=eps0, mu=problem.get("mu", 1.0),
                                params=params or D.make_params(tol=1e-13), probes=problem["probes"]).bind()
        self.dt = float(problem["dt"])
        self.d2g = np.asarray(problem["d2g"], dtype=np.float64)
        self.weight = float(problem.get("weight", 1.0))
        dev = torch.device("cuda")
        # the source's spatial pattern (input data: 1 on the source edges)
        self.pattern = torch.zeros(self.fs.n_dof, dtype=torch.float64, device=dev)
        self.pattern[torch.as_tensor(self.fs.dof_of_pairs(problem["source_pairs"]), device=dev)] = 1.0

    def set_eps(self, eps):
        """eps: [n_tets] float64 tensor (any device): new materials, then refactor."""
        e = eps.detach().to(device="cuda", dtype=torch.float64).contiguous()
        D.dd_set_eps(self.fs.h, e)
        self.fs.factor(self.dt)

    def close(self):
        if self.fs is not None:
            self.fs.close()
            self.fs = None


class ProbeObjective(torch.autograd.Function):
    @staticmethod
    def forward(ctx, eps, amp, problem, n_steps, checkpoint=100, params=None):
        """eps: [n_tets] float64 tensor (any device); amp: 0-dim float64 tensor.
        problem: a ProbeMarch (reused, left open) or its dict (a ProbeMarch is made
        for this evaluation and closed after the backward pass)."""
        own = not isinstance(problem, ProbeMarch)
        pm = ProbeMarch(problem, params) if own else problem
        pm.set_eps(eps)
        fs = pm.fs
        a = float(amp.detach().cpu())
        J = torch.zeros(1, dtype=torch.float64, device="cuda")
        ckpt = {}
        for k in range(n_steps):
            if k % checkpoint == 0:
                e_n, e_nm1, _ = fs.get_state()
                ckpt[k] = (e_n, e_nm1)
            D.dd_step_scaled(fs.h, pm.pattern, a * pm.d2g[k], stats=False)
            D.dd_probe_objective(fs.h, J, pm.weight)
        ctx.pm, ctx.own, ctx.ckpt, ctx.a = pm, own, ckpt, a
        ctx.n_steps, ctx.checkpoint = n_steps, checkpoint
        ctx.eps_device = eps.device
        if own and not (eps.requires_grad or amp.requires_grad):
            pm.close()
        return J[0]

    @staticmethod
    def backward(ctx, gJ):
        pm, n_steps, C = ctx.pm, ctx.n_steps, ctx.checkpoint
        fs = pm.fs
        dev = torch.device("cuda")
        n = fs.n_dof
        g = float(gJ.detach().cpu())
        grad_eps = torch.zeros(fs.n_tets, dtype=torch.float64, device=dev)
        grad_amp = torch.zeros(1, dtype=torch.float64, device=dev)
        seed = torch.empty(n, dtype=torch.float64, device=dev)
        D.dd_adjoint_reset(fs.h)
        starts = sorted(ctx.ckpt)
        for s0 in reversed(starts):
            s1 = min(s0 + C, n_steps)
            e_n, e_nm1 = ctx.ckpt[s0]
            fs.set_state(e_n, e_nm1, s0)
            fields = {s0: e_n, s0 - 1: e_nm1}        # fields[k] = e^k
            for k in range(s0, s1):
                out = torch.empty(n, dtype=torch.float64, device=dev)
                D.dd_step_scaled(fs.h, pm.pattern, ctx.a * pm.d2g[k], out, stats=False)
                fields[k + 1] = out
            for k in range(s1, s0, -1):
                D.dd_probe_seed(fs.h, fields[k], g * pm.weight, seed)
                D.dd_adjoint_step_scaled(fs.h, seed, fields[k], fields[k - 1], fields[k - 2], pm.pattern,
                                         pm.d2g[k - 1], grad_eps, grad_amp, stats=False)
            del fields
        if ctx.own:
            pm.close()
        ctx.pm = None
        return grad_eps.to(ctx.eps_device), grad_amp[0], None, None, None, None


def probe_objective(eps, amp, problem, n_steps, checkpoint=100, params=None):
    """J(eps, amp) with gradients through the GPU adjoint (see ProbeObjective).
    problem: a ProbeMarch (one handle reused across calls) or its dict."""
    return ProbeObjective.apply(eps, amp, problem, n_steps, checkpoint, params)
