"""Gradients of a probe objective through the DD time march (torch.autograd).

J(eps, a) = weight * sum_{k=1..N} sum_p |E(r_p; e^k)|^2, where e^k is the Newmark
march of the edge-element wave equation driven by the source a * d2g_hat^k and
solved step by step by MFETI-DP1 on the GPU (dd_step).  The backward pass runs
the library's discrete adjoint (dd_adjoint_step: same factors, the seed
dJ/de^k from dd_probe_seed) and returns dJ/deps per tet and dJ/da.

Checkpointing: the forward pass keeps (e^k, e^{k-1}) every `checkpoint` steps;
the backward pass recomputes each segment's forward fields from its checkpoint
and sweeps the adjoint back through it, so device memory holds one segment.
Changing eps re-runs the host tearing and the factorisation (the permittivity
enters the mass matrix of every subdomain).
"""
from __future__ import annotations

import numpy as np
import torch

from . import dd as D


class ProbeObjective(torch.autograd.Function):
    @staticmethod
    def forward(ctx, eps, amp, problem, n_steps, checkpoint=100, params=None):
        """eps: [n_tets] float64 tensor (any device); amp: 0-dim float64 tensor.
        problem: dict(xyz, tets, part, n_sub, mu, probes, source_pairs, d2g (per-step unit second
        differences, >= n_steps), dt, weight=1.0)."""
        dev = torch.device("cuda")
        fs = D.FieldSolver(problem["xyz"], problem["tets"], problem["part"], problem["n_sub"],
                           eps=eps.detach().cpu().numpy(), mu=problem.get("mu", 1.0),
                           params=params or D.make_params(tol=1e-13), probes=problem["probes"]).bind()
        fs.factor(problem["dt"])
        n = fs.n_dof
        pattern = torch.zeros(n, dtype=torch.float64, device=dev)
        pattern[torch.as_tensor(fs.dof_of_pairs(problem["source_pairs"]), device=dev)] = 1.0
        d2g = np.asarray(problem["d2g"], dtype=np.float64)
        a = float(amp.detach().cpu())
        weight = float(problem.get("weight", 1.0))
        src = torch.empty(n, dtype=torch.float64, device=dev)
        J = torch.zeros((), dtype=torch.float64, device=dev)
        ckpt = {}
        for k in range(n_steps):
            if k % checkpoint == 0:
                e_n, e_nm1, _ = fs.get_state()
                ckpt[k] = (e_n, e_nm1)
            torch.mul(pattern, a * d2g[k], out=src)
            fs.step(src, stats=False)
            pv = fs.probe()
            J += weight * torch.dot(pv, pv)
        ctx.fs, ctx.ckpt, ctx.pattern = fs, ckpt, pattern
        ctx.d2g, ctx.a, ctx.weight = d2g, a, weight
        ctx.n_steps, ctx.checkpoint = n_steps, checkpoint
        ctx.eps_device = eps.device
        return J

    @staticmethod
    def backward(ctx, gJ):
        fs, n_steps, C = ctx.fs, ctx.n_steps, ctx.checkpoint
        dev = torch.device("cuda")
        n = fs.n_dof
        g = float(gJ.detach().cpu())
        grad_eps = torch.zeros(fs.n_tets, dtype=torch.float64, device=dev)
        grad_amp = torch.zeros(1, dtype=torch.float64, device=dev)
        seed = torch.empty(n, dtype=torch.float64, device=dev)
        src = torch.empty(n, dtype=torch.float64, device=dev)
        d2g_hat = torch.empty(n, dtype=torch.float64, device=dev)
        D.dd_adjoint_reset(fs.h)
        starts = sorted(ctx.ckpt)
        for s0 in reversed(starts):
            s1 = min(s0 + C, n_steps)
            e_n, e_nm1 = ctx.ckpt[s0]
            fs.set_state(e_n, e_nm1, s0)
            fields = {s0: e_n, s0 - 1: e_nm1}        # fields[k] = e^k
            for k in range(s0, s1):
                torch.mul(ctx.pattern, ctx.a * ctx.d2g[k], out=src)
                out = torch.empty(n, dtype=torch.float64, device=dev)
                fs.step(src, out, stats=False)
                fields[k + 1] = out
            for k in range(s1, s0, -1):
                D.dd_probe_seed(fs.h, fields[k], g * ctx.weight, seed)
                torch.mul(ctx.pattern, ctx.d2g[k - 1], out=d2g_hat)
                D.dd_adjoint_step(fs.h, seed, fields[k], fields[k - 1], fields[k - 2], d2g_hat, grad_eps, grad_amp,
                                  stats=False)
            del fields
        fs.close()
        ctx.fs = None
        return grad_eps.to(ctx.eps_device), grad_amp[0], None, None, None, None


def probe_objective(eps, amp, problem, n_steps, checkpoint=100, params=None):
    """J(eps, amp) with gradients through the GPU adjoint (see ProbeObjective)."""
    return ProbeObjective.apply(eps, amp, problem, n_steps, checkpoint, params)
