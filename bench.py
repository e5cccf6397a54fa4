#!/usr/bin/env python
"""Benchmark of the MFETI-DP1 Maxwell field-solve time step on GB300.

One "step" is one implicit Newmark time step of the edge-element wave
equation solved by MFETI-DP1 (right-hand side SpMV, local solves, the
interface solve, recovery): every stage of the hot path.  The interface solve
is the coupled system of Eqs. F1lr + F1uc by GMRES(20) with the diagonal
preconditioner (the paper's Fig. fetiIter setting; --solver gmres, default)
or the Schur complement of Eq. f1schur by Jacobi CG (--solver cg); the line
also times the other solver and both at the paper's tolerance 1e-6.

Default workload: the mixed-precision configuration -- a PEC unit cube of
48^3 Kuhn cubes (663,552 tets, 753,552 interior edge unknowns) torn into
8x8x8 = 512 subdomains, Gaussian z-line pulse (t0 = 20 dt, sigma = 6 dt),
dt = 2x the explicit CFL limit.  Both precisions are timed on the same GPU:
the JSON line's `value` is the mixed-precision (FP32 application + FP64
refinement) rate, `fp64` holds the plain FP64 DD rate, and
`rel_err_mixed_vs_fp64` the relative L2 difference of the two fields after
the last step.  Inputs (14 GB of dense subdomain operators) are far larger
than L2, so no flush is needed between steps.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--config 1..5]

With --gpus N > 1 (launched by torchrun) every rank runs an independent
replica of the workload (the field solve uses one GPU; replicas only).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "DD field-solve steps/s, mixed vs FP64 at rel err 1e-8; % of HBM/tensor roofline"
FALLBACK_HBM_GBS = 6800.0
FP64_NOMINAL_TFLOPS = 1.25   # nominal GB300 FP64 rate (CUDA-core FMA)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--config", type=int, default=4)
    ap.add_argument("--tol64", type=float, default=1e-10, help="interface CG tolerance, FP64 DD")
    ap.add_argument("--tol32", type=float, default=1e-5, help="inner interface CG tolerance, mixed")
    ap.add_argument("--refine-tol", type=float, default=1e-10, help="FP64 step-residual target, mixed")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--only", choices=["fp64", "mixed"], default=None, help="time one precision only")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-profile", action="store_true", help="skip the per-stage event-profiled pass")
    ap.add_argument("--eager", action="store_true", help="time eager launches instead of the CUDA-graph step")
    ap.add_argument("--chunk", type=int, default=2, help="CG iterations per graph WHILE-body launch")
    ap.add_argument("--no-autotune", action="store_true", help="keep the default GEMV tiles")
    ap.add_argument("--tune-cache", default=None,
                    help="autotuner cache file: read when it holds this problem, else written after timing "
                         "(lets a profiled run reuse the tiles of an unprofiled one)")
    ap.add_argument("--warm", type=int, default=1, help="interface-CG warm start: 1 previous step, 2 extrapolated")
    ap.add_argument("--solver", choices=["cg", "gmres"], default="gmres",
                    help="interface solver of the headline runs: Schur CG (Eq. f1schur) or coupled GMRES(20)")
    ap.add_argument("--no-sym", action="store_true",
                    help="DD_MIXED GEMVs on the dense FP32 copy instead of the packed symmetric tiles")
    ap.add_argument("--ensemble", type=int, default=16,
                    help="members of the multi-RHS (ensemble) run beside the headline; 0 or 1 skips it")
    ap.add_argument("--ens-form", type=int, default=None, choices=[0, 1, 2, 3, 4],
                    help="pin the packed kernel form of the ensemble run's kinds instead of tuning them "
                         "(4: the tcgen05 form for the local solve, recovery and coupled operator)")
    ap.add_argument("--no-dp2", action="store_true",
                    help="skip the MFETI-DP2 runs (its own factorisation; coupled GMRES(20), FP64 at tol 1e-6 and mixed)")
    ap.add_argument("--no-other-configs", dest="other_configs", action="store_false",
                    help="skip the short runs of configs 3 (mixed/FP64), 5 (forward and adjoint) and 2 (PIC cycle)")
    ap.add_argument("--other-steps", type=int, default=10, help="timed steps of each other-config run")
    ap.add_argument("--no-sparse-study", dest="sparse_study", action="store_false",
                    help="skip the measured comparison with sparse local factors (cuSPARSE triangular solves)")
    ap.add_argument("--cpu-steps", type=int, default=3, help="oracle steps of the CPU baseline sample")
    ap.add_argument("--no-gmres", action="store_true",
                    help="skip the coupled-GMRES(20) vs Schur-CG comparison at the paper's tolerance 1e-6")
    ap.add_argument("--cavity", type=int, nargs=2, metavar=("N", "K"), default=None,
                    help="profiling case: unit PEC cavity of N^3 cubes in K^3 subdomains instead of --config "
                         "(dt = the 48^3 cavity's dt scaled by 48/N)")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def load_dt(cfg):
    table = json.load(open(os.path.join(ROOT, "tests", "golden", "cfl_dt.json")))
    return table[f"config{cfg}"]["dt"]


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        try:
            d = json.load(open(p))
            for k in ("hbm_gbs", "hbm_GBs", "hbm"):
                if k in d:
                    return float(d[k]), "measured", d
        except Exception:
            pass
    return FALLBACK_HBM_GBS, "fallback", {}


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during a timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except Exception:
            self.proc.kill()
            out, _ = self.proc.communicate()
        self.lines += [l for l in out.splitlines() if l.strip()]

    def summary(self):
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in self.lines:
            f = [x.strip() for x in l.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for name, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


# ----------------------------------------------------------------------------
# CPU baseline: the oracle's DD solver on a bounded sample of the workload
# ----------------------------------------------------------------------------

class OracleSample:
    """The CPU FP64 oracle's MFETI-DP1 march (scipy Cholesky per subdomain, Jacobi CG
    on Eq. f1schur, tol 1e-10) on a sample of the workload: a 2x2x2 block of
    subdomains of the workload's own subdomain size, mesh spacing and dt (PEC on
    the sample's walls, the z-line pulse through its centre).

    Why a sample: the oracle is a plain Python loop over subdomains with one
    single-right-hand-side triangular solve pair per subdomain and operator
    application; on the 48^3 cavity one of its steps takes minutes and its
    set-up (the Jacobi diagonal by one solve per multiplier) far longer, so it
    cannot run inside a benchmark.  Its cost per step is a sum over subdomains of
    identical work at the same interface iteration count (the Schur system's
    conditioning depends on the subdomain size H/h, which the sample keeps), so a
    full step is taken as the sample's measured step time times n_sub / 8.  The
    sample's factorisation is timed separately and is not part of the rate."""

    def __init__(self, cfg, dt):
        from oracle import dd as odd
        from oracle import fem
        from paper_2204_13254_gb300 import workloads as W
        wf = W.config(cfg)
        self.n_sub_full = wf.n_sub
        nx, ny, nz = wf.dims
        kx, ky, kz = {1: (2, 2, 2), 4: (8, 8, 8), 2: (4, 4, 8), 5: (8, 8, 4), 3: (4, 4, 4)}[cfg]
        bx, by, bz = nx // kx, ny // ky, nz // kz
        L = (2 * bx * wf.L[0] / nx, 2 * by * wf.L[1] / ny, 2 * bz * wf.L[2] / nz)
        self.w = W.box(2 * bx, 2 * by, 2 * bz, 2, 2, 2, L=L, steps=64)
        self.dt = dt
        t0 = time.perf_counter()
        space = fem.EdgeSpace(self.w.xyz, self.w.tets)
        self.maps = odd.DDMaps(space, self.w.part, self.w.n_sub)
        self.src = np.zeros(space.n)
        self.src[space.dof_of_pairs(self.w.source_pairs)] = 1.0
        self.t_setup = time.perf_counter() - t0
        t0 = time.perf_counter()
        self.dd = odd.DDSolver(space, self.maps, dt)
        self.t_factor = time.perf_counter() - t0
        self.d2g = self.w.d2G(dt, 64)
        self.space = space
        self.e_n = np.zeros(space.n)
        self.e_nm1 = np.zeros(space.n)
        self.k = 0
        self.iters = []
        self.desc = f"{2 * bx}x{2 * by}x{2 * bz}-cube sample, 2x2x2 subdomains of {bx}x{by}x{bz} cubes"

    def step(self):
        """One oracle time step of the sample (source steps 20.. so the pulse is on)."""
        b = self.dd.newmark_rhs(self.e_n, self.e_nm1, self.d2g[(20 + self.k) % 64] * self.src)
        x, lam, xc, it, res = self.dd.solve(b, tol=1e-10)
        e_np1 = self.dd.gather_global(x)
        self.e_nm1, self.e_n = self.e_n, e_np1
        self.iters.append(it)
        self.k += 1

    @property
    def scale(self):
        return self.n_sub_full / 8.0


def _threads():
    return int(os.environ.get("OMP_NUM_THREADS") or os.environ.get("OPENBLAS_NUM_THREADS") or os.cpu_count())


def cpu_baseline(cfg, dt, n_steps=3):
    """The oracle sample (OracleSample) for n_steps timed steps after one untimed
    warm-up step; the rate is scaled to the whole workload by subdomain count."""
    t0 = time.perf_counter()
    o = OracleSample(cfg, dt)
    o.step()
    t1 = time.perf_counter()
    for _ in range(n_steps):
        o.step()
    t_step = (time.perf_counter() - t1) / n_steps
    it = float(np.mean(o.iters[1:]))
    return {
        "value": 1.0 / (t_step * o.scale), "unit": "steps/s", "cores": _threads(), "kind": "oracle",
        "sample": (f"CPU FP64 oracle MFETI-DP1 (scipy Cholesky per subdomain, Jacobi CG on Eq. f1schur, tol 1e-10) "
                   f"on a {o.desc} (the workload's subdomain size, h and dt): {n_steps} steps measured after 1 "
                   f"warm-up, {t_step:.3f} s/step at {it:.1f} CG it/step; rate = 1 / (s/step x {o.scale:g} "
                   f"subdomain-count ratio); sample set-up {o.t_setup:.1f} s and factorisation "
                   f"{o.t_factor:.1f} s not in the rate"),
        "sample_s": time.perf_counter() - t0, "sample_step_s": t_step, "sample_iters_per_step": it,
        "os_cpu_count": os.cpu_count(),
    }


# ----------------------------------------------------------------------------
# GPU leg
# ----------------------------------------------------------------------------

def packed_kernel(tiles, stage, solver):
    """Name of the packed-tile kernel form the tuner chose for a stage's GEMV kind."""
    cfg = next((v for k, v in (tiles or {}).items() if k.startswith("packed")), {})
    kind = "local" if stage == "local_solve" else ("coupled" if solver == "gmres" else "iface_rows")
    ws = cfg.get(kind, (0, 0, 0, 0))[3]
    return {0: "k_symgemv<1>", 1: "k_symgemv_ws", 2: "k_symgemv<NR>", 3: "k_symgemv<2>"}.get(ws, "k_symgemv")


def _timed(fn, n, stream):
    """CUDA-event time (ms) of n calls of fn(i) on `stream`."""
    import torch
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    ev0.record(stream)
    for i in range(n):
        fn(i)
    ev1.record(stream)
    torch.cuda.synchronize()
    return ev0.elapsed_time(ev1)


def other_configs(args, dev):
    """Short timed runs of the other workloads (each: set-up, factorisation, tuning,
    warm-up, then --other-steps timed steps with CUDA events; the CUDA-graph step
    with the coupled GMRES(20), FP64 at tol 1e-10 and mixed at the headline's
    settings, no per-step readback):
      config 3 -- jittered 2x1x1 box, 300 RCB subdomains of uneven size;
      config 5 -- 32^3 cavity with eps ~ U[1,4]: forward steps, and the checkpointed
                  adjoint of the probe objective (100 forward steps, checkpoint 100:
                  the backward sweep recomputes the segment and runs 100 adjoint steps);
      config 2 -- the PIC cycle with the 1e5-particle beam (push, deposition, field
                  step, Faraday)."""
    import torch
    from paper_2204_13254_gb300 import adjoint as A
    from paper_2204_13254_gb300 import dd as D
    from paper_2204_13254_gb300 import workloads as W
    stream = torch.cuda.current_stream()
    K = args.other_steps
    Wu = 3
    out = {}

    def march(cfg, label_extra=None):
        w = W.config(cfg)
        dt = load_dt(cfg)
        t0 = time.perf_counter()
        pic = cfg == 2
        fs = D.FieldSolver(w.xyz, w.tets, w.part, w.n_sub, w.eps, w.mu, D.make_params(precision=D.DD_FP64),
                           probes=w.probes, device=dev)
        if pic:
            fs.set_beam(*W.beam(w, 100000, w.steps * dt, seed=0))
        fs.bind()
        t_setup = time.perf_counter() - t0
        t0 = time.perf_counter()
        fs.factor(dt)
        torch.cuda.synchronize()
        t_factor = time.perf_counter() - t0
        if not args.no_autotune:
            D.dd_autotune(fs.h, args.tune_cache)
        pat = torch.zeros(fs.n_dof, dtype=torch.float64, device=dev)
        pat[torch.as_tensor(fs.dof_of_pairs(w.source_pairs), device=dev)] = 1.0
        d2g = w.d2G(dt, Wu + K + 1)
        res = {"workload": w.name, "n_dof": int(fs.n_dof), "subdomains": int(w.n_sub), "setup_s": t_setup,
               "factor_s": t_factor}
        runs = [("fp64", D.make_params(precision=D.DD_FP64, tol=args.tol64, use_graph=1, chunk=args.chunk,
                                       solver=D.DD_SOLVER_COUPLED_GMRES)),
                ("mixed", D.make_params(precision=D.DD_MIXED, tol=args.tol32, refine_tol=args.refine_tol,
                                        max_refine=6, use_graph=1, chunk=args.chunk,
                                        solver=D.DD_SOLVER_COUPLED_GMRES))]
        fields = {}
        for name, prm in runs:
            fs.set_params(prm)
            if pic:
                fs.factor(dt)                 # restarts fields and particles
                step = lambda i, st=False: D.dd_pic_step(fs.h, st)
            else:
                zero = torch.zeros(fs.n_dof, dtype=torch.float64, device=dev)
                fs.set_state(zero, zero, 0)
                step = lambda i, st=False: D.dd_step_scaled(fs.h, pat, float(d2g[i]), stats=st)
            its = [step(i, True)["iters"] for i in range(Wu)]
            ms = _timed(lambda i: step(Wu + i), K, stream)
            # iteration counts from a readback pass over the next steps (not timed)
            its = [step(Wu + K + i, True)["iters"] for i in range(1)]
            e_last, _, _ = fs.get_state()
            fields[name] = e_last
            res[name] = {"steps_per_s": K * 1e3 / ms, "ms_per_step": ms / K, "iters_per_step": float(np.mean(its)),
                         "timed_steps": K}
        res["rel_err_mixed_vs_fp64"] = float(torch.linalg.norm(fields["mixed"] - fields["fp64"]) /
                                             torch.linalg.norm(fields["fp64"]))
        return fs, res, w, dt

    fs, res, _, _ = march(3)
    fs.close()
    out["config3"] = res
    fs, res, w5, dt5 = march(5)
    fs.close()
    # adjoint of the probe objective on config 5, FP64 CG at tol 1e-10, one handle
    n_adj = 100
    prob = dict(xyz=w5.xyz, tets=w5.tets, part=w5.part, n_sub=w5.n_sub, probes=w5.probes,
                source_pairs=w5.source_pairs, d2g=w5.d2G(dt5, n_adj), dt=dt5)
    pm = A.ProbeMarch(prob, params=D.make_params(precision=D.DD_FP64, tol=args.tol64, use_graph=1,
                                                 chunk=args.chunk, solver=D.DD_SOLVER_COUPLED_GMRES))
    eps = torch.tensor(w5.eps, dtype=torch.float64, device=dev, requires_grad=True)
    amp = torch.tensor(1.0, dtype=torch.float64, requires_grad=True)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    J = A.probe_objective(eps, amp, pm, n_adj, checkpoint=100)
    torch.cuda.synchronize()
    t_fwd = time.perf_counter() - t0
    t0 = time.perf_counter()
    J.backward()
    torch.cuda.synchronize()
    t_bwd = time.perf_counter() - t0
    pm.close()
    res["adjoint"] = {"steps": n_adj, "checkpoint": 100, "forward_s": t_fwd,
                      "backward_s": t_bwd, "adjoint_steps_per_s": n_adj / t_bwd,
                      "note": "wall clock (synchronised); the forward includes dd_set_eps and the refactorisation, "
                              "the backward recomputes the 100-step segment and runs 100 adjoint steps",
                      "dJ_da_over_2J": float(amp.grad) / (2.0 * float(J.detach()))}
    out["config5"] = res
    fs, res, _, _ = march(2)
    fs.close()
    out["config2_pic"] = res
    return out


def sparse_factor_study(cfg, dt, dev, reps=5):
    """Measured comparison for the choice of dense swept inverses over sparse local
    factors.  The sparse alternative: A_rr = L D L^T with a fill-reducing ordering
    (SuperLU, symmetric mode, minimum degree on A^T + A, no pivoting), applied by
    a forward and a backward triangular solve per local solve and per Arnoldi
    step (the coupled operator's F_rr and F_rc pieces need A_rr^-1 each time).
    The largest subdomain of the workload is factored on the host and replicated
    over all subdomains as one block-diagonal FP32 CSR matrix; the two
    triangular solves are timed on the GPU (cuSPARSE through torch, CUDA events),
    beside the bytes of the dense operators the library streams instead."""
    import scipy.sparse as sp
    import scipy.sparse.linalg as spla
    import torch
    from oracle import dd as odd
    from oracle import fem
    from paper_2204_13254_gb300 import workloads as W
    wf = W.config(cfg)
    nx, ny, nz = wf.dims
    kx, ky, kz = {1: (2, 2, 2), 4: (8, 8, 8), 2: (4, 4, 8), 5: (8, 8, 4), 3: (4, 4, 4)}[cfg]
    bx, by, bz = nx // kx, ny // ky, nz // kz
    L3 = (3 * bx * wf.L[0] / nx, 3 * by * wf.L[1] / ny, 3 * bz * wf.L[2] / nz)
    w = W.box(3 * bx, 3 * by, 3 * bz, 3, 3, 3, L=L3)     # the centre subdomain is an interior one
    space = fem.EdgeSpace(w.xyz, w.tets)
    maps = odd.DDMaps(space, w.part, w.n_sub)
    s = 13
    loc = maps.local[s]
    dof_map = -np.ones(space.n, dtype=np.int64)
    dof_map[loc] = np.arange(len(loc))
    Ts, Ss = space.assemble(maps.tets_of[s], dof_map, len(loc))
    nr, ns = int(maps.nr[s]), len(loc)
    nG = int(np.sum(maps.mult_sub[:, 0] == s) + np.sum(maps.mult_sub[:, 1] == s))
    A = (Ts + (dt * dt / 4.0) * Ss).tocsc()
    lu = spla.splu(A[:nr, :nr].tocsc(), permc_spec="MMD_AT_PLUS_A", diag_pivot_thresh=0.0,
                   options=dict(SymmetricMode=True))
    Lf = sp.tril(lu.L).tocsr().astype(np.float32)
    nnzL = int(Lf.nnz)
    nsub = wf.n_sub
    Lb = sp.block_diag([Lf] * nsub, format="csr")
    Lt = torch.sparse_csr_tensor(torch.tensor(Lb.indptr, dtype=torch.int32), torch.tensor(Lb.indices, dtype=torch.int32),
                                 torch.tensor(Lb.data), size=Lb.shape, device=dev)
    Ut = torch.sparse_csr_tensor(*(torch.tensor(a) for a in (lambda U: (U.indptr.astype(np.int32),
                                                                         U.indices.astype(np.int32), U.data))(
        Lb.T.tocsr())), size=Lb.shape, device=dev)
    b = torch.ones((Lb.shape[0], 1), dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()

    def solve():
        y = torch.triangular_solve(b, Lt, upper=False).solution
        return torch.triangular_solve(y, Ut, upper=True).solution

    solve()
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(reps):
        solve()
    ev1.record(stream)
    torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1) / reps
    nGc = ns - nr + nG   # [Gamma | c] of this subdomain
    return {
        "subdomain": f"interior subdomain of {bx}x{by}x{bz} cubes: {ns} local unknowns, {nr} in A_rr, "
                     f"{nG} interface + {ns - nr} corner",
        "nnz_L_minimum_degree": nnzL, "dense_triangle_A_rr^-1": nr * (nr + 1) // 2,
        "sparse_solve_pair_ms_all_subdomains": ms, "subdomains": nsub,
        "sparse_bytes_per_solve_pair_all_subdomains": 2.0 * nnzL * 8 * nsub,
        "dense_bytes_per_local_solve_all_subdomains (packed FP32)": nsub * 4.0 * (nr * (nr + 1) / 2 + (ns - nr) * nr),
        "dense_bytes_per_arnoldi_step_all_subdomains (packed FP32 [Gamma|c] block)": nsub * 4.0 * nGc * (nGc + 1) / 2,
        "note": ("a sparse factor needs one solve pair per local solve and per Arnoldi step (A_rr^-1 inside "
                 "F_rr and F_rc); the dense path reads the swept inverse for the local solve and only the "
                 "[Gamma|c] block per Arnoldi step"),
    }


def run_ours(args, rank, world, local):
    import torch
    from paper_2204_13254_gb300 import dd as D
    from paper_2204_13254_gb300 import workloads as W
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    cfg = args.config
    if args.cavity:
        w = W.cavity(args.cavity[0], args.cavity[1])
        dt = load_dt(4) * 48.0 / args.cavity[0]
    else:
        w = W.config(cfg)
        dt = load_dt(cfg)
    K, Wu = args.steps, args.warmup
    pic = cfg == 2 and not args.cavity      # config 2: the timed step is the whole PIC cycle
    t0 = time.perf_counter()
    fs = D.FieldSolver(w.xyz, w.tets, w.part, w.n_sub, w.eps, w.mu,
                       D.make_params(precision=D.DD_FP64, tol=args.tol64), device=dev)
    if pic:
        fs.set_beam(*W.beam(w, 100000, w.steps * dt, seed=0))
    fs.bind()
    t_setup = time.perf_counter() - t0
    sizes0 = fs.sizes
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    fs.factor(dt)
    torch.cuda.synchronize()
    t_factor = time.perf_counter() - t0
    t_tune, tiles = 0.0, None
    if not args.no_autotune:
        t_tune = D.dd_autotune(fs.h, args.tune_cache)
        tiles = D.dd_get_tiles(fs.h)
        tiles["packed_fp32 (CTAs per subdomain, ring depth, subdomains kept in L2, warp-specialised)"] = D.dd_get_sym_config(fs.h)
    n = fs.n_dof
    dofs = torch.tensor(fs.dof_of_pairs(w.source_pairs), device=dev)
    d2g = w.d2G(dt, Wu + K)
    D2G = torch.zeros((Wu + K, n), dtype=torch.float64, device=dev)
    for k in range(Wu + K):
        D2G[k, dofs] = float(d2g[k])
    zero = torch.zeros(n, dtype=torch.float64, device=dev)
    e_out = torch.empty(n, dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream()

    def barrier():
        if world > 1:
            torch.distributed.barrier()

    def one_step(k, stats):
        if pic:
            return fs.pic_step(stats=stats)
        return fs.step(D2G[k], stats=stats)

    def run_steps(params, profile, clocks=None, stats=True):
        """W warm-up steps, then K timed steps (CUDA events on the launch stream).
        stats=False: no per-step host readback (the CUDA-graph step runs without a
        round trip); iteration counts are then not collected."""
        fs.set_params(params)
        if pic:
            fs.factor(dt)                        # restarts fields and particles
        else:
            fs.set_state(zero, zero, 0)
        for k in range(Wu):
            one_step(k, True)
        barrier()
        torch.cuda.synchronize()
        fs.profile(enable=1, read=False)          # reset the launch counters
        if not profile:
            fs.profile(enable=0, read=False)      # count launches, record no events
        if clocks:
            clocks.start()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        its, refs = [], []
        for k in range(K):
            st = one_step(Wu + k, stats)
            if stats:
                its.append(st["iters"])
                refs.append(st["refinements"])
        ev1.record(stream)
        torch.cuda.synchronize()
        if clocks:
            clocks.stop()
        barrier()
        ms = ev0.elapsed_time(ev1)
        prof = fs.profile(enable=0, read=True)
        e_last, _, _ = fs.get_state()
        return ms, np.array(its), np.array(refs), prof, e_last.clone()

    clocks = Clocks(local)
    g = 0 if args.eager else 1
    ch = 8 if args.eager else args.chunk
    solver_of = {"cg": D.DD_SOLVER_SCHUR_CG, "gmres": D.DD_SOLVER_COUPLED_GMRES}
    sv = solver_of[args.solver]
    sym = 0 if args.no_sym else 1
    p64 = D.make_params(precision=D.DD_FP64, tol=args.tol64, use_graph=g, chunk=ch, warm_start=args.warm, solver=sv)
    p32 = D.make_params(precision=D.DD_MIXED, tol=args.tol32, refine_tol=args.refine_tol, max_refine=6, use_graph=g,
                        chunk=ch, warm_start=args.warm, solver=sv, sym_fp32=sym)
    # event profiling needs eager launches (events are recorded around every launch); one Krylov
    # iteration per host poll (chunk 1), so that no launch runs past convergence and exits at once
    # (those would count in a stage's time, not in its work)
    p64e = D.make_params(precision=D.DD_FP64, tol=args.tol64, warm_start=args.warm, solver=sv, chunk=1)
    p32e = D.make_params(precision=D.DD_MIXED, tol=args.tol32, refine_tol=args.refine_tol, max_refine=6,
                         warm_start=args.warm, solver=sv, sym_fp32=sym, chunk=1)
    nan = float("nan")
    ms64 = ms32 = nan
    it64 = it32 = ref32 = np.zeros(1)
    prof64 = prof32 = None
    e64 = e32 = None
    # headline timings: no event profiling inside the timed region
    # Each precision is timed twice over the same steps: with a stats readback per
    # step (iteration counts; a host round trip between steps) and without (the
    # graph step's own mode).  The rate without readback is the headline; the
    # two passes must give bitwise equal fields.
    ms64s = ms32s = nan
    same64 = same32 = None
    if args.only in (None, "fp64"):
        # launch counts come from the readback pass (graph launches are counted from the
        # iteration counts it reads); the pass without readback runs the same kernels
        ms64s, it64, _, prof64, e64s = run_steps(p64, False)
        ms64, _, _, _, e64 = run_steps(p64, False, clocks, stats=False)
        same64 = bool(torch.equal(e64, e64s))
    if args.only in (None, "mixed"):
        ms32s, it32, ref32, prof32, e32s = run_steps(p32, False)
        ms32, _, _, _, e32 = run_steps(p32, False, clocks, stats=False)
        same32 = bool(torch.equal(e32, e32s))
    rel = float(torch.linalg.norm(e32 - e64) / torch.linalg.norm(e64)) if e32 is not None and e64 is not None else nan
    # the paper's coupled solve (Eqs. F1lr + F1uc, GMRES(20), tol 1e-6, diagonal preconditioner)
    # beside the Schur CG at the same tolerance, both FP64, same launch mode
    gm = None
    if not args.no_gmres and not pic:
        tol_p = 1e-6
        pg = D.make_params(precision=D.DD_FP64, tol=tol_p, use_graph=g, chunk=ch, solver=D.DD_SOLVER_COUPLED_GMRES,
                           restart=20)
        pc = D.make_params(precision=D.DD_FP64, tol=tol_p, use_graph=g, chunk=ch)
        msg, itg, _, profg, eg = run_steps(pg, False)
        msc, itc, _, _, ec = run_steps(pc, False)
        gm = {"tol": tol_p, "restart": 20,
              "gmres": {"steps_per_s": K * 1e3 / msg, "ms_per_step": msg / K, "iters_per_step": float(np.mean(itg)),
                        "gpu_launches": int(profg["total_launches"])},
              "schur_cg": {"steps_per_s": K * 1e3 / msc, "ms_per_step": msc / K, "iters_per_step": float(np.mean(itc))},
              "rel_diff_fields": float(torch.linalg.norm(eg - ec) / torch.linalg.norm(ec))}
        # the other solver at the headline's mixed-precision settings
        other = "gmres" if args.solver == "cg" else "cg"
        po = D.make_params(precision=D.DD_MIXED, tol=args.tol32, refine_tol=args.refine_tol, max_refine=6,
                           use_graph=g, chunk=ch, warm_start=1, solver=solver_of[other], sym_fp32=sym)
        mso, ito, refo, profo, eo = run_steps(po, False)
        gm[f"mixed_{other}"] = {"steps_per_s": K * 1e3 / mso, "ms_per_step": mso / K,
                                "iters_per_step": float(np.mean(ito)), "refinements_per_step": float(np.mean(refo)),
                                "gpu_launches": int(profo["total_launches"]),
                                "rel_err_vs_fp64": (float(torch.linalg.norm(eo - e64) / torch.linalg.norm(e64))
                                                    if e64 is not None else None)}
    # per-stage breakdown: a second pass over the same steps with CUDA events around every launch
    launches64 = prof64["total_launches"] if prof64 else None
    launches32 = prof32["total_launches"] if prof32 else None
    if not args.no_profile:
        if args.only in (None, "fp64"):
            prof64 = run_steps(p64e, True)[3]
        if args.only in (None, "mixed"):
            prof32 = run_steps(p32e, True)[3]

    # end-to-end: per step, H2D of the source from pinned host memory, the C-ABI step, D2H of e^{n+1}
    ms_e2e = nan
    if not args.no_e2e and not pic:
        host_src = torch.zeros((K, n), dtype=torch.float64).pin_memory()
        host_src.copy_(D2G[Wu:].cpu())
        host_e = torch.empty(n, dtype=torch.float64).pin_memory()
        dsrc = torch.empty(n, dtype=torch.float64, device=dev)
        fs.set_params(p32 if args.only != "fp64" else p64)
        fs.set_state(zero, zero, 0)
        for k in range(Wu):
            fs.step(D2G[k], stats=False)
        barrier()
        torch.cuda.synchronize()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        for k in range(K):
            dsrc.copy_(host_src[k], non_blocking=True)
            fs.step(dsrc, e_out, stats=False)
            host_e.copy_(e_out, non_blocking=True)
        ev1.record(stream)
        torch.cuda.synchronize()
        barrier()
        ms_e2e = ev0.elapsed_time(ev1)

    # the factorisation with its trailing updates on the tensor cores (BF16 slices, FP64-accurate)
    # against the FP64 CUDA-core path: time, and the coupled operator of both factorisations
    tcf = None
    if not pic and world == 1:
        nu = int(fs.sizes.n_lambda + fs.sizes.n_corner)
        u = torch.randn(nu, dtype=torch.float64, device=dev, generator=torch.Generator(device=dev).manual_seed(5))
        pf = D.make_params(precision=D.DD_FP64, tol=args.tol64, solver=D.DD_SOLVER_COUPLED_GMRES,
                           factor_mode=D.DD_FACTOR_FP64)
        fs.set_params(pf)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        fs.factor(dt)
        torch.cuda.synchronize()
        t_f64 = time.perf_counter() - t0
        ref_apply = fs.coupled_apply(u)
        fs.set_params(D.make_params(precision=D.DD_FP64, tol=args.tol64, solver=D.DD_SOLVER_COUPLED_GMRES,
                                    factor_mode=D.DD_FACTOR_TENSOR))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        fs.factor(dt)
        torch.cuda.synchronize()
        t_tc = time.perf_counter() - t0
        got_apply = fs.coupled_apply(u)
        tcf = {"factor_s_fp64_cuda_cores": t_f64, "factor_s_tensor_cores": t_tc,
               "speedup": t_f64 / t_tc,
               "coupled_operator_rel_diff": float(torch.linalg.norm(got_apply - ref_apply) / torch.linalg.norm(ref_apply)),
               "method": "trailing updates from 7 x 7 BF16 slices (8 bits each, power-of-two row/column scaling), "
                         "weight classes summed exactly in FP32 tensor memory by tcgen05 MMAs, combined in FP64"}
        # (the runs below refactor with their own settings)

    # MFETI-DP2 (Sec. III-B): refactor with the Robin term, FP64 at the paper's tolerance and
    # the headline's mixed settings; last, so that the runs above keep the DP1 factorisation
    dp2 = None
    if not args.no_dp2 and not pic:
        pd = D.make_params(precision=D.DD_FP64, tol=1e-6, use_graph=g, chunk=ch,
                           solver=D.DD_SOLVER_COUPLED_GMRES, scheme=D.DD_SCHEME_DP2, restart=20)
        fs.set_params(pd)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        fs.factor(dt)
        torch.cuda.synchronize()
        t_f2 = time.perf_counter() - t0
        msd, itd, _, _, ed = run_steps(pd, False)
        pm = D.make_params(precision=D.DD_MIXED, tol=args.tol32, refine_tol=args.refine_tol, max_refine=6,
                           use_graph=g, chunk=ch, solver=D.DD_SOLVER_COUPLED_GMRES, scheme=D.DD_SCHEME_DP2,
                           restart=20, sym_fp32=sym)
        msm, itm, refm, _, em = run_steps(pm, False)
        dp2 = {"factor_s": t_f2,
               "fp64_tol_1e-6": {"steps_per_s": K * 1e3 / msd, "ms_per_step": msd / K,
                                 "iters_per_step": float(np.mean(itd))},
               "mixed": {"steps_per_s": K * 1e3 / msm, "ms_per_step": msm / K, "iters_per_step": float(np.mean(itm)),
                         "refinements_per_step": float(np.mean(refm)),
                         "rel_err_vs_fp64_dp1": (float(torch.linalg.norm(em - e64) / torch.linalg.norm(e64))
                                                 if e64 is not None else None)}}

    # multi-RHS batching: R members (the headline source at amplitudes 1, -1/2, 2, 1/4, ...) marched
    # together with one copy of the factored operators, headline mixed settings, coupled GMRES
    ens = None
    if args.ensemble > 1 and not pic:
        R = args.ensemble
        pe = D.make_params(precision=D.DD_MIXED, tol=args.tol32, refine_tol=args.refine_tol, max_refine=6,
                           use_graph=g, chunk=ch, solver=D.DD_SOLVER_COUPLED_GMRES, sym_fp32=sym, members=R)
        t0 = time.perf_counter()
        fe = D.FieldSolver(w.xyz, w.tets, w.part, w.n_sub, w.eps, w.mu, pe, device=dev).bind()
        t_se = time.perf_counter() - t0
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        fe.factor(dt)
        torch.cuda.synchronize()
        t_fe = time.perf_counter() - t0
        if not args.no_autotune:
            D.dd_autotune(fe.h, args.tune_cache)
        if args.ens_form is not None:
            for kind in ("local", "recover", "coupled"):
                D.dd_set_sym_config(fe.h, kind, 1, 2, 0, args.ens_form)
        ens_forms = D.dd_get_sym_config(fe.h)
        amps = [[1.0, -0.5, 2.0, 0.25][r % 4] * (1 + r // 4) for r in range(R)]
        ne = fe.n_dof
        De = torch.zeros((Wu + K, ne), dtype=torch.float64, device=dev)
        for r in range(R):
            de = torch.tensor(fe.dof_of_pairs(w.source_pairs, member=r), device=dev)
            for k in range(Wu + K):
                De[k, de] = amps[r] * float(d2g[k])
        for k in range(Wu):
            fe.step(De[k], stats=True)
        barrier()
        torch.cuda.synchronize()
        fe.profile(enable=1, read=False)
        fe.profile(enable=0, read=False)
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        ite, rfe = [], []
        for k in range(K):
            st = fe.step(De[Wu + k], stats=True)
            ite.append(st["iters"])
            rfe.append(st["refinements"])
        ev1.record(stream)
        torch.cuda.synchronize()
        barrier()
        mse = ev0.elapsed_time(ev1)
        pe_prof = fe.profile(enable=0, read=True)
        ee, _, _ = fe.get_state()
        ee = ee.view(R, -1)
        ens_stages = None
        if not args.no_profile:   # per-stage split: an eager pass over a few steps with events per launch
            fe.set_params(D.make_params(precision=D.DD_MIXED, tol=args.tol32, refine_tol=args.refine_tol,
                                        max_refine=6, solver=D.DD_SOLVER_COUPLED_GMRES, sym_fp32=sym, members=R))
            fe.profile(enable=1, read=False)
            ks = min(K, 4)
            for k in range(ks):
                fe.step(De[Wu + k], stats=True)
            ens_stages = stage_table(fe.profile(enable=0, read=True), ks)
        ens = {"members": R, "amplitudes": amps, "member_steps_per_s": R * K * 1e3 / mse, "ms_per_step": mse / K,
               "iters_per_step": float(np.mean(ite)), "refinements_per_step": float(np.mean(rfe)),
               "gpu_launches": int(pe_prof["total_launches"]), "setup_s": t_se, "factor_s": t_fe,
               "operator_bytes_fp64": int(fe.sizes.dense_bytes_fp64),
               "packed_forms (CTAs per subdomain, ring depth, subdomains kept in L2, form: 4 = tcgen05 BF16x3 MMA "
               "over 16 members)": ens_forms,
               "rel_err_member0_vs_single_mixed": (float(torch.linalg.norm(ee[0] - e32) / torch.linalg.norm(e32))
                                                   if e32 is not None and args.solver == "gmres" else None),
               "stages (eager pass, CUDA events per launch)": ens_stages}
        fe.close()
        del De

    def allmax(x):
        if world == 1:
            return x
        t = torch.tensor([x], dtype=torch.float64, device=dev)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        return float(t.item())

    sparse = None
    if args.sparse_study and not args.cavity and not pic and world == 1:
        try:
            sparse = sparse_factor_study(cfg, dt, dev)
        except Exception as ex:   # context only: never fail the GPU line on it
            sparse = {"error": repr(ex)[:300]}
    # bytes of one launch of each packed / dense GEMV kind, algorithmic and streamed
    gemv_bytes = {p_name: {kind: D.dd_get_gemv_bytes(fs.h, kind, prec) for kind in ("local", "iface_rows", "coupled",
                                                                                     "recover")}
                  for p_name, prec in (("fp64", D.DD_FP64), ("mixed", D.DD_MIXED))}
    fs.set_params(p32)
    gemv_bytes["mixed"] = {kind: D.dd_get_gemv_bytes(fs.h, kind, D.DD_MIXED)
                           for kind in ("local", "iface_rows", "coupled", "recover")}
    fp64_tflops = D.dd_measure_fp64_rate()
    others = None
    if args.other_configs and not args.cavity and cfg == 4 and world == 1:
        fs.close()
        fs = None
        torch.cuda.empty_cache()
        others = other_configs(args, dev)

    ms64, ms32, ms_e2e = allmax(ms64), allmax(ms32), allmax(ms_e2e)
    ms64s, ms32s = allmax(ms64s), allmax(ms32s)
    sizes = dict(n_dof=int(sizes0.n_dof), n_lambda=int(sizes0.n_lambda), n_corner=int(sizes0.n_corner),
                 dense_bytes_fp64=int(sizes0.dense_bytes_fp64))
    res = dict(fs=fs, K=K, ms64=ms64, ms32=ms32, ms64s=ms64s, ms32s=ms32s, same64=same64, same32=same32,
               gemv_bytes=gemv_bytes, fp64_tflops=fp64_tflops, others=others, sparse=sparse, tcf=tcf,
               ms_e2e=ms_e2e, it64=it64, it32=it32, ref32=ref32, prof64=prof64,
               prof32=prof32, rel=rel, launches64=launches64, launches32=launches32, t_setup=t_setup, t_factor=t_factor, clocks=clocks.summary(), sizes=sizes,
               workload=w, dt=dt, t_tune=t_tune, tiles=tiles, pic=pic, gmres=gm, dp2=dp2, ens=ens)
    return res


def aggregate_replicas(ms_local, steps, world, reduce_max):
    """Whole-job rate of `world` independent replicas: every rank timed `steps`
    steps in ms_local; the job takes the slowest rank's time (max over ranks)."""
    ms = reduce_max(ms_local)
    return ms, world * steps / (ms / 1e3)


def stage_table(prof, K):
    out = {}
    if not prof:
        return out
    for name, st in prof["stages"].items():
        if st["launches"] == 0:
            continue
        gbs = st["bytes"] / (st["ms"] * 1e6) if st["ms"] > 0 else None
        out[name] = {"ms_per_step": st["ms"] / K, "launches_per_step": st["launches"] / K,
                     "full_launches_per_step": st["work"] / K, "algorithmic_GB_per_step": st["bytes"] / K / 1e9,
                     "achieved_GBs": gbs}
    return out


def _fp64_roofline(st64, fp64_tflops):
    """FP64 path: the dominant GEMV is FP64-ALU bound on GB300 (2 flops per 8-byte
    matrix element), against the FP64 FMA rate measured in the same run."""
    cand = {k: v for k, v in st64.items() if k not in ("vector", "factor") and v.get("achieved_GBs")}
    if not cand:
        return None
    dom = max(cand, key=lambda k: cand[k]["ms_per_step"])
    gflops = cand[dom]["achieved_GBs"] / 8.0 * 2.0
    peak = fp64_tflops * 1e3 if fp64_tflops else FP64_NOMINAL_TFLOPS * 1e3
    return {"bound": "alu", "kernel": f"k_gemv<double> ({dom})", "achieved": gflops, "peak": peak,
            "unit": "GFLOP/s", "frac": gflops / peak,
            "peak_source": ("measured in this run: dd_measure_fp64_rate (FMA chains on every SM, CUDA events)"
                            if fp64_tflops else "nominal GB300 FP64 rate (1.25 TFLOP/s)")}


def _clean(x):
    """JSON-safe copy: NaN/inf -> None."""
    if isinstance(x, dict):
        return {k: _clean(v) for k, v in x.items()}
    if isinstance(x, (list, tuple)):
        return [_clean(v) for v in x]
    if isinstance(x, float) and not np.isfinite(x):
        return None
    if isinstance(x, (np.floating,)):
        return _clean(float(x))
    if isinstance(x, (np.integer,)):
        return int(x)
    return x


def main():
    args = parse()
    rank, world, local = dist_env()
    if world > 1:
        import torch
        import torch.distributed as dist
        backend = "nccl" if args.impl == "ours" else "gloo"
        if args.impl == "ours":
            torch.cuda.set_device(local)
        dist.init_process_group(backend)
    if args.impl == "reference":
        if rank == 0:
            dt = load_dt(args.config)
            from paper_2204_13254_gb300 import workloads as W
            # the oracle sample: W untimed steps, then K timed steps, each one oracle step
            # of the sample, reported per full-workload step (x n_sub / 8)
            t0 = time.perf_counter()
            o = OracleSample(args.config, dt)
            for _ in range(args.warmup):
                o.step()
            t1 = time.perf_counter()
            for _ in range(args.steps):
                o.step()
            t_step = (time.perf_counter() - t1) / max(1, args.steps)
            it = float(np.mean(o.iters[args.warmup:])) if args.steps else 0.0
            val = 1.0 / (t_step * o.scale)
            cb = {"value": val, "unit": "steps/s", "cores": _threads(), "kind": "oracle",
                  "sample": (f"each step: one step of the CPU FP64 oracle MFETI-DP1 on a {o.desc} (the "
                             f"workload's subdomain size, h and dt), {t_step:.3f} s at {it:.1f} CG it/step, "
                             f"reported per full step (x {o.scale:g} subdomains); set-up {o.t_setup:.1f} s and "
                             f"factorisation {o.t_factor:.1f} s untimed"),
                  "sample_s": time.perf_counter() - t0, "os_cpu_count": os.cpu_count()}
            line = {"metric": METRIC, "impl": "reference", "value": val, "unit": "steps/s", "n_gpus": 0,
                    "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_step * 1e3,
                    "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
                    "data": "synthetic", "config": {"workload": W.config(args.config).name},
                    "cpu_baseline": cb,
                    "e2e": {"value": cb["value"], "unit": "steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
            print(json.dumps(line), flush=True)
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()
        return

    r = run_ours(args, rank, world, local)
    if rank != 0:
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()
        return
    K = r["K"]
    peak, peak_kind, peaks = load_peaks()
    st32 = stage_table(r["prof32"], K)
    st64 = stage_table(r["prof64"], K)
    head = "mixed" if args.only != "fp64" else "fp64"
    st_head = st32 if head == "mixed" else st64
    cand = {k: v for k, v in st_head.items() if k not in ("vector", "factor")}
    dom = max(cand, key=lambda k: cand[k]["ms_per_step"]) if cand else None
    achieved = cand[dom]["achieved_GBs"] if dom else None
    kind_of_stage = {"local_solve": "local", "iface_apply": "coupled" if args.solver == "gmres" else "iface_rows",
                     "recover": "recover"}
    gb_head = r["gemv_bytes"].get(head, {}).get(kind_of_stage.get(dom)) if dom else None
    sizes = r["sizes"]
    w = r["workload"]
    ms_head = r["ms32"] if head == "mixed" else r["ms64"]       # the pass without per-step readback
    same = lambda x: x          # times were already max-reduced over ranks in run_ours
    value = aggregate_replicas(ms_head, K, world, same)[1]
    v64 = aggregate_replicas(r["ms64"], K, world, same)[1]
    v32 = aggregate_replicas(r["ms32"], K, world, same)[1]
    cb = None
    if world == 1 and not args.no_cpu_baseline and not args.cavity and not r["pic"]:
        try:
            cb = cpu_baseline(args.config, r["dt"], args.cpu_steps)
        except Exception as ex:  # the baseline is context only; never fail the GPU line on it
            cb = {"error": repr(ex)[:200]}
    traffic = None
    tpath = os.path.join(ROOT, "profiles", "traffic.json")
    if os.path.exists(tpath) and dom:
        try:
            tj = json.load(open(tpath))
            traffic = tj.get(f"config{args.config}", {}).get(f"{head}:{dom}")
        except Exception:
            traffic = None
    prof_head = r["prof32"] if head == "mixed" else r["prof64"]
    line = {
        "metric": METRIC, "value": value, "unit": "steps/s", "n_gpus": world, "steps": K, "warmup": args.warmup,
        "ms_per_step": ms_head / K, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32+f64" if head == "mixed" else "f64", "data": "synthetic",
        "config": {"workload": w.name,
                   "mesh": ("PIC cycle (1e5-particle beam push + Whitney deposition + DD field solve + Faraday), "
                            if r["pic"] else "") + (f"PEC box {w.dims[0]}x{w.dims[1]}x{w.dims[2]} Kuhn cubes, {len(w.tets)} tets, "
                            f"{sizes['n_dof']} edge dofs, {w.n_sub} subdomains, {sizes['n_lambda']} multipliers, "
                            f"{sizes['n_corner']} corners, Gaussian z-line pulse, dt=2xCFL={r['dt']:.6g}"),
                   "l2_policy": "inputs larger than L2 (dense subdomain operators "
                                f"{sizes['dense_bytes_fp64'] / 1e9:.1f} GB FP64 + half that FP32), no flush",
                   "parallelism": f"replicas x{world}" if world > 1 else "1 GPU",
                   "stage_profile": ("separate eager pass over the same steps with CUDA events per launch, one Krylov "
                                     "iteration per host poll (no launch past convergence)")},
        "mixed": {"steps_per_s": v32, "ms_per_step": r["ms32"] / K, "iters_per_step": float(np.mean(r["it32"])),
                  "refinements_per_step": float(np.mean(r["ref32"])), "inner_tol": args.tol32,
                  "refine_tol": args.refine_tol,
                  "with_stats_readback": {"steps_per_s": K * 1e3 / r["ms32s"], "ms_per_step": r["ms32s"] / K,
                                          "fields_bitwise_equal": r["same32"]},
                  "stages": st32},
        "fp64": {"steps_per_s": v64, "ms_per_step": r["ms64"] / K, "iters_per_step": float(np.mean(r["it64"])),
                 "tol": args.tol64,
                 "with_stats_readback": {"steps_per_s": K * 1e3 / r["ms64s"], "ms_per_step": r["ms64s"] / K,
                                         "fields_bitwise_equal": r["same64"]},
                 "stages": st64},
        "timing": ("value and fp64/mixed steps_per_s: CUDA-graph steps without per-step host readback; "
                   "with_stats_readback: the same steps reading iteration counts back after every step"),
        "other_configs": r["others"],
        "sparse_factor_study": r["sparse"],
        "factor_tensor_cores": r["tcf"],
        "speedup_mixed_vs_fp64": v32 / v64,
        "coupled_gmres_vs_schur_cg": r["gmres"],
        "mfeti_dp2": r["dp2"],
        "ensemble": (dict(r["ens"], member_steps_vs_single=r["ens"]["member_steps_per_s"] / v32)
                     if r["ens"] else None),
        "rel_err_mixed_vs_fp64": r["rel"],
        "setup_s": r["t_setup"], "factor_s": r["t_factor"], "autotune_s": r["t_tune"],
        "gemv_tiles": r["tiles"],
        "fp64_roofline": _fp64_roofline(st64, r["fp64_tflops"]),
        "fp64_fma_tflops_measured": r["fp64_tflops"],
        "roofline": {"bound": "hbm", "kernel": (f"{packed_kernel(r['tiles'], dom, args.solver)} (packed FP32 tiles, {dom})"
                                                if head == "mixed" and not args.no_sym and dom in ("local_solve", "iface_apply")
                                                else f"k_gemv<{'float' if head == 'mixed' else 'double'}> ({dom})"),
                     "achieved": achieved, "peak": peak,
                     "unit": "GB/s", "frac": (achieved / peak) if achieved else None, "traffic": traffic,
                     "bytes": ("algorithmic: the distinct elements of the symmetric operator the product needs "
                               "(FP32) plus vectors, from the library's per-launch count (dd_get_gemv_bytes); "
                               "traffic: ncu DRAM bytes per launch of the same kernel (profiles/)"),
                     "algorithmic_bytes_per_launch": gb_head[0] if gb_head else None,
                     "streamed_tile_bytes_per_launch": gb_head[1] if gb_head else None,
                     "peak_source": f"{peak_kind} hbm_gbs" + ("" if peak_kind == "measured" else " (no MEASURED_PEAKS.json)")},
        "gemv_bytes_per_launch": {p_: {k_: {"algorithmic": v_[0], "streamed": v_[1]} for k_, v_ in d_.items()}
                                  for p_, d_ in r["gemv_bytes"].items()},
        "cpu_baseline": cb,
        "e2e": {"value": aggregate_replicas(r["ms_e2e"], K, world, same)[1], "unit": "steps/s",
                "h2d_bytes_per_step": int(sizes["n_dof"] * 8), "d2h_bytes_per_step": int(sizes["n_dof"] * 8)},
        "gpu_launches": int(r["launches32"] if head == "mixed" else r["launches64"]),
        "launch_mode": "eager" if args.eager else f"CUDA graph per step (Krylov loop as WHILE node, {args.chunk} it/body)",
        "fp32_storage": "dense" if args.no_sym else "packed symmetric 64x64 tiles (local solve, interface rows, coupled operator; the recovery too for ensembles)",
        "interface_solver": {"cg": "Schur complement (Eq. f1schur), Jacobi CG",
                             "gmres": "coupled Eqs. F1lr + F1uc, GMRES(20), diagonal preconditioner"}[args.solver],
        "warm_start": {1: "previous step's multipliers", 2: "extrapolated multipliers 2l(n-1)-l(n-2)"}.get(args.warm, args.warm),
        "clocks": r["clocks"],
    }
    print(json.dumps(_clean(line)), flush=True)
    if r["fs"] is not None:
        r["fs"].close()
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
