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
    ap.add_argument("--ensemble", type=int, default=4,
                    help="members of the multi-RHS (ensemble) run beside the headline; 0 or 1 skips it")
    ap.add_argument("--no-dp2", action="store_true",
                    help="skip the MFETI-DP2 runs (its own factorisation; coupled GMRES(20), FP64 at tol 1e-6 and mixed)")
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

def cpu_baseline(cfg, dt, full_iters, n_sub_full, n_steps=6):
    """Times the CPU FP64 oracle (scipy/numpy, host cores) on a sample of the
    workload: a 2x2x2 block of subdomains cut from the same mesh (same h, same
    6^3-cube subdomain blocks, same dt), PEC on the sample's walls.  The per-step
    time is scaled to the full workload by the subdomain count and by the number
    of local solves per step (2 + 3 per interface iteration, oracle algorithm),
    using the GPU-measured iterations of the full workload."""
    from oracle import dd as odd
    from oracle import fem
    from paper_2204_13254_gb300 import workloads as W
    wf = W.config(cfg)
    nx, ny, nz = wf.dims
    kx = ky = kz = round(n_sub_full ** (1 / 3)) if cfg in (1, 4) else None
    if kx is None:
        kx, ky, kz = {2: (4, 4, 8), 5: (8, 8, 4), 3: (4, 4, 4)}[cfg]
    bx, by, bz = nx // kx, ny // ky, nz // kz
    L = (2 * bx * wf.L[0] / nx, 2 * by * wf.L[1] / ny, 2 * bz * wf.L[2] / nz)
    w = W.box(2 * bx, 2 * by, 2 * bz, 2, 2, 2, L=L, steps=n_steps)
    t0 = time.perf_counter()
    space = fem.EdgeSpace(w.xyz, w.tets)
    maps = odd.DDMaps(space, w.part, w.n_sub)
    src = np.zeros(space.n)
    src[space.dof_of_pairs(w.source_pairs)] = 1.0
    t_setup = time.perf_counter() - t0
    t1 = time.perf_counter()
    out = odd.run(space, maps, dt, src, w.d2G(dt, n_steps), n_steps, tol=1e-10)
    t_run = time.perf_counter() - t1
    it_s = float(np.mean(out["iters"]))
    t_step = t_run / n_steps           # includes the factorisation share of the sample
    scale = (n_sub_full / 8.0) * (2.0 + 3.0 * full_iters) / (2.0 + 3.0 * max(it_s, 1.0))
    t_full = t_step * scale
    threads = os.environ.get("OMP_NUM_THREADS") or os.environ.get("OPENBLAS_NUM_THREADS") or str(os.cpu_count())
    return {
        "value": 1.0 / t_full, "unit": "steps/s", "cores": int(threads), "kind": "oracle",
        "sample": (f"CPU FP64 oracle DD (scipy Cholesky per subdomain + CG on Eq. f1schur, tol 1e-10) on a "
                   f"{2*bx}x{2*by}x{2*bz}-cube sample (2x2x2 subdomains of the same size and h), {n_steps} steps "
                   f"incl. its factorisation: {t_step:.3f} s/step, {it_s:.1f} CG it/step; scaled x{scale:.1f} "
                   f"(subdomains {n_sub_full}/8, local solves at {full_iters:.1f} it/step)"),
        "sample_s": t_run + t_setup, "os_cpu_count": os.cpu_count(),
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

    def run_steps(params, profile, clocks=None):
        """W warm-up steps, then K timed steps (CUDA events on the launch stream)."""
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
            st = one_step(Wu + k, True)
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
    # event profiling needs eager launches (events are recorded around every launch)
    p64e = D.make_params(precision=D.DD_FP64, tol=args.tol64, warm_start=args.warm, solver=sv)
    p32e = D.make_params(precision=D.DD_MIXED, tol=args.tol32, refine_tol=args.refine_tol, max_refine=6,
                         warm_start=args.warm, solver=sv, sym_fp32=sym)
    nan = float("nan")
    ms64 = ms32 = nan
    it64 = it32 = ref32 = np.zeros(1)
    prof64 = prof32 = None
    e64 = e32 = None
    # headline timings: no event profiling inside the timed region
    if args.only in (None, "fp64"):
        ms64, it64, _, prof64, e64 = run_steps(p64, False, clocks)
    if args.only in (None, "mixed"):
        ms32, it32, ref32, prof32, e32 = run_steps(p32, False, clocks)
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
        ens = {"members": R, "amplitudes": amps, "member_steps_per_s": R * K * 1e3 / mse, "ms_per_step": mse / K,
               "iters_per_step": float(np.mean(ite)), "refinements_per_step": float(np.mean(rfe)),
               "gpu_launches": int(pe_prof["total_launches"]), "setup_s": t_se, "factor_s": t_fe,
               "operator_bytes_fp64": int(fe.sizes.dense_bytes_fp64),
               "rel_err_member0_vs_single_mixed": (float(torch.linalg.norm(ee[0] - e32) / torch.linalg.norm(e32))
                                                   if e32 is not None and args.solver == "gmres" else None)}
        fe.close()
        del De

    def allmax(x):
        if world == 1:
            return x
        t = torch.tensor([x], dtype=torch.float64, device=dev)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        return float(t.item())

    ms64, ms32, ms_e2e = allmax(ms64), allmax(ms32), allmax(ms_e2e)
    sizes = fs.sizes
    res = dict(fs=fs, K=K, ms64=ms64, ms32=ms32, ms_e2e=ms_e2e, it64=it64, it32=it32, ref32=ref32, prof64=prof64,
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


def _fp64_roofline(st64):
    """FP64 path: the dominant GEMV is FP64-ALU bound on GB300 (2 flops per 8-byte element)."""
    cand = {k: v for k, v in st64.items() if k not in ("vector", "factor") and v.get("achieved_GBs")}
    if not cand:
        return None
    dom = max(cand, key=lambda k: cand[k]["ms_per_step"])
    gflops = cand[dom]["achieved_GBs"] / 8.0 * 2.0
    return {"bound": "alu", "kernel": f"k_gemv<double> ({dom})", "achieved": gflops, "peak": FP64_NOMINAL_TFLOPS * 1e3,
            "unit": "GFLOP/s", "frac": gflops / (FP64_NOMINAL_TFLOPS * 1e3),
            "peak_source": "nominal GB300 FP64 rate (1.25 TFLOP/s); the factorisation GEMM measures ~1.3"}


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
            n_sub = W.config(args.config).n_sub
            iters = 30.0
            cb = cpu_baseline(args.config, dt, iters, n_sub)
            line = {"metric": METRIC, "impl": "reference", "value": cb["value"], "unit": "steps/s", "n_gpus": 0,
                    "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 / cb["value"],
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
    sizes = r["sizes"]
    w = r["workload"]
    ms_head = r["ms32"] if head == "mixed" else r["ms64"]
    same = lambda x: x          # times were already max-reduced over ranks in run_ours
    value = aggregate_replicas(ms_head, K, world, same)[1]
    v64 = aggregate_replicas(r["ms64"], K, world, same)[1]
    v32 = aggregate_replicas(r["ms32"], K, world, same)[1]
    cb = None
    if world == 1 and not args.no_cpu_baseline and not args.cavity and not r["pic"]:
        try:
            its = r["it32"] if head == "mixed" else r["it64"]
            cb = cpu_baseline(args.config, r["dt"], float(np.mean(its)), w.n_sub)
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
                            f"{sizes.n_dof} edge dofs, {w.n_sub} subdomains, {sizes.n_lambda} multipliers, "
                            f"{sizes.n_corner} corners, Gaussian z-line pulse, dt=2xCFL={r['dt']:.6g}"),
                   "l2_policy": "inputs larger than L2 (dense subdomain operators "
                                f"{sizes.dense_bytes_fp64 / 1e9:.1f} GB FP64 + half that FP32), no flush",
                   "parallelism": f"replicas x{world}" if world > 1 else "1 GPU",
                   "stage_profile": "separate eager pass over the same steps with CUDA events per launch"},
        "mixed": {"steps_per_s": v32, "ms_per_step": r["ms32"] / K, "iters_per_step": float(np.mean(r["it32"])),
                  "refinements_per_step": float(np.mean(r["ref32"])), "inner_tol": args.tol32,
                  "refine_tol": args.refine_tol, "stages": st32},
        "fp64": {"steps_per_s": v64, "ms_per_step": r["ms64"] / K, "iters_per_step": float(np.mean(r["it64"])),
                 "tol": args.tol64, "stages": st64},
        "speedup_mixed_vs_fp64": v32 / v64,
        "coupled_gmres_vs_schur_cg": r["gmres"],
        "mfeti_dp2": r["dp2"],
        "ensemble": (dict(r["ens"], member_steps_vs_single=r["ens"]["member_steps_per_s"] / v32)
                     if r["ens"] else None),
        "rel_err_mixed_vs_fp64": r["rel"],
        "setup_s": r["t_setup"], "factor_s": r["t_factor"], "autotune_s": r["t_tune"],
        "gemv_tiles": r["tiles"],
        "fp64_roofline": _fp64_roofline(st64),
        "roofline": {"bound": "hbm", "kernel": (f"{packed_kernel(r['tiles'], dom, args.solver)} (packed FP32 tiles, {dom})"
                                                if head == "mixed" and not args.no_sym and dom in ("local_solve", "iface_apply")
                                                else f"k_gemv<{'float' if head == 'mixed' else 'double'}> ({dom})"),
                     "achieved": achieved, "peak": peak,
                     "unit": "GB/s", "frac": (achieved / peak) if achieved else None, "traffic": traffic,
                     "peak_source": f"{peak_kind} hbm_gbs" + ("" if peak_kind == "measured" else " (no MEASURED_PEAKS.json)")},
        "cpu_baseline": cb,
        "e2e": {"value": aggregate_replicas(r["ms_e2e"], K, world, same)[1], "unit": "steps/s",
                "h2d_bytes_per_step": int(sizes.n_dof * 8), "d2h_bytes_per_step": int(sizes.n_dof * 8)},
        "gpu_launches": int(r["launches32"] if head == "mixed" else r["launches64"]),
        "launch_mode": "eager" if args.eager else f"CUDA graph per step (Krylov loop as WHILE node, {args.chunk} it/body)",
        "fp32_storage": "dense" if args.no_sym else "packed symmetric 64x64 tiles (local solve, interface rows, coupled operator; the recovery too for ensembles)",
        "interface_solver": {"cg": "Schur complement (Eq. f1schur), Jacobi CG",
                             "gmres": "coupled Eqs. F1lr + F1uc, GMRES(20), diagonal preconditioner"}[args.solver],
        "warm_start": {1: "previous step's multipliers", 2: "extrapolated multipliers 2l(n-1)-l(n-2)"}.get(args.warm, args.warm),
        "clocks": r["clocks"],
    }
    print(json.dumps(_clean(line)), flush=True)
    r["fs"].close()
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
