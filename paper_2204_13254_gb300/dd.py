"""Thin Python binding of libdd.so (C ABI in include/dd.h).

Argument marshalling only: every step of the field solve runs in the CUDA
library.  Device buffers are torch tensors; their data pointers and the current
torch stream are passed straight through.  If libdd.so is missing the import
fails loudly -- there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libdd.so")

DD_OK, DD_ERR_ARG, DD_ERR_MESH, DD_ERR_PARTITION, DD_ERR_NOT_SPD = 0, 1, 2, 3, 4
DD_ERR_NO_CONVERGENCE, DD_ERR_NONFINITE, DD_ERR_TIMEOUT, DD_ERR_CUDA, DD_ERR_STATE = 5, 6, 7, 8, 9
DD_FP64, DD_MIXED = 0, 1
DD_SOLVER_SCHUR_CG, DD_SOLVER_COUPLED_GMRES = 0, 1
DD_MAX_RESTART = 32
DD_SCHEME_DP1, DD_SCHEME_DP2 = 0, 1
DD_FACTOR_FP64, DD_FACTOR_TENSOR = 0, 1

SYMBOLS = ["dd_setup", "dd_set_params", "dd_get_sizes", "dd_get_maps", "dd_set_probes", "dd_bind_workspace",
           "dd_factor", "dd_step", "dd_schur_apply", "dd_schur_apply_static", "dd_coupled_apply", "dd_dp2_apply",
           "dd_get_interface_mass", "dd_probe", "dd_adjoint_reset", "dd_adjoint_step", "dd_probe_seed", "dd_autotune",
           "dd_get_tiles", "dd_get_sym_config", "dd_set_sym_config", "dd_set_beam", "dd_pic_step", "dd_pic_state",
           "dd_get_state", "dd_set_state", "dd_profile", "dd_destroy", "dd_last_error", "dd_step_scaled",
           "dd_adjoint_step_scaled", "dd_probe_objective", "dd_set_eps", "dd_set_wait_limit", "dd_measure_fp64_rate",
           "dd_get_gemv_bytes", "dd_tc_selftest"]
N_STAGES = 9
STAGES = ["rhs", "local_solve", "iface_apply", "coarse", "corner", "recover", "vector", "refine", "factor"]


class dd_mesh(C.Structure):
    _fields_ = [("n_nodes", C.c_int64), ("n_tets", C.c_int64), ("xyz", C.POINTER(C.c_double)),
                ("tets", C.POINTER(C.c_int32)), ("eps", C.POINTER(C.c_double)), ("mu", C.c_double)]


class dd_params(C.Structure):
    _fields_ = [("precision", C.c_int), ("tol", C.c_double), ("max_it", C.c_int), ("precond", C.c_int),
                ("warm_start", C.c_int), ("refine_tol", C.c_double), ("max_refine", C.c_int), ("chunk", C.c_int),
                ("use_graph", C.c_int), ("solver", C.c_int), ("restart", C.c_int), ("sym_fp32", C.c_int),
                ("scheme", C.c_int), ("robin_alpha", C.c_double), ("members", C.c_int), ("factor_mode", C.c_int)]


class dd_sizes(C.Structure):
    _fields_ = [("n_edges", C.c_int64), ("n_dof", C.c_int64), ("n_sub", C.c_int32), ("n_lambda", C.c_int64),
                ("n_corner", C.c_int64), ("n_local", C.c_int64), ("nnz_local", C.c_int64), ("max_nr", C.c_int32),
                ("max_ns", C.c_int32), ("workspace_bytes", C.c_size_t), ("dense_bytes_fp64", C.c_int64),
                ("members", C.c_int32)]


class dd_maps(C.Structure):
    _fields_ = [("edges", C.c_void_p), ("dof_edge", C.c_void_p), ("sub_ptr", C.c_void_p), ("local_dof", C.c_void_p),
                ("n_int", C.c_void_p), ("n_gam", C.c_void_p), ("n_cor", C.c_void_p), ("mult_dof", C.c_void_p),
                ("mult_sub", C.c_void_p), ("mult_loc", C.c_void_p), ("corner_dof", C.c_void_p),
                ("owner", C.c_void_p)]


class dd_stats(C.Structure):
    _fields_ = [("iters", C.c_int), ("refinements", C.c_int), ("resid", C.c_double), ("status", C.c_int)]


class dd_beam(C.Structure):
    _fields_ = [("n_particles", C.c_int64), ("x_inj", C.POINTER(C.c_double)), ("v_inj", C.POINTER(C.c_double)),
                ("t_inj", C.POINTER(C.c_double)), ("q", C.c_double), ("qm", C.c_double)]


class dd_profile_stats(C.Structure):
    _fields_ = [("launches", C.c_int64 * N_STAGES), ("work", C.c_int64 * N_STAGES), ("ms", C.c_double * N_STAGES),
                ("bytes", C.c_double * N_STAGES), ("total_launches", C.c_int64)]


def load_library(path: str = LIB_PATH):
    if not os.path.exists(path):
        raise ImportError(f"libdd.so not built at {path}; run paper_2204_13254_gb300.build.build()")
    lib = C.CDLL(path)
    vp, i32, i64 = C.c_void_p, C.c_int32, C.c_int64
    sig = {
        "dd_setup": (C.c_int, [C.POINTER(dd_mesh), C.POINTER(C.c_int32), i32, C.POINTER(dd_params), C.POINTER(vp)]),
        "dd_set_params": (C.c_int, [vp, C.POINTER(dd_params)]),
        "dd_get_sizes": (C.c_int, [vp, C.POINTER(dd_sizes)]),
        "dd_get_maps": (C.c_int, [vp, C.POINTER(dd_maps)]),
        "dd_set_probes": (C.c_int, [vp, i32, C.POINTER(C.c_double)]),
        "dd_bind_workspace": (C.c_int, [vp, vp, C.c_size_t, vp]),
        "dd_factor": (C.c_int, [vp, C.c_double, vp]),
        "dd_step": (C.c_int, [vp, vp, vp, C.POINTER(dd_stats), vp]),
        "dd_schur_apply": (C.c_int, [vp, vp, vp, vp]),
        "dd_schur_apply_static": (C.c_int, [vp, vp, vp, vp]),
        "dd_coupled_apply": (C.c_int, [vp, vp, vp, vp]),
        "dd_dp2_apply": (C.c_int, [vp, vp, vp, vp]),
        "dd_get_interface_mass": (C.c_int, [vp, C.POINTER(i64), vp, vp, vp]),
        "dd_probe": (C.c_int, [vp, vp, vp]),
        "dd_get_state": (C.c_int, [vp, vp, vp, C.POINTER(i64), vp]),
        "dd_set_state": (C.c_int, [vp, vp, vp, i64, vp]),
        "dd_profile": (C.c_int, [vp, C.c_int, C.POINTER(dd_profile_stats), vp]),
        "dd_adjoint_reset": (C.c_int, [vp, vp]),
        "dd_adjoint_step": (C.c_int, [vp, vp, vp, vp, vp, vp, vp, vp, vp, C.POINTER(dd_stats), vp]),
        "dd_probe_seed": (C.c_int, [vp, vp, C.c_double, vp, vp]),
        "dd_autotune": (C.c_int, [vp, C.c_char_p, C.POINTER(C.c_double), vp]),
        "dd_get_tiles": (C.c_int, [vp, C.POINTER(C.c_int32), C.POINTER(C.c_int32)]),
        "dd_get_sym_config": (C.c_int, [vp, C.POINTER(C.c_int32), C.POINTER(C.c_int32), C.POINTER(C.c_int32),
                                        C.POINTER(C.c_int32)]),
        "dd_set_sym_config": (C.c_int, [vp, C.c_int32, C.c_int32, C.c_int32, C.c_int32, C.c_int32, vp]),
        "dd_set_beam": (C.c_int, [vp, C.POINTER(dd_beam)]),
        "dd_pic_step": (C.c_int, [vp, C.POINTER(dd_stats), vp]),
        "dd_pic_state": (C.c_int, [vp, vp, vp, vp, vp, C.POINTER(C.c_int64), vp]),
        "dd_step_scaled": (C.c_int, [vp, vp, C.c_double, vp, C.POINTER(dd_stats), vp]),
        "dd_adjoint_step_scaled": (C.c_int, [vp, vp, vp, vp, vp, vp, C.c_double, vp, vp, vp, C.POINTER(dd_stats),
                                             vp]),
        "dd_probe_objective": (C.c_int, [vp, vp, C.c_double, vp, vp]),
        "dd_set_eps": (C.c_int, [vp, vp, vp]),
        "dd_set_wait_limit": (C.c_int, [vp, C.c_int32, vp]),
        "dd_measure_fp64_rate": (C.c_int, [C.POINTER(C.c_double), vp]),
        "dd_get_gemv_bytes": (C.c_int, [vp, C.c_int32, C.c_int32, C.POINTER(C.c_double), C.POINTER(C.c_double)]),
        "dd_tc_selftest": (C.c_int, [C.POINTER(C.c_int32), vp]),
        "dd_destroy": (None, [vp]),
        "dd_last_error": (C.c_char_p, [vp]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    return lib


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = load_library()
    return _lib


class DDError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"dd status {code}: {msg}")
        self.code = code


def _ptr(t):
    return None if t is None else C.c_void_p(t.data_ptr())


def _stream(stream=None):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


def make_params(precision=DD_FP64, tol=1e-12, max_it=500, precond=1, warm_start=1, refine_tol=1e-12, max_refine=4,
                chunk=8, use_graph=0, solver=DD_SOLVER_SCHUR_CG, restart=20, sym_fp32=1, scheme=DD_SCHEME_DP1,
                robin_alpha=0.0, members=1, factor_mode=DD_FACTOR_TENSOR):
    return dd_params(precision, tol, max_it, precond, warm_start, refine_tol, max_refine, chunk, use_graph, solver,
                     restart, sym_fp32, scheme, robin_alpha, members, factor_mode)


# ---- C-ABI-named wrappers ------------------------------------------------------

def dd_setup(xyz, tets, part, n_sub, eps=None, mu=1.0, params=None):
    """Host tearing (no GPU work).  Returns an opaque handle (c_void_p)."""
    L = lib()
    xyz = np.ascontiguousarray(xyz, dtype=np.float64)
    tets = np.ascontiguousarray(tets, dtype=np.int32)
    part = np.ascontiguousarray(part, dtype=np.int32)
    epsa = None if eps is None else np.ascontiguousarray(eps, dtype=np.float64)
    m = dd_mesh(len(xyz), len(tets), xyz.ctypes.data_as(C.POINTER(C.c_double)),
                tets.ctypes.data_as(C.POINTER(C.c_int32)),
                None if epsa is None else epsa.ctypes.data_as(C.POINTER(C.c_double)), float(mu))
    h = C.c_void_p()
    prm = params if params is not None else make_params()
    rc = L.dd_setup(C.byref(m), part.ctypes.data_as(C.POINTER(C.c_int32)), int(n_sub), C.byref(prm), C.byref(h))
    if rc != DD_OK:
        msg = L.dd_last_error(h).decode() if h.value else ""
        if h.value:
            L.dd_destroy(h)
        raise DDError(rc, msg)
    return h


def _check(h, rc):
    if rc != DD_OK:
        raise DDError(rc, lib().dd_last_error(h).decode())


def dd_get_sizes(h):
    s = dd_sizes()
    _check(h, lib().dd_get_sizes(h, C.byref(s)))
    return s


def dd_get_maps(h):
    s = dd_get_sizes(h)
    out = dict(
        edges=np.zeros((s.n_edges, 2), np.int64), dof_edge=np.zeros(s.n_dof, np.int64),
        sub_ptr=np.zeros(s.n_sub + 1, np.int64), local_dof=np.zeros(s.n_local, np.int64),
        n_int=np.zeros(s.n_sub, np.int32), n_gam=np.zeros(s.n_sub, np.int32), n_cor=np.zeros(s.n_sub, np.int32),
        mult_dof=np.zeros(s.n_lambda, np.int64), mult_sub=np.zeros((s.n_lambda, 2), np.int32),
        mult_loc=np.zeros((s.n_lambda, 2), np.int32), corner_dof=np.zeros(s.n_corner, np.int64),
        owner=np.zeros(s.n_dof, np.int32))
    m = dd_maps(*[out[k].ctypes.data for k, _ in dd_maps._fields_])
    _check(h, lib().dd_get_maps(h, C.byref(m)))
    return out


def dd_set_probes(h, points):
    p = np.ascontiguousarray(points, dtype=np.float64).reshape(-1, 3)
    _check(h, lib().dd_set_probes(h, len(p), p.ctypes.data_as(C.POINTER(C.c_double))))


def dd_bind_workspace(h, ws, stream=None):
    _check(h, lib().dd_bind_workspace(h, _ptr(ws), ws.numel() * ws.element_size(), _stream(stream)))


def dd_factor(h, dt, stream=None):
    _check(h, lib().dd_factor(h, float(dt), _stream(stream)))


def dd_step(h, d2g=None, e_out=None, stats=True, stream=None, raise_on_error=True):
    st = dd_stats()
    rc = lib().dd_step(h, _ptr(d2g), _ptr(e_out), C.byref(st) if stats else None, _stream(stream))
    if raise_on_error:
        _check(h, rc)
    return dict(rc=rc, iters=st.iters, refinements=st.refinements, resid=st.resid, status=st.status)


def dd_step_scaled(h, d2g, scale, e_out=None, stats=True, stream=None, raise_on_error=True):
    """dd_step with the source scale * d2g (d2g: device pattern, scale: host scalar)."""
    st = dd_stats()
    rc = lib().dd_step_scaled(h, _ptr(d2g), float(scale), _ptr(e_out), C.byref(st) if stats else None,
                              _stream(stream))
    if raise_on_error:
        _check(h, rc)
    return dict(rc=rc, iters=st.iters, refinements=st.refinements, resid=st.resid, status=st.status)


def dd_probe_objective(h, J, weight=1.0, e=None, stream=None):
    """J (device scalar) += weight * sum_p |E(r_p; e)|^2, e = the current e^n when None."""
    _check(h, lib().dd_probe_objective(h, _ptr(e), float(weight), _ptr(J), _stream(stream)))


def dd_set_eps(h, eps, stream=None):
    """New per-tet permittivity (device tensor [n_tets]); factor again afterwards."""
    _check(h, lib().dd_set_eps(h, _ptr(eps), _stream(stream)))


def dd_set_wait_limit(h, first_wait_polls, stream=None):
    """Failure-path testing aid: the first packed-GEMV wait of every CTA gives up after this many polls."""
    _check(h, lib().dd_set_wait_limit(h, int(first_wait_polls), _stream(stream)))


def dd_measure_fp64_rate(stream=None):
    """FP64 FMA throughput of the current device (TFLOP/s, CUDA-event timed)."""
    v = C.c_double()
    rc = lib().dd_measure_fp64_rate(C.byref(v), _stream(stream))
    if rc != DD_OK:
        raise DDError(rc, "dd_measure_fp64_rate failed")
    return v.value


def dd_get_gemv_bytes(h, kind, precision):
    """(algorithmic, streamed) bytes of one full launch of a GEMV kind (name or index)."""
    k = GEMV_KINDS.index(kind) if isinstance(kind, str) else int(kind)
    a, b = C.c_double(), C.c_double()
    _check(h, lib().dd_get_gemv_bytes(h, k, int(precision), C.byref(a), C.byref(b)))
    return a.value, b.value


def dd_tc_selftest(stream=None):
    """Bitmask of the tcgen05 operand layouts whose 128x16x64 BF16 MMA matched the CUDA cores exactly."""
    m = C.c_int32()
    rc = lib().dd_tc_selftest(C.byref(m), _stream(stream))
    if rc != DD_OK:
        raise DDError(rc, "dd_tc_selftest failed")
    return m.value


def dd_schur_apply(h, lam, out, stream=None):
    _check(h, lib().dd_schur_apply(h, _ptr(lam), _ptr(out), _stream(stream)))


def dd_schur_apply_static(h, lam, out, stream=None):
    """dd_schur_apply without any device allocation (scratch in a fixed device array)."""
    _check(h, lib().dd_schur_apply_static(h, _ptr(lam), _ptr(out), _stream(stream)))


def dd_coupled_apply(h, u, out, stream=None):
    """out = [F_rr u_l + F_rc u_c ; -F_rc^T u_l + K~cc u_c] (Eqs. F1lr + F1uc), u = [u_l; u_c]."""
    _check(h, lib().dd_coupled_apply(h, _ptr(u), _ptr(out), _stream(stream)))


def dd_dp2_apply(h, u, out, stream=None):
    """out = DP2 coupled operator (Eqs. f2imp1 + F2un) applied to u = [l1; l2; x_c]."""
    _check(h, lib().dd_dp2_apply(h, _ptr(u), _ptr(out), _stream(stream)))


def dd_get_interface_mass(h):
    """Host CSR (ptr, col, val) of the interface tangential mass on the multiplier edges."""
    nnz = C.c_int64()
    _check(h, lib().dd_get_interface_mass(h, C.byref(nnz), None, None, None))
    s = dd_get_sizes(h)
    ptr = np.zeros(s.n_lambda + 1, np.int64)
    col = np.zeros(max(nnz.value, 1), np.int32)
    val = np.zeros(max(nnz.value, 1), np.float64)
    _check(h, lib().dd_get_interface_mass(h, C.byref(nnz), ptr.ctypes.data, col.ctypes.data, val.ctypes.data))
    return ptr, col[:nnz.value], val[:nnz.value]


def dd_probe(h, out, stream=None):
    _check(h, lib().dd_probe(h, _ptr(out), _stream(stream)))


def dd_get_state(h, e_n, e_nm1, stream=None):
    step = C.c_int64()
    _check(h, lib().dd_get_state(h, _ptr(e_n), _ptr(e_nm1), C.byref(step), _stream(stream)))
    return step.value


def dd_set_state(h, e_n, e_nm1, step, stream=None):
    _check(h, lib().dd_set_state(h, _ptr(e_n), _ptr(e_nm1), int(step), _stream(stream)))


def dd_adjoint_reset(h, stream=None):
    _check(h, lib().dd_adjoint_reset(h, _stream(stream)))


def dd_adjoint_step(h, seed, e_k=None, e_km1=None, e_km2=None, d2g_hat=None, grad_eps=None, grad_amp=None,
                    mu_out=None, stats=True, stream=None):
    st = dd_stats()
    rc = lib().dd_adjoint_step(h, _ptr(seed), _ptr(e_k), _ptr(e_km1), _ptr(e_km2), _ptr(d2g_hat), _ptr(grad_eps),
                               _ptr(grad_amp), _ptr(mu_out), C.byref(st) if stats else None, _stream(stream))
    _check(h, rc)
    return dict(rc=rc, iters=st.iters, refinements=st.refinements, resid=st.resid, status=st.status)


def dd_adjoint_step_scaled(h, seed, e_k, e_km1, e_km2, d2g_hat, d2g_scale, grad_eps=None, grad_amp=None,
                           mu_out=None, stats=True, stream=None):
    """dd_adjoint_step with the unit source d2g_scale * d2g_hat."""
    st = dd_stats()
    rc = lib().dd_adjoint_step_scaled(h, _ptr(seed), _ptr(e_k), _ptr(e_km1), _ptr(e_km2), _ptr(d2g_hat),
                                      float(d2g_scale), _ptr(grad_eps), _ptr(grad_amp), _ptr(mu_out),
                                      C.byref(st) if stats else None, _stream(stream))
    _check(h, rc)
    return dict(rc=rc, iters=st.iters, refinements=st.refinements, resid=st.resid, status=st.status)


def dd_probe_seed(h, e, weight, seed, stream=None):
    _check(h, lib().dd_probe_seed(h, _ptr(e), float(weight), _ptr(seed), _stream(stream)))


def dd_set_beam(h, x_inj, v_inj, t_inj, q, qm):
    x = np.ascontiguousarray(x_inj, dtype=np.float64).reshape(-1, 3)
    v = np.ascontiguousarray(v_inj, dtype=np.float64).reshape(-1, 3)
    t = np.ascontiguousarray(t_inj, dtype=np.float64)
    dp = C.POINTER(C.c_double)
    b = dd_beam(len(x), x.ctypes.data_as(dp), v.ctypes.data_as(dp), t.ctypes.data_as(dp), float(q), float(qm))
    _check(h, lib().dd_set_beam(h, C.byref(b)))


def dd_pic_step(h, stats=True, stream=None):
    st = dd_stats()
    _check(h, lib().dd_pic_step(h, C.byref(st) if stats else None, _stream(stream)))
    return dict(iters=st.iters, refinements=st.refinements, resid=st.resid, status=st.status)


def dd_pic_state(h, x=None, status=None, G=None, b=None, stream=None):
    nf = C.c_int64()
    _check(h, lib().dd_pic_state(h, _ptr(x), _ptr(status), _ptr(G), _ptr(b), C.byref(nf), _stream(stream)))
    return nf.value


GEMV_KINDS = ["local", "corner_rows", "corner_coupling", "recover", "coarse", "iface_rows", "coupled"]


def dd_autotune(h, cache_path=None, stream=None):
    """Time candidate GEMV tiles on the factored operators; returns wall seconds."""
    secs = C.c_double()
    _check(h, lib().dd_autotune(h, cache_path.encode() if cache_path else None, C.byref(secs), _stream(stream)))
    return secs.value


def dd_get_tiles(h):
    nk = len(GEMV_KINDS)
    lpr = (C.c_int32 * (2 * nk))()
    rows = (C.c_int32 * (2 * nk))()
    _check(h, lib().dd_get_tiles(h, lpr, rows))
    return {("fp64", "fp32")[p]: {GEMV_KINDS[k]: (lpr[nk * p + k], rows[nk * p + k]) for k in range(nk)}
            for p in range(2)}


def dd_get_sym_config(h):
    """Packed symmetric GEMV kinds: {kind: (CTAs per subdomain, TMA ring depth, subdomains kept in L2,
    kernel form: 1 warp-specialised, 0 CTA-synchronous)}."""
    nk = len(GEMV_KINDS)
    cl = (C.c_int32 * nk)()
    st = (C.c_int32 * nk)()
    keep = (C.c_int32 * nk)()
    ws = (C.c_int32 * nk)()
    _check(h, lib().dd_get_sym_config(h, cl, st, keep, ws))
    return {GEMV_KINDS[k]: (cl[k], st[k], keep[k], ws[k]) for k in range(nk) if cl[k]}


def dd_set_sym_config(h, kind, cl, st, keep=0, ws=0):
    """Pins the packed-tile launch of GEMV kind `kind` ("local", "iface_rows" or "coupled")."""
    _check(h, lib().dd_set_sym_config(h, GEMV_KINDS.index(kind), cl, st, keep, ws, _stream()))


def dd_profile(h, enable=-1, read=True, stream=None):
    """enable: 1 reset+start, 0 stop, -1 unchanged.  Returns per-stage dict when read."""
    st = dd_profile_stats()
    _check(h, lib().dd_profile(h, int(enable), C.byref(st) if read else None, _stream(stream)))
    if not read:
        return None
    return dict(total_launches=st.total_launches,
                stages={STAGES[k]: dict(launches=st.launches[k], work=st.work[k], ms=st.ms[k], bytes=st.bytes[k])
                        for k in range(N_STAGES)})


def dd_destroy(h):
    if h is not None and h.value:
        lib().dd_destroy(h)


# ---- convenience wrapper ---------------------------------------------------------

class FieldSolver:
    """Owns a handle and its torch-allocated workspace on one CUDA device."""

    def __init__(self, xyz, tets, part, n_sub, eps=None, mu=1.0, params=None, probes=None, device="cuda"):
        self.h = dd_setup(xyz, tets, part, n_sub, eps, mu, params)
        self.n_tets = len(tets)
        self.sizes = dd_get_sizes(self.h)
        self.n_dof = self.sizes.n_dof
        self.n_lambda = self.sizes.n_lambda
        self.members = self.sizes.members          # ensemble size: member r owns dofs [r, r + 1) * n_dof_member
        self.n_dof_member = self.n_dof // self.members
        self.n_nodes = len(xyz)
        if probes is not None:
            dd_set_probes(self.h, probes)
        self.n_probe = 0 if probes is None else len(np.asarray(probes).reshape(-1, 3))
        self.device = device
        self.ws = None

    def bind(self):
        import torch
        nbytes = self.sizes.workspace_bytes
        self.ws = torch.empty(nbytes + 256, dtype=torch.uint8, device=self.device)
        off = (-self.ws.data_ptr()) % 256
        self.ws_view = self.ws[off:off + nbytes]
        dd_bind_workspace(self.h, self.ws_view)
        return self

    def maps(self):
        return dd_get_maps(self.h)

    def dof_of_pairs(self, pairs, member=0):
        """dof ids of node pairs (lo, hi) of ensemble member `member` -- host
        marshalling for source vectors."""
        pairs = np.asarray(pairs) + member * self.n_nodes
        m = self.maps()
        edges = m["edges"][m["dof_edge"]]
        n = int(max(edges.max(), np.max(pairs))) + 1
        keys = edges[:, 0] * n + edges[:, 1]
        pk = pairs[:, 0] * n + pairs[:, 1]
        pos = np.searchsorted(keys, pk)
        assert np.all(keys[pos] == pk), "pair is not an interior edge"
        return pos

    def factor(self, dt):
        dd_factor(self.h, dt)

    def set_params(self, params):
        _check(self.h, lib().dd_set_params(self.h, C.byref(params)))

    def step(self, d2g=None, e_out=None, stats=True, raise_on_error=True):
        return dd_step(self.h, d2g, e_out, stats, raise_on_error=raise_on_error)

    def schur_apply(self, lam):
        import torch
        out = torch.empty_like(lam)
        dd_schur_apply(self.h, lam, out)
        return out

    def coupled_apply(self, u):
        import torch
        out = torch.empty_like(u)
        dd_coupled_apply(self.h, u, out)
        return out

    def set_beam(self, x_inj, v_inj, t_inj, q, qm):
        """Particles for dd_pic_step (before bind())."""
        dd_set_beam(self.h, x_inj, v_inj, t_inj, q, qm)
        self.n_particles = len(np.asarray(t_inj))
        self.sizes = dd_get_sizes(self.h)
        return self

    def pic_step(self, stats=True):
        return dd_pic_step(self.h, stats)

    def pic_state(self):
        import torch
        nf = dd_pic_state(self.h)
        x = torch.empty(3 * self.n_particles, dtype=torch.float64, device=self.device)
        st = torch.empty(self.n_particles, dtype=torch.int32, device=self.device)
        G = torch.empty(self.n_dof, dtype=torch.float64, device=self.device)
        b = torch.empty(nf, dtype=torch.float64, device=self.device)
        dd_pic_state(self.h, x, st, G, b)
        return x.view(-1, 3), st, G, b

    def probe(self):
        import torch
        out = torch.empty(3 * self.n_probe, dtype=torch.float64, device=self.device)
        dd_probe(self.h, out)
        return out

    def get_state(self):
        import torch
        a = torch.empty(self.n_dof, dtype=torch.float64, device=self.device)
        b = torch.empty_like(a)
        step = dd_get_state(self.h, a, b)
        return a, b, step

    def set_state(self, e_n, e_nm1, step):
        dd_set_state(self.h, e_n, e_nm1, step)

    def profile(self, enable=-1, read=True):
        return dd_profile(self.h, enable, read)

    def close(self):
        dd_destroy(self.h)
        self.h = None
        self.ws = None

    def __del__(self):
        try:
            if getattr(self, "h", None) is not None:
                self.close()
        except Exception:
            pass
