"""Failure handling on the GPU without a GPU fault: a bounded device wait that
gives up is reported as DD_ERR_TIMEOUT, the step is not taken, and the context
stays usable.

The packed-tile GEMV (DD_MIXED, sym_fp32) waits on mbarriers for its tile
copies, each wait bounded.  dd_set_wait_limit makes the first wait of every CTA
poll an mbarrier that nothing completes for a few polls and give up -- the same
path a lost copy would take (error word, bounded drain of the copies in flight,
exit).  The test checks the status in eager and graph mode, that the time
level did not move, and that the next steps with normal waits match the
oracle's monolithic march."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import fem, newmark
from paper_2204_13254_gb300 import dd as D
from paper_2204_13254_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


@pytest.mark.parametrize("form", [None, 5])
@pytest.mark.parametrize("use_graph", [0, 1])
@pytest.mark.parametrize("solver", [D.DD_SOLVER_SCHUR_CG, D.DD_SOLVER_COUPLED_GMRES])
def test_wait_timeout_reported_and_recovered(use_graph, solver, form):
    """form None: the default packed forms; 5: the persistent queues (a consumer
    that gives up stops the producer and the stager warps too)."""
    need_gpu()
    n = 10
    w = W.cavity(4, 2, steps=n)
    space = fem.EdgeSpace(w.xyz, w.tets)
    T, S = space.assemble()
    dt = 2.0 * newmark.cfl_dt(T, S)
    src = np.zeros(space.n)
    src[space.dof_of_pairs(w.source_pairs)] = 1.0
    d2g = w.d2G(dt, n)
    ref = newmark.run(T, S, dt, src, d2g, n, keep=True)["fields"]

    fs = D.FieldSolver(w.xyz, w.tets, w.part, w.n_sub,
                       params=D.make_params(precision=D.DD_MIXED, tol=1e-6, max_refine=6, solver=solver,
                                            use_graph=use_graph, sym_fp32=1)).bind()
    try:
        fs.factor(dt)
        if form is not None:
            for kind in ("local", "recover", "iface_rows", "coupled"):
                D.dd_set_sym_config(fs.h, kind, 1, 4, 0, form)
        pat = torch.zeros(fs.n_dof, dtype=torch.float64, device="cuda")
        pat[torch.as_tensor(fs.dof_of_pairs(w.source_pairs), device="cuda")] = 1.0
        out = torch.empty_like(pat)
        for k in range(3):                       # three good steps
            D.dd_step_scaled(fs.h, pat, d2g[k], out)
        e_n, e_nm1, step = fs.get_state()
        assert step == 3
        D.dd_set_wait_limit(fs.h, 4)
        st = D.dd_step_scaled(fs.h, pat, d2g[3], out, stats=True, raise_on_error=False)
        assert st["rc"] == D.DD_ERR_TIMEOUT, st
        assert "wait" in D.lib().dd_last_error(fs.h).decode()
        e_n2, e_nm12, step2 = fs.get_state()
        assert step2 == 3                         # the step was not taken
        assert torch.equal(e_n2, e_n) and torch.equal(e_nm12, e_nm1)
        D.dd_set_wait_limit(fs.h, 0)              # normal waits: the march carries on
        worst = 0.0
        for k in range(3, n):
            D.dd_step_scaled(fs.h, pat, d2g[k], out)
            e = out.cpu().numpy()
            worst = max(worst, np.linalg.norm(e - ref[k]) / np.linalg.norm(ref[k]))
        assert worst <= 1e-8, worst
    finally:
        fs.close()
