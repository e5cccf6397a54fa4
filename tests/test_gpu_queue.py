"""The persistent packed form (dd_set_sym_config ws = 5, cl = consumer groups):
the subdomains are dealt out, largest first, to as many CTAs as the SMs hold,
and each CTA streams the tiles of its whole queue through one ring while
helper warps stage x of the next subdomain and store y of the last.  With one
consumer group it does the arithmetic of the warp-specialised form in the same
order, so its marches are bitwise those of that form; with 2 or 4 groups the
tiles alternate between groups (other FP32 sums, still deterministic).  On the
48^3 cavity (512 subdomains over 152 to 304 CTAs) every CTA serves several
subdomains."""
import json
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import fem, newmark
from paper_2204_13254_gb300 import dd as D
from paper_2204_13254_gb300 import workloads as W

pytestmark = pytest.mark.gpu
GOLD = os.path.join(os.path.dirname(__file__), "golden")
DT = json.load(open(os.path.join(GOLD, "cfl_dt.json")))
PACKED = ("local", "recover", "iface_rows", "coupled")


def need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def marches(w, dt, n, configs, solver=D.DD_SOLVER_COUPLED_GMRES):
    """One handle, factored once; for every configuration the n-step mixed march
    from rest.  A configuration is (cl, st, keep, ws) for every packed kind, or a
    pair of them: the first for the local solve and the recovery (whose index
    range, and so the staged x and partial y, spans the whole subdomain), the
    second for the interface rows and the coupled operator."""
    fs = D.FieldSolver(w.xyz, w.tets, w.part, w.n_sub, w.eps, w.mu,
                       params=D.make_params(precision=D.DD_MIXED, tol=1e-5, refine_tol=1e-10, max_refine=6,
                                            solver=solver, use_graph=1, chunk=2)).bind()
    fs.factor(dt)
    pat = torch.zeros(fs.n_dof, dtype=torch.float64, device="cuda")
    pat[torch.as_tensor(fs.dof_of_pairs(w.source_pairs), device="cuda")] = 1.0
    d2g = w.d2G(dt, n)
    zero = torch.zeros(fs.n_dof, dtype=torch.float64, device="cuda")
    out = []
    try:
        for cfg in configs:
            per = dict(zip(PACKED, (cfg[0], cfg[0], cfg[1], cfg[1]) if isinstance(cfg[0], tuple) else (cfg,) * 4))
            for kind in PACKED:
                D.dd_set_sym_config(fs.h, kind, *per[kind])
            assert all(D.dd_get_sym_config(fs.h)[k] == tuple(per[k]) for k in PACKED)
            fs.set_state(zero, zero, 0)
            e = torch.empty_like(zero)
            fields, its = [], []
            for k in range(n):
                st = D.dd_step_scaled(fs.h, pat, d2g[k], e)
                assert st["status"] == 0, (cfg, st)
                its.append((st["iters"], st["refinements"]))
                fields.append(e.clone())
            out.append((torch.stack(fields), its))
    finally:
        fs.close()
    return out


@pytest.mark.parametrize("solver", [D.DD_SOLVER_SCHUR_CG, D.DD_SOLVER_COUPLED_GMRES])
def test_queue_form_bitwise_equals_warp_specialised_and_oracle(solver):
    need_gpu()
    """Eight subdomains of 6^3 cubes (the bench's subdomain size), one queue
    entry per CTA; rings of 4 to 10 tiles, one or two CTAs per SM, L2-kept
    subsets."""
    n = 12
    w = W.cavity(12, 2, steps=n)
    dt = 0.04
    runs = marches(w, dt, n, [(1, 2, 0, 1), (1, 6, 0, 5), ((1, 8, 3, 5), (1, 10, 8, 5)), (1, 6, 0, 5),
                              ((2, 4, 3, 5), (2, 6, 0, 5)), ((2, 2, 0, 5), (4, 8, 3, 5)), ((2, 4, 3, 5), (2, 6, 0, 5))],
                   solver)
    ref_f, ref_its = runs[0]
    for f, its in runs[1:4]:   # one consumer group: the warp-specialised form's sums, bitwise
        assert torch.equal(f, ref_f)
        assert its == ref_its
    assert torch.equal(runs[4][0], runs[6][0]) and runs[4][1] == runs[6][1]   # deterministic
    space = fem.EdgeSpace(w.xyz, w.tets)
    T, S = space.assemble()
    src = np.zeros(space.n)
    src[space.dof_of_pairs(w.source_pairs)] = 1.0
    mono = newmark.run(T, S, dt, src, w.d2G(dt, n), n, keep=True)["fields"]
    for f, _ in runs[1:]:
        F = f.cpu().numpy()
        worst = max(np.linalg.norm(F[k] - mono[k]) / np.linalg.norm(mono[k]) for k in range(2, n))
        assert worst <= 1e-8, worst


def test_queue_form_fullsize_cavity48():
    """512 subdomains of 6^3 cubes: queues of three to four subdomains per CTA."""
    need_gpu()
    w = W.config(4)
    dt = DT["config4"]["dt"]
    runs = marches(w, dt, 5, [(1, 2, 99, 1), (1, 8, 99, 5), ((1, 6, 19, 5), (1, 4, 0, 5)),
                              ((2, 4, 0, 5), (4, 8, 99, 5)), ((2, 4, 0, 5), (4, 8, 99, 5))])
    for f, its in runs[1:3]:   # one consumer group: bitwise the warp-specialised form
        assert torch.equal(f, runs[0][0])
        assert its == runs[0][1]
    assert torch.equal(runs[3][0], runs[4][0])   # several groups: other FP32 sums, deterministic
    rel = torch.linalg.norm(runs[3][0][-1] - runs[0][0][-1]) / torch.linalg.norm(runs[0][0][-1])
    assert rel <= 1e-8, float(rel)


def test_queue_form_rejects_bad_values():
    need_gpu()
    w = W.config(1)
    fs = D.FieldSolver(w.xyz, w.tets, w.part, w.n_sub, w.eps, w.mu,
                       D.make_params(precision=D.DD_MIXED, tol=1e-5)).bind()
    fs.factor(DT["config1"]["dt"])
    try:
        before = D.dd_get_sym_config(fs.h)["coupled"]
        for args in [("coupled", 3, 4, 0, 5), ("coupled", 4, 2, 0, 5), ("coupled", 1, 11, 0, 5),
                     ("coupled", 1, 1, 0, 5), ("coupled", 1, 4, w.n_sub + 1, 5), ("coupled", 8, 8, 0, 5),
                     ("coupled", 4, 6, 0, 5), ("coupled", 2, 3, 0, 5)]:
            with pytest.raises(RuntimeError):
                D.dd_set_sym_config(fs.h, *args)
            assert D.dd_get_sym_config(fs.h)["coupled"] == before
        D.dd_set_sym_config(fs.h, "coupled", 4, 4, 1, 5)
        assert D.dd_get_sym_config(fs.h)["coupled"] == (4, 4, 1, 5)
    finally:
        fs.close()
