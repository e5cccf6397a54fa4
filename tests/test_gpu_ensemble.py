"""Multi-RHS batching (dd_params.members = R): R independent field problems on one
mesh, marched together with the factored operators stored once.

Every member is checked against its own oracle march (the monolithic sparse LU
of the Newmark matrix, the member's own source), so the batched path must give
each member the fields it would get alone, to the parity bounds of the single
problem: FP64 <= 1e-10, DD_MIXED <= 1e-8 relative L2 per step.  The members
differ in source line and amplitude (one is -2 times another: linearity), and
the tests cover MFETI-DP1 and DP2, eager and graph launches, a block split and a
ragged RCB split of a jittered mesh."""
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
G = D.DD_SOLVER_COUPLED_GMRES


def need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def member_sources(w, dims):
    """(node pairs, amplitude) per member: the workload's line, another z-line, and
    the workload's line at -2x."""
    nx, ny, nz = dims
    other = W.z_line_node_pairs(nx, ny, nz, nx // 2 - 1, ny // 2 + 1)
    return [(w.source_pairs, 1.0), (other, 0.5), (w.source_pairs, -2.0)]


def oracle_member(w, dt, n, pairs, amp):
    space = fem.EdgeSpace(w.xyz, w.tets, w.eps, w.mu)
    T, S = space.assemble()
    src = np.zeros(space.n)
    src[space.dof_of_pairs(pairs)] = amp
    return newmark.run(T, S, dt, src, w.d2G(dt, n), n, keep=True)["fields"]


def run_ensemble(w, dt, n, prm, sources, after_factor=None):
    fs = D.FieldSolver(w.xyz, w.tets, w.part, w.n_sub, w.eps, w.mu, prm).bind()
    fs.factor(dt)
    if after_factor:
        after_factor(fs)
    R, nd = fs.members, fs.n_dof_member
    assert R == len(sources)
    d2g = w.d2G(dt, n)
    dofs = [fs.dof_of_pairs(p, member=r) for r, (p, _) in enumerate(sources)]
    src = torch.zeros(fs.n_dof, dtype=torch.float64, device="cuda")
    out = torch.empty_like(src)
    fields, stats = [], []
    for k in range(n):
        src.zero_()
        for r, (_, amp) in enumerate(sources):
            src[dofs[r]] = amp * float(d2g[k])
        st = fs.step(src, out)
        stats.append(st)
        fields.append(out.cpu().numpy().reshape(R, nd).copy())
    fs.close()
    return np.array(fields), stats     # [n, R, nd]


def rel_err(a, b):
    return np.linalg.norm(a - b, axis=-1) / np.maximum(np.linalg.norm(b, axis=-1), 1e-300)


CASES = {
    "dp1_fp64": (D.make_params(tol=1e-13, solver=G, max_it=3000, members=3), 1e-10),
    "dp1_mixed_graph": (D.make_params(precision=D.DD_MIXED, tol=1e-5, refine_tol=1e-12, max_refine=8, solver=G,
                                      use_graph=1, chunk=2, members=3), 1e-8),
    "dp2_mixed": (D.make_params(precision=D.DD_MIXED, tol=1e-5, refine_tol=1e-12, max_refine=8, solver=G,
                                scheme=D.DD_SCHEME_DP2, members=3), 1e-8),
}


@pytest.mark.parametrize("name", list(CASES))
def test_ensemble_members_match_their_oracles(name):
    need_gpu()
    prm, bound = CASES[name]
    w = W.config(1)
    dt = DT["config1"]["dt"]
    n = 40
    sources = member_sources(w, w.dims)
    f, stats = run_ensemble(w, dt, n, prm, sources)
    assert all(s["status"] == 0 for s in stats)
    for r, (pairs, amp) in enumerate(sources):
        ref = oracle_member(w, dt, n, pairs, amp)
        err = rel_err(f[:, r], ref)
        assert err[2:].max() <= bound, (name, r, err.max())
    # linearity: member 2 is -2 x member 0
    assert np.abs(f[:, 2] + 2.0 * f[:, 0]).max() <= 10 * bound * np.abs(f[:, 0]).max()


def test_ensemble_ragged_rcb_mixed():
    """Jittered mesh, ragged RCB split (group sizes not multiples of the tile edge)."""
    need_gpu()
    nx, ny, nz = 10, 8, 8
    L = (1.2, 1.0, 1.0)
    xyz, tets = W.kuhn_box(nx, ny, nz, *L)
    xyz, rng = W.jitter_nodes(xyz, L[0] / nx, L, 0.2, seed=9)
    part = W.rcb_partition(W.tet_centroids(xyz, tets), 6, rng.uniform(0.6, 1.4, size=6))
    w = W.Workload("ragged", xyz, tets, part, 6, rng.uniform(1, 4, size=len(tets)), 1.0, 30,
                   W.z_line_node_pairs(nx, ny, nz, 5, 4))
    space = fem.EdgeSpace(xyz, tets, w.eps)
    T, S = space.assemble()
    dt = 2.0 * newmark.cfl_dt(T, S)
    n = 30
    sources = member_sources(w, (nx, ny, nz))[:2]
    prm = D.make_params(precision=D.DD_MIXED, tol=1e-5, refine_tol=1e-12, max_refine=8, solver=G, members=2)
    f, stats = run_ensemble(w, dt, n, prm, sources)
    assert all(s["status"] == 0 for s in stats)
    for r, (pairs, amp) in enumerate(sources):
        err = rel_err(f[:, r], oracle_member(w, dt, n, pairs, amp))
        assert err[2:].max() <= 1e-8, (r, err.max())


@pytest.mark.parametrize("form", [(2, 1, 2, 0), (2, 2, 3, 2), (2, 8, 4, 1), (3, 1, 2, 0), (3, 4, 3, 1), (0, 2, 3, 1),
                                  (1, 1, 4, 0)])
def test_packed_kernel_forms_for_ensembles(form):
    """Each packed-tile kernel form (ws, cl, st, keep) pinned for every packed kind
    (for an ensemble the recovery reads the packed tiles too): form 2 serves the
    copies of a subdomain from one CTA (3 members: a group of 4 with one empty
    slot); every member matches its oracle."""
    need_gpu()
    ws, cl, st, keep = form
    w = W.config(1)
    dt = DT["config1"]["dt"]
    n = 30
    sources = member_sources(w, w.dims)

    def pin(fs):
        for kind in ("local", "recover", "iface_rows", "coupled"):   # the recovery is packed for ensembles
            D.dd_set_sym_config(fs.h, kind, cl, st, keep, ws)
        assert set(D.dd_get_sym_config(fs.h)) == {"local", "recover", "iface_rows", "coupled"}

    prm = D.make_params(precision=D.DD_MIXED, tol=1e-5, refine_tol=1e-12, max_refine=8, solver=G, members=3)
    f, stats = run_ensemble(w, dt, n, prm, sources, after_factor=pin)
    assert all(s["status"] == 0 for s in stats)
    for r, (pairs, amp) in enumerate(sources):
        err = rel_err(f[:, r], oracle_member(w, dt, n, pairs, amp))
        assert err[2:].max() <= 1e-8, (form, r, err.max())


def test_silent_member_stays_zero_and_the_other_matches_the_single_problem():
    """A member without source keeps exactly zero fields (the operator is block
    diagonal over members, so its Krylov components stay 0); the other member
    matches the same problem solved alone."""
    need_gpu()
    w = W.config(1)
    dt = DT["config1"]["dt"]
    n = 20
    kw = dict(precision=D.DD_MIXED, tol=1e-5, refine_tol=1e-12, max_refine=8, solver=G)
    f, _ = run_ensemble(w, dt, n, D.make_params(members=2, **kw), [(w.source_pairs, 1.0), (w.source_pairs, 0.0)])
    one, _ = run_ensemble(w, dt, n, D.make_params(**kw), [(w.source_pairs, 1.0)])
    assert not np.any(f[:, 1])
    assert rel_err(f[:, 0], one[:, 0])[2:].max() <= 1e-9


def test_ensemble_rejects_single_problem_features():
    need_gpu()
    w = W.config(1)
    fs = D.FieldSolver(w.xyz, w.tets, w.part, w.n_sub, w.eps, w.mu,
                       D.make_params(solver=G, members=2)).bind()
    fs.factor(DT["config1"]["dt"])
    lam = torch.zeros(fs.n_lambda, dtype=torch.float64, device="cuda")
    with pytest.raises(D.DDError) as e:
        fs.schur_apply(lam)
    assert e.value.code == D.DD_ERR_STATE
    with pytest.raises(D.DDError) as e:
        D.dd_set_probes(fs.h, np.array([[0.3, 0.4, 0.5]]))
    assert e.value.code == D.DD_ERR_STATE
    with pytest.raises(D.DDError) as e:
        fs.set_params(D.make_params(solver=G, members=3))
    assert e.value.code == D.DD_ERR_ARG
    fs.close()


def test_five_members_two_groups():
    """R = 5 with the multi-member form: groups of 4 and 1 copies per CTA; member r
    carries the workload's source at amplitude a_r, so it equals a_r times the
    oracle's unit-source march."""
    need_gpu()
    w = W.config(1)
    dt = DT["config1"]["dt"]
    n = 25
    amps = [1.0, -0.5, 2.0, 0.25, -3.0]
    sources = [(w.source_pairs, a) for a in amps]

    def pin(fs):
        for kind in ("local", "recover", "iface_rows", "coupled"):
            D.dd_set_sym_config(fs.h, kind, 1, 2, 0, 2)

    prm = D.make_params(precision=D.DD_MIXED, tol=1e-5, refine_tol=1e-12, max_refine=8, solver=G, members=5)
    f, stats = run_ensemble(w, dt, n, prm, sources, after_factor=pin)
    assert all(s["status"] == 0 for s in stats)
    ref = oracle_member(w, dt, n, w.source_pairs, 1.0)
    for r, a in enumerate(amps):
        err = rel_err(f[:, r], a * ref)
        assert err[2:].max() <= 1e-8, (r, err.max())


def _pin_tensor_core(fs):
    """The tensor-core form (ws = 4) for the local solve, the recovery and the coupled
    operator; the interface rows keep the CTA-synchronous packed form."""
    for kind in ("local", "recover", "coupled"):
        D.dd_set_sym_config(fs.h, kind, 1, 2, 0, 4)
    D.dd_set_sym_config(fs.h, "iface_rows", 1, 2, 0, 0)
    cfg = D.dd_get_sym_config(fs.h)
    assert all(cfg[k][3] == 4 for k in ("local", "recover", "coupled"))


@pytest.mark.parametrize("amps", [(1.0, -0.5, 2.0), tuple((-1.0) ** r * (1 + r % 5) for r in range(18))])
def test_tensor_core_form_every_member_matches_oracle(amps):
    """tcgen05 form: a CTA applies each BF16x3 operator panel to 16 members by MMA
    (3 members: one group with 13 empty slots; 18 members: groups of 16 and 2);
    member r carries the source at amplitude a_r and equals a_r times the oracle's
    unit-source march to 1e-8 after FP64 refinement."""
    need_gpu()
    w = W.config(1)
    dt = DT["config1"]["dt"]
    n = 25
    sources = [(w.source_pairs, a) for a in amps]
    prm = D.make_params(precision=D.DD_MIXED, tol=1e-5, refine_tol=1e-12, max_refine=8, solver=G,
                        members=len(amps))
    f, stats = run_ensemble(w, dt, n, prm, sources, after_factor=_pin_tensor_core)
    assert all(s["status"] == 0 for s in stats)
    ref = oracle_member(w, dt, n, w.source_pairs, 1.0)
    for r, a in enumerate(amps):
        err = rel_err(f[:, r], a * ref)
        assert err[2:].max() <= 1e-8, (r, err.max())


def test_tensor_core_form_ragged_rcb():
    """tcgen05 form on a jittered mesh with a ragged RCB split (rectangles not
    multiples of the 128 x 64 panel), eps per tet: every member within 1e-8 of its
    oracle march."""
    need_gpu()
    nx, ny, nz = 10, 8, 8
    L = (1.2, 1.0, 1.0)
    xyz, tets = W.kuhn_box(nx, ny, nz, *L)
    xyz, rng = W.jitter_nodes(xyz, L[0] / nx, L, 0.2, seed=9)
    part = W.rcb_partition(W.tet_centroids(xyz, tets), 6, rng.uniform(0.6, 1.4, size=6))
    w = W.Workload("ragged", xyz, tets, part, 6, rng.uniform(1, 4, size=len(tets)), 1.0, 30,
                   W.z_line_node_pairs(nx, ny, nz, 5, 4))
    space = fem.EdgeSpace(xyz, tets, w.eps)
    T, S = space.assemble()
    dt = 2.0 * newmark.cfl_dt(T, S)
    n = 30
    sources = member_sources(w, (nx, ny, nz))[:2]
    prm = D.make_params(precision=D.DD_MIXED, tol=1e-5, refine_tol=1e-12, max_refine=8, solver=G, members=2)
    f, stats = run_ensemble(w, dt, n, prm, sources, after_factor=_pin_tensor_core)
    assert all(s["status"] == 0 for s in stats)
    for r, (pairs, amp) in enumerate(sources):
        err = rel_err(f[:, r], oracle_member(w, dt, n, pairs, amp))
        assert err[2:].max() <= 1e-8, (r, err.max())
