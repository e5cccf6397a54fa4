"""Pins of the oracle's Newmark time march (no GPU).

The recurrence A e^{n+1} = B e^n - A e^{n-1} - d2g (Sec. II-B, Eq. maxnmb,
edge-only reading) is checked against: a dense brute-force solve, its exact
quadratic energy invariant once the source is off (unconditional stability at
dt = 2 x the explicit limit), the discrete Gauss law D0^T (T e^n + g^n) = 0
that the integrated-current source guarantees (Sec. II-A), and the resonance
of the PEC cavity seen in the probe spectrum.
"""
import json
import os

import numpy as np
import pytest

from oracle import fem, newmark
from paper_2204_13254_gb300 import workloads as W

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def setup(w, dt=None):
    space = fem.EdgeSpace(w.xyz, w.tets, w.eps, w.mu)
    T, S = space.assemble()
    if dt is None:
        dt = 2.0 * newmark.cfl_dt(T, S)
    src = np.zeros(space.n)
    src[space.dof_of_pairs(w.source_pairs)] = 1.0
    return space, T, S, dt, src


@pytest.mark.parametrize("n", [2, 3, 4])
def test_dense_bruteforce_matches_sparse(n):
    w = W.cavity(n, 1, steps=30) if n % 2 == 0 else W.box(n, n, n, 1, 1, 1, src_ij=(1, 1), steps=30)
    space, T, S, dt, src = setup(w)
    d2g = w.d2G(dt, 30)
    a = newmark.run(T, S, dt, src, d2g, 30, keep=True)
    b = newmark.run(T, S, dt, src, d2g, 30, keep=True, dense=True)
    scale = np.abs(a["fields"]).max()
    assert scale > 0
    assert np.abs(a["fields"] - b["fields"]).max() <= 1e-13 * scale
    # the march really solves the recurrence
    f = a["fields"]
    for k in range(2, 30):
        r, sc = newmark.step_residual(T, S, dt, f[k], f[k - 1], f[k - 2], d2g[k] * src)
        assert np.linalg.norm(r) <= 1e-13 * sc


def test_energy_invariant_and_stability():
    w = W.config(1)
    dt = json.load(open(os.path.join(GOLD, "cfl_dt.json")))["config1"]["dt"]
    space, T, S, dt, src = setup(w, dt)
    n = 200
    out = newmark.run(T, S, dt, src, w.d2G(dt, n), n, keep=True)
    f = out["fields"]
    # source is off to double precision after t0 + 10 sigma = 80 dt (exp(-50) ~ 2e-22)
    Wn = np.array([newmark.energy(T, S, dt, f[k + 1], f[k]) for k in range(81, n - 1)])
    assert Wn[0] > 0
    assert np.abs(Wn / Wn[0] - 1).max() < 1e-12
    assert np.isfinite(f).all()


def test_gauss_law_with_open_line_current():
    """A current segment ending inside the cavity deposits charge at its ends;
    D0^T (T e^n + g^n) stays zero to round-off (charge conservation)."""
    w = W.cavity(6, 1)
    space, T, S, dt, src = setup(w)
    pairs = w.source_pairs[2:4]           # z-edges k=2..3 only: endpoints are interior nodes
    src = np.zeros(space.n)
    src[space.dof_of_pairs(pairs)] = 1.0
    D0 = space.gradient_matrix()
    assert np.abs(D0.T @ src).max() == 1.0   # the segment has two charged ends
    n = 120
    G = w.G_at_steps(dt, n)[1:]              # G^0 .. G^n
    out = newmark.run(T, S, dt, src, w.d2G(dt, n), n, keep=True)
    f = out["fields"]
    worst = 0.0
    for k in range(n):
        r = D0.T @ (T @ f[k] + G[k + 1] * src)
        worst = max(worst, np.abs(r).max() / max(np.abs(T @ f[k]).max(), 1e-300))
    assert worst < 1e-11


def test_cavity_probe_spectrum():
    """The probe signal peaks at the Newmark-dispersed FEM frequency of the TM110 mode,
    and within discretisation error of the analytic f = sqrt(2)/2."""
    import scipy.linalg as sla
    w = W.config(1)
    dt = json.load(open(os.path.join(GOLD, "cfl_dt.json")))["config1"]["dt"]
    space, T, S, dt, src = setup(w, dt)
    n = 200
    P = space.probe_operator(w.probes)
    out = newmark.run(T, S, dt, src, w.d2G(dt, n), n, P=P)
    sig = out["probes"][:, 2]
    pad = 16 * n
    spec = np.abs(np.fft.rfft(sig * np.hanning(n), pad))
    freqs = np.fft.rfftfreq(pad, dt)
    k = int(np.argmax(spec))
    y0, y1, y2 = spec[k - 1], spec[k], spec[k + 1]
    f_peak = freqs[k] + 0.5 * (y0 - y2) / (y0 - 2 * y1 + y2) * (freqs[1] - freqs[0])
    lam, vec = sla.eigh(S.toarray(), T.toarray())
    nz = lam > 1e-8 * lam.max()
    overlap = np.abs(vec[:, nz].T @ src)
    # lowest mode the z-line source excites (TE modes of the (1,1,0) triplet have E_z ~ 0)
    om_h = np.sqrt(lam[nz][overlap > 1e-6 * overlap.max()].min())
    f_d = (2.0 / dt) * np.arctan(om_h * dt / 2.0) / (2 * np.pi)
    assert abs(f_peak - f_d) < 0.05 / (n * dt)
    assert abs(f_peak - np.sqrt(2) / 2) < 0.05 * np.sqrt(2) / 2
