"""Pins of the oracle's discrete adjoint (no GPU).

The adjoint gradients are checked against quantities that do not use the
adjoint: central finite differences of the objective computed by forward
solves only, and the closed form dJ/da = 2 J / a (J is quadratic in the source
amplitude because the march is linear in it).
"""
import numpy as np

from oracle import adjoint, fem, newmark
from paper_2204_13254_gb300 import workloads as W


def small_case(seed=3, n=4, steps=30):
    w = W.box(n, n, n, 2, 2, 2, steps=steps, probes=W.PROBES_ADJOINT)
    rng = np.random.default_rng(seed)
    eps = rng.uniform(1.0, 4.0, size=len(w.tets))
    space = fem.EdgeSpace(w.xyz, w.tets, eps)
    T, S = space.assemble()
    dt = 2.0 * newmark.cfl_dt(T, S)
    src = np.zeros(space.n)
    src[space.dof_of_pairs(w.source_pairs)] = 1.0
    P = space.probe_operator(w.probes)
    return w, eps, space, dt, src, P


def J_of(w, eps, dt, src, steps, P, amp=1.0):
    space = fem.EdgeSpace(w.xyz, w.tets, eps)
    T, S = space.assemble()
    return adjoint.objective(P, adjoint.forward_fields(T, S, dt, src, w.d2G(dt, steps), steps, amp))


def test_adjoint_matches_central_differences():
    steps = 30
    w, eps, space, dt, src, P = small_case(steps=steps)
    J, g_eps, g_amp, _ = adjoint.gradients(space, dt, src, w.d2G(dt, steps), steps, P)
    assert J > 0
    rng = np.random.default_rng(0)
    h = 1e-6
    for K in rng.choice(len(eps), size=6, replace=False):
        ep, em = eps.copy(), eps.copy()
        ep[K] += h
        em[K] -= h
        fd = (J_of(w, ep, dt, src, steps, P) - J_of(w, em, dt, src, steps, P)) / (2 * h)
        assert abs(fd - g_eps[K]) <= 1e-5 * np.abs(g_eps).max() + 1e-6 * abs(fd), (K, fd, g_eps[K])


def test_amplitude_gradient_closed_form():
    steps = 30
    w, eps, space, dt, src, P = small_case(steps=steps)
    for amp in (1.0, 0.37):
        J, _, g_amp, _ = adjoint.gradients(space, dt, src, w.d2G(dt, steps), steps, P, amp=amp)
        assert abs(g_amp - 2.0 * J / amp) <= 1e-10 * abs(2.0 * J / amp)


def test_directional_derivative():
    """<dJ/deps, v> equals the central difference of J along a random direction v."""
    steps = 25
    w, eps, space, dt, src, P = small_case(seed=5, steps=steps)
    J, g_eps, _, _ = adjoint.gradients(space, dt, src, w.d2G(dt, steps), steps, P)
    v = np.random.default_rng(1).standard_normal(len(eps))
    h = 1e-6
    fd = (J_of(w, eps + h * v, dt, src, steps, P) - J_of(w, eps - h * v, dt, src, steps, P)) / (2 * h)
    assert abs(fd - g_eps @ v) <= 1e-6 * abs(fd)
