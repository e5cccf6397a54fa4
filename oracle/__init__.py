"""CPU FP64 oracle for the MFETI-DP1 Maxwell field solve (test infrastructure only).

This package is a plain, slow, obviously-correct restatement of what the
method computes, written from the paper (Crawford et al., "Domain Decomposition
Framework for Maxwell Finite Element Solvers and Application to PIC"):

* ``fem``      -- Whitney 1-form (edge) elements on tetrahedra, PEC edge removal,
                  mass T and curl-curl S assembly, discrete gradient D0, probes
                  (Sec. II-B "Spatial Discretization").
* ``newmark``  -- the implicit Newmark-beta (gamma=1/2, beta=1/4) time march of the
                  edge-element wave equation, solved monolithically by a sparse
                  direct factorisation (Sec. II-B "Temporal Discretization",
                  Eq. maxnmb, edge-only reading); energy and Gauss-law diagnostics.
* ``dd``       -- the MFETI-DP1 tearing, signed/unsigned Boolean maps and the
                  Schur-complement interface solve (Sec. III-A, Eqs. rF1, F1lr,
                  F1uc, f1schur) with real local solves and CG.
* ``adjoint``  -- the discrete adjoint of the Newmark recurrence for gradients of
                  a probe objective (not in the paper; derived from the recurrence).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It shares no code with the CUDA library
and imports nothing from it.
"""
