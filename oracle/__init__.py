"""FP64 CPU oracle for the semi-implicit SPH viscous solve (arXiv 2206.14780).

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import, call or link
this package: only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` use it.  It shares no
code with the CUDA library (no kernel, table, constant generator or helper); the
two meet only through the seeded scenes of the ``scenes`` module.

Everything here is plain, slow and in float64, written from the paper:

* ``kernel``     Wendland psi_{3,1} w(q), f(q) and W, F (Sec. 5.2)
* ``neighbors``  the neighbour predicate, brute force O(N^2) and a k-d tree
                 candidate search filtered by the same predicate
* ``operator``   K_ab and the viscous matrix A(dt) for dummy and dynamic walls
                 (Eqs. kab, diag, offdiag, implicit-system-dyn-full,
                 implicit-system-dummy-full), its Jacobi diagonal, A v, the
                 true residual, the row norms of D^-1 A and the closed-form wall-row
                 scale of the diagonal preconditioner-scale head
* ``solvers``    textbook BiCGSTAB, the paper's restructured BiCGSTAB with its
                 per-component state machine (Sec. 4.2), the rotated CG (Sec. 4.1),
                 dense LU and a hand-written Gaussian elimination
* ``rheology``   velocity gradient, strain rate, second invariant and the
                 Papanastasiou viscosity with the truncated series (Sec. 2.4)
* ``mlp``        the warm-start network (forward, loss, backward) in float64,
                 optionally with the bf16 rounding points of the GPU kernels
* ``features``   the sixteen per-particle inputs of that network (shared by the
                 warm start and the preconditioner-scale head)
* ``warmstart``  x0 = v + U y with the dummy-wall closure (Eq. dummyvel), the
                 residual training loss and its MSE pseudo-targets
* ``step``       one semi-implicit predictor/corrector step (Sec. 3.3): Cole's
                 equation of state, the dummy-wall pressure (Eq. dummyP), the
                 inviscid acceleration and continuity, two viscous solves

Readings of the paper where it is garbled or silent:
X1 the kernel gradient factor F enters K_ab as a magnitude, so the fluid rows are
diag 1 + dt sum c, off-diagonal -dt c; X2 the tolerance floor is a max; X4 the
second invariant is D = sqrt(2 g:g); X6 fluid-wall pairs use the fluid row's own
viscosity; X7 a dummy wall row with an empty fluid Shepard sum is an identity row;
X10 the neighbour predicate is the strict d.d < (2h)^2 in float64 on the float32
inputs, with the minimum image on periodic axes.

Parity status: every function is pinned by a test in ``tests/test_oracle_*.py``
against closed forms, invariants, brute force or library routines.  Iteration
counts of the paper's experiments are NOT pinned (different stiffness regime):
parity unpinned for iteration counts only.
"""
from . import kernel, neighbors, operator, solvers, rheology, mlp, features, warmstart, step  # noqa: F401
