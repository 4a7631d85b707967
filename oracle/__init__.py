"""FP64 CPU oracle for the pressure-stress Stokes step (test infrastructure only).

This package is the slow, plain reference that the CUDA path is checked
against.  It is test infrastructure: only the test suite, the smoke check in
``__graft_entry__`` and the ``cpu_baseline`` / ``--impl reference`` legs of
``bench.py`` may import it.  The product path never calls it and shares no
code with it.

Everything here is FP64 numpy/scipy, follows the paper's notation and cites
the passage it implements:

* ``fractions``  -- control-volume fractions W_L, W_F (Section 5, the
  discretization paragraph on volume fractions; estimator of our own choice,
  see the module docstring).
* ``operators``  -- staggered centred-difference operators G (gradient) and
  the reduced deformation operator D (Section 5).
* ``system``     -- weights, null-space elimination (Section 8), the SPD
  pressure-stress matrix (eq. stokesmixedsystemspd), its right-hand side with
  prescribed solid velocities (Section 6.2), the indefinite KKT system
  (eq. stokesmixedsystem) and velocity recovery.
* ``solve``      -- dense Cholesky, sparse direct and Jacobi-PCG solves.
* ``analytic``   -- the closed-form 2D test solutions of Section 9.
* ``unet``       -- CPU FP64 forward/backward of the learned preconditioner.
"""
