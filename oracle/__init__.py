"""FP64 CPU oracle for differentiable Projective Dynamics (DiffPD, arXiv 2101.05917).

TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
benchmark's CPU-baseline leg may import anything from this package.  It shares
no code with the CUDA path and the CUDA path never calls it.

What it computes is the plain definition of one implicit-Euler step and of
its adjoint (Sec. 3, Eqns 1-12):
  * forward: solve grad g(x) = 0 with g(x) = |x - y|_M^2 / (2 h^2) + E(x) by
    Newton's method with a sparse direct solve and a line search (Eqns 5-7);
  * backward: the full-linearisation adjoint  Hess g(x) z = dL/dx  solved
    directly (Eqns 8-12), and the parameter / state gradients that follow.
The PD energies (Eqns 16-17) and their projections follow the supplement's
energy definitions (corotated, volume-preserving, muscle fibre) and Sec. 5.1
(penalty contact and friction added to f_ext).

Modules:
  mesh         voxel hex mesh, trilinear shape gradients, lumped mass
  projections  projections onto the constraint manifolds and their Jacobians
  model        energy, gradient, Hessian and the PD matrix A
  newton       Newton forward rollout (the reference forward)
  adjoint      full-linearisation backward rollout (the reference gradient)
  pd_cpu       an independent CPU PD + L-BFGS forward (second forward, for
               meshes where Newton is too slow) and the A-preconditioned
               MINRES adjoint that goes with it
  structure    the index structures (incidence CSR, nested dissection,
               supernodes, level sets) re-derived from their definitions

Parity unpinned: no printed trajectory, loss or gradient of the paper is
reproducible (its meshes are not available and its losses are normalised),
so the oracle is pinned by invariants, closed forms, library routines, brute
force and finite differences instead (tests/test_oracle_*.py).
"""
