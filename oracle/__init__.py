"""CPU oracle for the JFNK + physics-based-preconditioning hot path.

TEST INFRASTRUCTURE ONLY.  This package is a plain, slow, float64 restatement
of the method of Viallet et al. (A&A, "A Jacobian-free Newton-Krylov method
for time-implicit multidimensional hydrodynamics"), written with PyTorch CPU
tensor operations.  Only the test suite, the smoke check of the package entry
point and the benchmark's CPU-baseline / reference arms may import it.  The
CUDA library never calls it, and it shares no code with the CUDA library: the
only common module is the seeded input generator `workloads`.

Modules
  discretization  Sect. 2: EOS, conserved variables U(X), the finite-volume
                  right-hand side R_U(X) on the staggered grid, and the
                  Crank-Nicolson residual F_U(X) (Eq. crank_nicholson).
  jfnk            Sect. 4.1-4.2: scaling L, R (Eq. jacobian_system_norm), the
                  finite-difference Jacobian-vector product (Eqs.
                  jacobian_free, pert_old, pert_new), right-preconditioned
                  GMRES (Eq. forcing_term, lin_sys_rp) and the Newton loop
                  (Eq. nr_terminate).
  precond         Sects. 3.2-3.4 and 4.3: transformation matrices dV/dU,
                  dX/dV (App. B), the semi-implicit sound-wave and
                  sound-wave + thermal-diffusion systems in delta form, a
                  geometric multigrid V-cycle for them and a sparse direct
                  solve used as the exact reference.
  adjoint         Gradients through one implicit step: vector-Jacobian
                  products of the residual (reverse-mode derivatives of the
                  discretisation above) and the transposed Newton-system solve.

Readings of points the paper leaves open are stated where they are used.
"""

