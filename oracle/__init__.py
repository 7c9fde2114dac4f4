"""FP64 CPU oracle for the enriched Taylor--Hood (Q2--Q1*) Stokes/Oseen solvers.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path imports this package:
only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may use it.  It shares no code, constants or helpers with the
CUDA library; both sides receive the same seeded inputs from
``paper_2303_10233_gb300.workloads``, which holds no arithmetic of the method.

Everything here is plain NumPy/SciPy in float64, written from the paper
(Pestana & Silvester, "Fast solution of incompressible flow problems with
two-level pressure approximation"):

* ``fem``      -- Q2 velocity, Q1 + P0 pressure frame (Sec. 2.1, Eq. eth_spec),
                  element matrices by 3x3 Gauss quadrature, CSR assembly of
                  A, N(w), B = [B1; B0], M_Q = [Qk R^T; R Q0] (Sec. 2.3),
                  velocity mass, Q1 mass/Laplacian/convection (Sec. 3.1).
* ``problem``  -- Dirichlet elimination, the saddle systems of Eq.
                  saddle_point (Stokes) and Eq. oseen-system (Oseen), the null
                  vectors of Eq. pressure_null_vector.
* ``direct``   -- bordered sparse direct solve (the exact discrete solution).
* ``krylov``   -- preconditioned MINRES (Algorithm 1), right-preconditioned
                  GMRES(m), the block preconditioners P1 (Sec. 2.4),
                  M_1 (Eq. nse-precon-ref) and Q1 PCD (Eq.
                  discrete-commutator1x), and the two-stage method (Sec. 3.1).
* ``adjoint``  -- adjoint solve and gradients w.r.t. body force and viscosity.
* ``rows``     -- selected entries of K x element by element (no assembly), for
                  sampled parity at full grid sizes.
* ``picard``   -- Picard iteration for steady Navier-Stokes with direct Oseen solves.
* ``lsc``      -- least-squares commutator approximation M_S of the Schur complement for
                  the two-field pressure and the block-triangular M_3 (Sec. 3.2).
* ``step``     -- inflow-outflow flow on a masked uniform grid (the flow over a step,
                  Sec. 3 Test problem 3): natural outflow, null space [0; k] only.
* ``mqcheb``   -- Chebyshev semi-iteration on multicolour symmetric Gauss-Seidel for the
                  singular M_Q (the M_cheb block of the cheaper preconditioner P_2).
* ``infsup``   -- the discrete inf-sup constant gamma^2 (dense pencil, Sec. 2.4) and
                  its EST-MINRES estimate from the Lanczos scalars of MINRES.

Parity pins live in ``tests/test_oracle_*.py``.  Functions with no pin say
"parity unpinned" in their docstring.
"""
