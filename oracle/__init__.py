"""CPU oracle for the element-based convex limited CG-WENO stage.

TEST INFRASTRUCTURE ONLY: a plain, slow FP64 implementation written from
the paper (Kuzmin, Hajduk, Vedral, arXiv 2509.04673).  Only tests/,
__graft_entry__.smoke() and the cpu_baseline / reference legs of bench.py
may import it.  It shares no code with the CUDA path: the library never
imports, links or calls anything here.

Parity status per function (what pins it, tests/test_oracle_*.py):
  tables.tables          exact rationals; pinned by partition of unity,
                         closed-form mass entries, derivative identities
  physics.flux           Euler: Rankine-Hugoniot on exact normal shocks,
                         Jacobian eigenvalues and the textbook Jacobian;
                         KPP: the speed of a small perturbation
  physics.max_speed      an upper bound of the exact Riemann speeds
  scheme.cell_averages   quadrature mean of u_h; conservation; LO identity
  scheme.low_order_facets, pseudo_time_steps
                         pinned by the LO finite-volume identity and IDP
  scheme.high_order_facets
                         face mean of the group flux by quadrature
  scheme.sensor          pinned by special cases (constant, linear and
                         polynomial data give gamma = 1) and a brute-force
                         semi-norm; the candidate construction is a reading
                         (parity of the exact gamma_e values unpinned)
  scheme.gradient_projection
                         pinned against a dense consistent-mass solve
  scheme.element_residual, fe_stage
                         pinned by brute-force global assembly (Theorem of
                         Sec. 4: MCL with alpha = beta = 1 equals CG-WENO),
                         the weak form against a strong-form assembly for
                         the nonlinear fluxes, f_i^e from eq. (aec) by
                         quadrature, zero-sum, conservation, free stream,
                         dt_e independence and the p+1 convergence rate
  scheme.flux_limit, slope_limit
                         pinned by IDP invariants, maximality, closed forms
  scheme.euler_alpha     admissibility and maximality derived from the
                         definition of the limited state
  scheme.subcell_time_steps, aec_q1, reduced_time_steps, boundary data
                         pinned by closed forms and invariants in their
                         own test files
  tables.lgl_points, lgl_tables, and the LGL basis of OracleMesh (basis 1:
  Lagrange at the Lobatto points, m_i^e = |K| w_a w_b, face weights w_a)
                         closed-form Lobatto points and weights, exactness
                         to degree 2p - 1, tables against the independent
                         product formula, Q1 equal to Bernstein Q1, u^e,
                         f^H and f_i^e by brute force, conservation, free
                         stream, invariant domain, optimal HO rate
"""
