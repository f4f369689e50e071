"""CPU oracle for the f-thermostat hot path.

TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and bench.py's CPU
baseline leg may import, call, link or run anything in this package; the library
(paper_1402_2095_gb300) never does, and shares no code with it.  Everything here is
a plain, slow, FP64 restatement of the paper's method:
  native.py / fth_oracle.c   Philox4x32-10 + Box-Muller noise, the FP64 GLE velocity
                             Verlet integrator with block-averaged <x_i x_j>;
  gle.py                     T = exp(-A_p dt/2), S = chol(C_p - T C_p T^T) and the
                             exact stationary covariance of each normal mode of the
                             discretised GLE (discrete Lyapunov), plus the dt -> 0
                             continuous Lyapunov limit and tau_{p^2};
  matfun.py                  f(M) and g(M) by eigendecomposition, Chebyshev route for
                             large sparse lattices;
  fth.py                     OracleFTH, the step-by-step driver.
Parity status: every function above is pinned by tests/test_oracle_*.py against
closed forms, brute force, library routines or published known-answer values; the
fitted-GLE bias against f(M) has no pin in the paper (its parameters are in the
unavailable Supporting Information) and is reported, not asserted ("parity unpinned").
"""
