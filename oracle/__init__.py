"""Plain FP64 CPU oracle for the density-fitted GW self-energy.

TEST INFRASTRUCTURE ONLY. Nothing in the product path imports, calls or
links this package: only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may use it. It shares no code with the CUDA
path. Every function restates one passage of the paper (arXiv 2406.18479,
Sec. 2) in float64/complex128 with numpy, one equation at a time, so that it
can be checked against the paper by eye:

  grids.py  Chebyshev tau grid and the tau <-> i Omega transform matrices (Eq. P0t_to_P0w)
  gw.py     P0(tau) (Eq. tilde_P0_tau), P(i Omega) (Eq. tilde_P_omega), Sigma(tau)
            (Eqs. sigma_gw, tilde_W_DF2), the G Dyson equation (Eq. dyson) and mixing,
            the static part (Eq. sigma_inf), the mu search, DIIS/CDIIS and the full loop
  gf2.py    the second-order self-energy (Eq. sigma2)
  kinterp.py  the Wannier-like k-space interpolation (Sec. 2.5)
  ir.py     intermediate-representation tau grids and transforms (the paper's Lambda = 1e4 grids)

Parity status: every function is pinned (tests/test_oracle_pins.py,
tests/test_oracle_loop_pins.py, tests/test_oracle_gf2_pins.py,
tests/test_oracle_kinterp_pins.py, tests/test_oracle_ir_pins.py) against
closed forms, brute force with 4-index integrals, the pole-pair sum and
invariants. No function is "parity unpinned".
"""
