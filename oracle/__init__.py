"""Plain, slow CPU FP64 oracle of the ADER-DG element update (TEST INFRASTRUCTURE).

This package is the independent reference the CUDA path is checked against.
It is test infrastructure only: `tests/`, `__graft_entry__.smoke()` and the
`cpu_baseline` / `--impl reference` legs of `bench.py` may import it; the
product library never does, and the product path fails loudly when its CUDA
extension is missing instead of falling back to this code.

It shares no code with the CUDA path (no common kernels, headers, tables or
constant generators).  Everything is written out from the paper
(Krenz et al., SC'21, "3D acoustic-elastic coupling with gravity"):
  * basis and reference operators: Sec. 4.1 (Dubiner basis, B_N = C(N+3,3));
  * Cauchy-Kovalewski predictor and corrector: Sec. 4.1, Eq. (taylor) and the
    time-integrated semi-discrete form, Eq. (semi-discrete-form);
  * Godunov flux with the elastic-acoustic middle state: Sec. 4.2,
    Eqs. (rankine-hugoniot)-(numerical-flux);
  * gravitational free surface and its (eta, H) ODE: Sec. 4.3,
    Eqs. (free-surface-boundary-state)-(coupled-ode-system);
  * CFL condition and rate-2 local time stepping: Sec. 4.4;
  * fault conditions: Sec. 3, Eq. (bc-dynrup).

Readings of points the paper leaves open are listed in each module header.
Pinned by the `-m "not gpu"` tests in tests/test_oracle_*.py.
"""
