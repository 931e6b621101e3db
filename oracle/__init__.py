"""CPU oracle for the pivoting-free interior-point method.

TEST INFRASTRUCTURE ONLY. The product (the CUDA library and its Python binding)
never imports, links or calls anything here. Only ``tests/``, the smoke check in
``__graft_entry__`` and the benchmark's CPU-baseline leg use it.

Plain single-threaded FP64 C (``oracle.c``) behind ctypes. Every function
follows the paper's equations step by step:
  - ``analyze``: symbolic analysis with the ordering given (Sec. 2),
  - ``assemble``: the primal condensed matrix of Eq. (5),
  - ``factor`` / ``solve``: left-looking Cholesky without pivoting and
    forward/backward substitution (Sec. 2, "LDL^T Factorization"),
  - ``ipm_lp``: the interior-point method on the LP, KKT conditions (2),
    Newton system (3) condensed to (5),
  - ``factor_ldlt`` / ``solve_ldlt``: LDL^T without pivoting of a
    quasi-definite matrix, and ``forms``: the Newton direction through the
    augmented system (4) and the dual condensed system (6).

Pins (tests/test_oracle_*.py): numpy.linalg.cholesky on dense SPD matrices,
brute-force symbolic factorisation, dense solves of the full Newton system (3),
brute-force vertex enumeration of tiny LPs and scipy's HiGHS on the small LP.
"""
from .oracle import (  # noqa: F401
    OracleSymbolic,
    analyze,
    assemble,
    build,
    factor,
    factor_ldlt,
    ipm_lp,
    k_dense,
    l_dense,
    kmatvec,
    lp_direction,
    lib_path,
    solve,
    solve_ldlt,
)
