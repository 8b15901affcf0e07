"""FP64 CPU oracle for the OTLM scaling algorithm.

TEST INFRASTRUCTURE ONLY.  Nothing on the product path imports this package: only `tests/`,
`__graft_entry__.smoke()` and the CPU legs of `bench.py` (`cpu_baseline`, `--impl reference`)
may import or run it.  It shares no code with the CUDA path.
"""
from .otlm import (  # noqa: F401
    DATAFITS, PENALTIES, gibbs_kernel, generalized_kl, lambert_w0, wright_omega,
    prox_datafit, datafit_loss, penalty_value, penalty_term, mm_step, mm_step_log, majorizer_G, prox_objective_V,
    solve, solve_log, solve_converged, solve_log_banded, band_to_dense, primal_objective, dual_objective, objective_and_dual, marginal_violation,
)
