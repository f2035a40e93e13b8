"""FP64 CPU oracle for batched nonlinear solves.

TEST INFRASTRUCTURE ONLY: imported by the tests, by the smoke check and by
the benchmark's CPU-baseline leg.  The GPU library and its Python binding
never import it.  See ``nls_oracle.c`` for what it computes and which
passage of the paper each step follows.
"""
from .oracle import (  # noqa: F401
    ALG_NEWTON, ALG_NEWTON_BACKTRACK, ALG_TRUST_DOGLEG,
    ALG_POTRA_PTAK, ALG_HALLEY, ALG_BROYDEN, ALG_MOD_BROYDEN, ALG_TRUST_DOGLEG_NW,
    ST_SUCCESS, ST_MAXITERS, ST_SINGULAR, ST_NONFINITE, ST_LS_FAILED, ST_TR_STALLED,
    build, residual, jacobian, lu_factor, lu_solve, dogleg, solve_one, solve_trace,
    solve_batch, polish, polish_batch, adjoint, hvv, broyden_update,
)
