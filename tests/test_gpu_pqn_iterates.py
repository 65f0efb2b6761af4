"""GPU PQN iterates against the oracle, one iteration at a time.

A converged solution cannot tell a correct quasi-Newton method from any other
convergent one (a prox fed the wrong point still ends at the LCP solution, only
more slowly).  These tests stop the GPU solvers after k iterations (kmax = k)
and compare each truncated iterate x_k with the oracle's Algorithm 1 / 4 under
the same options (scaled B_0, forcing, memory bound), so a wrong direction,
prox, step or secant update shows up at the first iteration it touches.

Tolerance: 1e-8 relative in the max norm.  The GPU's high-fidelity MVP agrees
with the oracle's dense A to ~1e-11, and a CPU experiment that perturbs A by
1e-11 moves every truncated iterate of these instances by at most 3e-11, so
1e-8 leaves room for rounding while any algorithmic difference (a different
direction or step at some iteration) moves x_k by O(1e-2) or more.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2604_10089_gb300 as L  # noqa: E402
from oracle import pqn as P  # noqa: E402

from .cases import dense_case  # noqa: E402

TOL_ITERATE = 1e-8


def rel(a, b):
    return float(np.abs(np.asarray(a) - np.asarray(b)).max() / max(np.abs(np.asarray(b)).max(), 1e-300))


def gpu_truncated(inst, method, k, precision=L.LCP_FP64):
    ctx = L.lcp_setup(L.config_for(inst, precision, kmax=k), inst.centers, inst.axes)
    try:
        x, st, status = L.lcp_solve(ctx, method, inst.tol, allow_not_converged=True)
    finally:
        L.lcp_destroy(ctx)
    return x, st, status


@pytest.mark.parametrize("precision", [L.LCP_FP64, L.LCP_MIXED])
@pytest.mark.parametrize("index", [0, 1, 4])
def test_mono_pqn_iterates_match_oracle(index, precision):
    case = dense_case("spheres8_grid7x14", index)
    inst, A, b = case["inst"], case["A"], case["b"]
    n = b.size
    full = P.mono_pqn(lambda v: A @ v, b, np.zeros(n), tol=inst.tol, scale0=True, r_max=32)
    assert full.converged and full.resets == 0 and full.prox_fallbacks == 0
    for k in range(1, full.iterations + 1):
        ref = P.mono_pqn(lambda v: A @ v, b, np.zeros(n), tol=inst.tol, kmax=k, scale0=True, r_max=32)
        x, st, status = gpu_truncated(inst, L.LCP_MONO_PQN, k, precision)
        assert rel(x, ref.x) <= TOL_ITERATE, (k, rel(x, ref.x))
        assert st["iterations"] == ref.iterations and st["hi_mvps"] == ref.mvps, (k, st, ref.mvps)
        assert st["resets"] == 0 and st["ssn_fallbacks"] == 0, st
        assert (status == L.LCP_OK) == ref.converged
        assert abs(st["kkt_abs"] - ref.kkt) <= 1e-8 * max(1.0, ref.history[0])


@pytest.mark.parametrize("precision", [L.LCP_FP64, L.LCP_MIXED])
@pytest.mark.parametrize("index", [0, 1, 4])
def test_bi_pqn_iterates_match_oracle(index, precision):
    """Algorithm 4 with the RPY low fidelity (which the GPU applies to 1e-13 of
    the oracle): the low-fidelity initialisation, every subproblem, the
    high-fidelity BFGS correction and the secant carry-over all feed x_k."""
    case = dense_case("spheres8_grid7x14", index)
    inst, A, Ahat, b = case["inst"], case["A"], case["Ahat"], case["b"]
    n = b.size
    cfg = L.config_for(inst)

    def oracle(k):
        return P.bi_pqn(lambda v: A @ v, lambda v: Ahat @ v, b, np.zeros(n), tol=inst.tol, kmax=k,
                        kmax_inner=cfg.kmax_inner, forcing=cfg.forcing, r_max=cfg.memory, scale0=True,
                        init_forcing=cfg.init_forcing)

    full = oracle(100)
    assert full.converged and full.resets == 0 and full.prox_fallbacks == 0
    for k in range(1, full.outer_iterations + 1):
        ref = oracle(k)
        x, st, status = gpu_truncated(inst, L.LCP_BI_PQN, k, precision)
        assert rel(x, ref.x) <= TOL_ITERATE, (k, rel(x, ref.x))
        assert st["hi_mvps"] == ref.hi_mvps and st["lo_mvps"] == ref.lo_mvps, (k, st, ref.hi_mvps, ref.lo_mvps)
        assert st["resets"] == 0 and st["ssn_fallbacks"] == 0, st
        assert (status == L.LCP_OK) == ref.converged

