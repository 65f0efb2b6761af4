"""Reuse across the mobility solves of one configuration (cfg.recycle, Fischer's
projection for successive right-hand sides; the paper names reuse across solves
as future work).  Where the right-hand sides are close (a repeated force, a
multiple, a small perturbation) a projected start is taken, the result is the
same mobility to the GMRES tolerance (the oracle's dense mobility decides), and
fewer GMRES iterations reach it.  Where they are not (the search directions of a
PQN solve), the start falls back to zero and the LCP result is unchanged."""
import os
import sys

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import paper_2604_10089_gb300 as L  # noqa: E402
from oracle.bie import DenseMobility  # noqa: E402

from .cases import SELF_QUADRATURE, dense_case, kkt_bound  # noqa: E402


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(b), 1e-300))


def force_sequence(M, seed=7):
    """A force, its double, a 1e-4 perturbation of it, then an unrelated force."""
    rng = np.random.default_rng(seed)
    F = rng.standard_normal(6 * M)
    return [F, 2.0 * F, F + 1e-4 * rng.standard_normal(6 * M), rng.standard_normal(6 * M)]


def solve_sequence(ctx, seq, fidelity=L.LCP_HIGH):
    out, its, rec = [], [], []
    for F in seq:
        s0, g0, r0 = L.lcp_solve_counters(ctx, fidelity)
        out.append(L.mobility_apply(ctx, F, fidelity=fidelity))
        s1, g1, r1 = L.lcp_solve_counters(ctx, fidelity)
        assert s1 == s0 + 1
        its.append(g1 - g0)
        rec.append(r1 - r0)
    return out, its, rec


@pytest.mark.parametrize("precision", [L.LCP_FP64, L.LCP_MIXED])
def test_projected_start_same_mobility_fewer_iterations(precision):
    case = dense_case("spheres8_grid7x14", 0)
    inst, Mob = case["inst"], case["Mob"]
    seq = force_sequence(inst.n_bodies)
    on = L.lcp_setup(L.config_for(inst, precision, recycle=8), inst.centers, inst.axes)
    off = L.lcp_setup(L.config_for(inst, precision, recycle=0), inst.centers, inst.axes)
    try:
        U_on, its_on, rec_on = solve_sequence(on, seq)
        U_off, its_off, rec_off = solve_sequence(off, seq)
        assert rec_off == [0, 0, 0, 0]
        # the double and the perturbation start from the projection, the unrelated force does not
        assert rec_on[1] == 1 and rec_on[2] == 1 and rec_on[3] == 0, rec_on
        assert its_on[1] < its_off[1] and its_on[2] < its_off[2], (its_on, its_off)
        for F, a, b in zip(seq, U_on, U_off):
            expect = Mob @ F
            assert rel(a, expect) <= 1e-9 and rel(b, expect) <= 1e-9
            assert rel(a, b) <= 1e-10
    finally:
        L.lcp_destroy(on)
        L.lcp_destroy(off)


def test_projected_start_on_the_low_fidelity_grid():
    """FP32-only GMRES of the coarse grid: the exact start residual is taken with the
    FP32 operator, and the result matches the coarse grid's dense oracle mobility to
    the low-fidelity tolerance."""
    case = dense_case("spheres8_grid7x14", 0)
    inst = case["inst"]
    lo = dict(lowfi_n_theta=5, lowfi_n_phi=10, lowfi_tol=1e-6)
    Mlo = DenseMobility(inst.centers, 5, 10, a=inst.radius, mu=inst.viscosity, self_quadrature=SELF_QUADRATURE).matrix()
    seq = force_sequence(inst.n_bodies, seed=11)
    on = L.lcp_setup(L.config_for(inst, L.LCP_MIXED, recycle=4, **lo), inst.centers, inst.axes)
    off = L.lcp_setup(L.config_for(inst, L.LCP_MIXED, recycle=0, **lo), inst.centers, inst.axes)
    try:
        U_on, its_on, rec_on = solve_sequence(on, seq, L.LCP_LOW_BIE)
        U_off, its_off, rec_off = solve_sequence(off, seq, L.LCP_LOW_BIE)
        assert rec_off == [0, 0, 0, 0] and rec_on[1] == 1 and rec_on[2] == 1 and rec_on[3] == 0, rec_on
        assert its_on[1] < its_off[1] and its_on[2] < its_off[2], (its_on, its_off)
        for F, a, b in zip(seq, U_on, U_off):
            assert rel(a, Mlo @ F) <= 1e-5 and rel(b, Mlo @ F) <= 1e-5
    finally:
        L.lcp_destroy(on)
        L.lcp_destroy(off)


def test_full_set_restarts_and_stays_correct():
    """Three kept pairs and two alternating forces (scaled, perturbed): the set fills
    (the slip solve of the set-up is its first pair), restarts from the newest
    solve, and keeps projecting; every result matches the oracle."""
    case = dense_case("spheres8_grid7x14", 2)
    inst, Mob = case["inst"], case["Mob"]
    rng = np.random.default_rng(5)
    base = rng.standard_normal((2, 6 * inst.n_bodies))
    ctx = L.lcp_setup(L.config_for(inst, L.LCP_MIXED, recycle=3), inst.centers, inst.axes)
    try:
        rec = []
        for k in range(8):
            F = base[k % 2] * (1.0 + 0.1 * k) + 1e-6 * rng.standard_normal(6 * inst.n_bodies)
            r0 = L.lcp_solve_counters(ctx)[2]
            assert rel(L.mobility_apply(ctx, F), Mob @ F) <= 1e-9, k
            rec.append(L.lcp_solve_counters(ctx)[2] - r0)
        # cold: the first of each force; projected: every later one (the restart keeps the newest
        # solution, whose force the next-but-one solve repeats up to scale and noise)
        assert rec[0] == 0 and rec[1] == 0 and sum(rec) >= 4, rec
    finally:
        L.lcp_destroy(ctx)


@pytest.mark.parametrize("method", [L.LCP_MONO_PQN, L.LCP_BI_PQN])
def test_lcp_solve_with_recycling_matches_the_oracle(method):
    case = dense_case("spheres8_grid7x14", 1)
    inst, A, b = case["inst"], case["A"], case["b"]
    ctx = L.lcp_setup(L.config_for(inst, L.LCP_MIXED, recycle=8), inst.centers, inst.axes)
    try:
        x, st, _ = L.lcp_solve(ctx, method, inst.tol)
        g_gpu = L.lcp_apply_A(ctx, x) + L.lcp_get_b(ctx)
        g = A @ x + b
        eps_op, _ = kkt_bound(inst.tol, x, g, g_gpu, b, st["hi_mvps"])
        assert np.linalg.norm(np.minimum(x, g)) <= inst.tol + eps_op
        assert st["converged"] == 1
    finally:
        L.lcp_destroy(ctx)
