"""Warm starts along a trajectory (lcp_step).

The slip-driven density of the U_nc solve changes little over one time step,
so starting GMRES from the previous step's density reaches the same tolerance
in fewer iterations.  The next LCP's b must not change: it is compared with a
cold-started run at every step and with the oracle after the first step.  The
next LCP solve starts from the previous step's forces on the contacts whose
body pairs persist: checked against a start built here by matching the pairs,
and against the oracle's KKT error at the advanced configuration.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2604_10089_gb300 as L  # noqa: E402
from oracle.bie import DenseMobility  # noqa: E402
from oracle.contacts import contact_matrix, detect_contacts  # noqa: E402
from oracle.lcp import lcp_data  # noqa: E402
from workloads import make_instance  # noqa: E402

from .cases import SELF_QUADRATURE, dense_case, kkt_bound  # noqa: E402


def rel(a, b):
    return float(np.abs(np.asarray(a) - np.asarray(b)).max() / max(np.abs(np.asarray(b)).max(), 1e-300))


def _rotate(e, w, dt):
    th = np.linalg.norm(w) * dt
    if th == 0.0:
        return e
    k = w / np.linalg.norm(w)
    out = e * np.cos(th) + np.cross(k, e) * np.sin(th) + k * (k @ e) * (1 - np.cos(th))
    return out / np.linalg.norm(out)


@pytest.mark.parametrize("precision", [L.LCP_FP64, L.LCP_MIXED])
def test_warm_started_slip_solve_same_b_fewer_iterations(precision):
    inst = make_instance("spheres8_grid7x14", 2)
    warm = L.lcp_setup(L.config_for(inst, precision, warm_start=L.LCP_WARM_SLIP), inst.centers, inst.axes)
    cold = L.lcp_setup(L.config_for(inst, precision, warm_start=0), inst.centers, inst.axes)
    try:
        its_w, its_c = [], []
        for step in range(4):
            # both LCPs from x = 0, so that only the slip solve's start differs
            n = L.lcp_sizes(warm)[2]
            xw, sw, _ = L.lcp_solve(warm, L.LCP_MONO_PQN, inst.tol, x0=np.zeros(n))
            xc, sc, _ = L.lcp_solve(cold, L.LCP_MONO_PQN, inst.tol, x0=np.zeros(n))
            assert sw["converged"] == 1 and sc["converged"] == 1
            assert sw["unc_warm_started"] == (1 if step > 0 else 0) and sc["unc_warm_started"] == 0
            if step > 0:
                its_w.append(sw["unc_gmres_iterations"])
                its_c.append(sc["unc_gmres_iterations"])
            np.testing.assert_allclose(xw, xc, atol=1e-7 * max(1.0, np.abs(xc).max()))
            L.lcp_step(warm, inst.dt)
            L.lcp_step(cold, inst.dt)
            assert rel(L.lcp_get_b(warm), L.lcp_get_b(cold)) <= 1e-10
            assert rel(L.lcp_get_unc(warm), L.lcp_get_unc(cold)) <= 1e-10
        n = L.lcp_sizes(warm)[2]
        _, sw, _ = L.lcp_solve(warm, L.LCP_MONO_PQN, inst.tol, x0=np.zeros(n))
        _, sc, _ = L.lcp_solve(cold, L.LCP_MONO_PQN, inst.tol, x0=np.zeros(n))
        its_w.append(sw["unc_gmres_iterations"])
        its_c.append(sc["unc_gmres_iterations"])
        assert all(w > 0 for w in its_w)
        assert sum(its_w) < sum(its_c), (its_w, its_c)
    finally:
        L.lcp_destroy(warm)
        L.lcp_destroy(cold)


def test_warm_started_step_matches_oracle():
    """Eq. (dvi) with the warm-started slip solve: the next b against the oracle."""
    case = dense_case("spheres8_grid7x14", 4)
    inst = case["inst"]
    ctx = L.lcp_setup(L.config_for(inst, L.LCP_MIXED, warm_start=L.LCP_WARM_SLIP), inst.centers, inst.axes)
    try:
        x, _, _ = L.lcp_solve(ctx, L.LCP_MONO_PQN, inst.tol)
        c_new, a_new = L.lcp_step(ctx, inst.dt)
        U = (case["U_nc"] + case["Mob"] @ (case["D"] @ x)).reshape(-1, 6)
        c_ref = inst.centers + inst.dt * U[:, :3]
        a_ref = np.array([_rotate(inst.axes[i], U[i, 3:], inst.dt) for i in range(inst.n_bodies)])
        mob = DenseMobility(c_ref, inst.n_theta, inst.n_phi, a=inst.radius, self_quadrature=SELF_QUADRATURE)
        pairs, normals, gaps = detect_contacts(c_ref, inst.contact_radius, inst.delta)
        D = contact_matrix(inst.n_bodies, pairs, normals)
        u_nc = mob.apply(np.zeros(6 * inst.n_bodies), axes=a_ref)
        _, b_next = lcp_data(D, np.eye(6 * inst.n_bodies), u_nc, gaps, inst.dt)
        _, st, _ = L.lcp_solve(ctx, L.LCP_MONO_PQN, inst.tol)
        assert st["unc_warm_started"] == 1
        assert rel(L.lcp_get_unc(ctx), u_nc) <= 1e-9
        assert rel(L.lcp_get_b(ctx), b_next) <= 1e-9
    finally:
        L.lcp_destroy(ctx)


def carried(x, pairs_prev, pairs_next):
    """The previous forces on the next contacts, matched by body pair (0 for new pairs)."""
    prev = {}
    for l, (i, j) in enumerate(map(tuple, pairs_prev)):
        prev.setdefault((int(i), int(j)), x[l])
    return np.array([prev.get((int(i), int(j)), 0.0) for i, j in pairs_next])


@pytest.mark.parametrize("method", [L.LCP_MONO_PQN, L.LCP_BI_PQN])
def test_lcp_warm_start_carries_forces_by_body_pair(method):
    """After lcp_step the next solve starts from the previous forces on persisting pairs:
    bitwise the same solve as one started from that x0 built here."""
    inst = make_instance("spheres8_grid7x14", 3)
    ctx = L.lcp_setup(L.config_for(inst, L.LCP_MIXED, warm_start=L.LCP_WARM_FORCES), inst.centers, inst.axes)
    try:
        x, st, _ = L.lcp_solve(ctx, method, inst.tol)
        assert st["warm_x0"] == 0
        kept = new = 0
        for step in range(3):
            pairs_prev = L.lcp_get_contacts(ctx)[0]
            L.lcp_step(ctx, inst.dt)
            pairs = L.lcp_get_contacts(ctx)[0]
            x0 = carried(x, pairs_prev, pairs)
            xa, sa, _ = L.lcp_solve(ctx, method, inst.tol)            # carried start
            xb, sb, _ = L.lcp_solve(ctx, method, inst.tol, x0=x0)     # the same start, given
            assert sa["warm_x0"] == 1 and sb["warm_x0"] == 0
            assert sa["converged"] == 1
            assert np.array_equal(xa, xb)
            kept += int(np.count_nonzero(x0))
            new += int(x0.size - np.count_nonzero(x0))
            x = xa
        assert kept > 0
        # an update to an arbitrary configuration starts from zero again
        L.lcp_update(ctx, inst.centers, inst.axes)
        _, sc, _ = L.lcp_solve(ctx, method, inst.tol)
        assert sc["warm_x0"] == 0
    finally:
        L.lcp_destroy(ctx)


@pytest.mark.parametrize("flags", [L.LCP_WARM_SLIP | L.LCP_WARM_FORCES, L.LCP_WARM_FORCES | L.LCP_WARM_NO_INIT])
def test_lcp_warm_started_trajectory_matches_oracle(flags):
    """Three warm-started steps (with Bi-PQN's low-fidelity initialisation, or with the
    carried forces taken as x(0) directly): each solution's KKT error against the
    oracle's dense A and b at the advanced configuration."""
    inst = make_instance("spheres8_grid7x14", 4)
    warm = L.lcp_setup(L.config_for(inst, L.LCP_MIXED, warm_start=flags), inst.centers, inst.axes)
    cold = L.lcp_setup(L.config_for(inst, L.LCP_MIXED, warm_start=0), inst.centers, inst.axes)
    try:
        L.lcp_solve(warm, L.LCP_BI_PQN, inst.tol)
        L.lcp_solve(cold, L.LCP_BI_PQN, inst.tol)
        for step in range(3):
            c, a = L.lcp_step(warm, inst.dt)
            L.lcp_step(cold, inst.dt)
            x, st, _ = L.lcp_solve(warm, L.LCP_BI_PQN, inst.tol)
            _, sc, _ = L.lcp_solve(cold, L.LCP_BI_PQN, inst.tol)
            assert st["warm_x0"] == 1 and sc["warm_x0"] == 0
            mob = DenseMobility(c, inst.n_theta, inst.n_phi, a=inst.radius, self_quadrature=SELF_QUADRATURE)
            pairs, normals, gaps = detect_contacts(c, inst.contact_radius, inst.delta)
            assert np.array_equal(pairs, L.lcp_get_contacts(warm)[0])
            D = contact_matrix(inst.n_bodies, pairs, normals)
            A, b = lcp_data(D, mob.matrix(), mob.apply(np.zeros(6 * inst.n_bodies), axes=a), gaps, inst.dt)
            g = A @ x + b
            g_gpu = L.lcp_apply_A(warm, x) + L.lcp_get_b(warm)
            eps_op, _ = kkt_bound(inst.tol, x, g, g_gpu, b, st["hi_mvps"])
            assert np.linalg.norm(np.minimum(x, g)) <= inst.tol + eps_op
    finally:
        L.lcp_destroy(warm)
        L.lcp_destroy(cold)
