"""High-order self-interaction quadrature (cfg.self_quadrature, the default) on the GPU.

The library adds one 3 ns x 3 ns correction per body to the pair sums (FP32 in FP32
applies, FP64 in FP64 and double-FP32 applies).  The plain product rule stays available
(self_quadrature = 0) and is checked against the plain oracle.  Checked against the oracle's operator
with its independently built correction, against exact two-sphere Stokes flow, and
through complete LCP solves against the corrected oracle's A and b.
"""
import os
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import paper_2604_10089_gb300 as L  # noqa: E402
from oracle.bie import DenseMobility, self_correction  # noqa: E402
from oracle.contacts import contact_matrix, detect_contacts  # noqa: E402
from oracle.lcp import kkt_abs, lcp_data, pgs  # noqa: E402
from oracle.mf import MatrixFreeMobility  # noqa: E402
from workloads import make_instance  # noqa: E402

from .cases import active_set, kkt_bound  # noqa: E402
from .exact_stokes import brenner_approach, jeffery_rotation, stimson_jeffery  # noqa: E402

DEV = "cuda"


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(b), 1e-300))


@pytest.mark.parametrize("precision,tol", [(L.LCP_FP64, 1e-12), (L.LCP_MIXED, 1e-5), (L.LCP_DF64, 1e-12)])
def test_corrected_operator_matches_oracle(precision, tol):
    inst = make_instance("spheres8_grid7x14", 1)
    mob = DenseMobility(inst.centers, inst.n_theta, inst.n_phi, a=inst.radius, self_quadrature=True)
    ctx = L.lcp_setup(L.config_for(inst, self_quadrature=1), inst.centers, inst.axes)
    try:
        phi = np.random.default_rng(3).standard_normal(mob.x.shape[0] * 3)
        out = torch.empty(phi.size, dtype=torch.float64, device=DEV)
        L.lcp_stokes_apply_dev(ctx, torch.tensor(phi, device=DEV), out, precision)
        assert rel(out.cpu().numpy(), (mob.K + mob.P) @ phi) <= tol
    finally:
        L.lcp_destroy(ctx)


@pytest.mark.parametrize("precision,tol", [(L.LCP_FP64, 1e-12), (L.LCP_MIXED, 1e-5), (L.LCP_DF64, 1e-12)])
def test_corrected_operator_many_tiles(precision, tol):
    """64 spheres x 162 nodes (many target blocks, several source splits): the matrix-free
    oracle operator plus the oracle's correction on every body."""
    inst = make_instance("spheres64_grid9x18", 0)
    ctx = L.lcp_setup(L.config_for(inst, self_quadrature=1), inst.centers, None)
    try:
        mf = MatrixFreeMobility(inst.centers, inst.n_theta, inst.n_phi, a=inst.radius)
        C = self_correction(inst.n_theta, inst.n_phi, inst.radius)
        phi = np.random.default_rng(5).standard_normal(mf.x.shape[0] * 3)
        ref = mf.apply_operator(phi) + (phi.reshape(inst.n_bodies, -1) @ C.T).reshape(-1)
        out = torch.empty(phi.size, dtype=torch.float64, device=DEV)
        L.lcp_stokes_apply_dev(ctx, torch.tensor(phi, device=DEV), out, precision)
        assert rel(out.cpu().numpy(), ref) <= tol
    finally:
        L.lcp_destroy(ctx)


@pytest.mark.parametrize("precision", [L.LCP_FP64, L.LCP_MIXED])
@pytest.mark.parametrize("R,bound", [(4.0, 2e-9), (6.0, 1e-10)])
def test_exact_two_sphere_flows_with_self_quadrature(precision, R, bound):
    cfg = L.lcp_default_config(n_theta=11, n_phi=22, radius=1.0, contact_radius=1.25, precision=precision,
                               self_quadrature=1)
    ctx = L.lcp_setup(cfg, np.array([[0.0, 0.0, -R / 2], [0.0, 0.0, R / 2]]))
    try:
        cases = (((2, 8), 1.0, stimson_jeffery(R), 6.0), ((2, 8), -1.0, brenner_approach(R), 6.0),
                 ((5, 11), 1.0, jeffery_rotation(R, same_sense=True), 8.0),
                 ((5, 11), -1.0, jeffery_rotation(R, same_sense=False), 8.0))
        for (i, j), sign, exact, k in cases:
            FT = np.zeros(12)
            FT[i], FT[j] = 1.0, sign
            U = L.mobility_apply(ctx, FT)
            assert abs(1.0 / (k * np.pi * U[i]) - exact) <= bound * exact, (i, sign)
    finally:
        L.lcp_destroy(ctx)


@pytest.mark.parametrize("method", [L.LCP_MONO_PQN, L.LCP_BI_PQN])
@pytest.mark.parametrize("precision", [L.LCP_FP64, L.LCP_MIXED])
def test_lcp_solve_with_self_quadrature_matches_oracle(method, precision):
    inst = make_instance("spheres8_grid7x14", 2)
    mob = DenseMobility(inst.centers, inst.n_theta, inst.n_phi, a=inst.radius, self_quadrature=True)
    pairs, normals, gaps = detect_contacts(inst.centers, inst.contact_radius, inst.delta)
    D = contact_matrix(inst.n_bodies, pairs, normals)
    A, b = lcp_data(D, mob.matrix(), mob.apply(np.zeros(6 * inst.n_bodies), axes=inst.axes), gaps, inst.dt)
    xs = pgs(A, b)
    ctx = L.lcp_setup(L.config_for(inst, precision, self_quadrature=1), inst.centers, inst.axes)
    try:
        assert rel(L.lcp_get_b(ctx), b) <= 1e-9
        x, st, status = L.lcp_solve(ctx, method, inst.tol)
        assert status == L.LCP_OK and st["converged"] == 1
        g = A @ x + b
        g_gpu = L.lcp_apply_A(ctx, x) + L.lcp_get_b(ctx)
        eps_op, _ = kkt_bound(inst.tol, x, g, g_gpu, b, st["hi_mvps"])
        assert kkt_abs(x, g) <= inst.tol + eps_op
        act, amb = active_set(x, g)
        act_ref, amb_ref = active_set(xs, A @ xs + b)
        assert act - amb_ref == act_ref - amb
    finally:
        L.lcp_destroy(ctx)


def test_coarse_low_fidelity_grid_gets_its_own_correction():
    """The coarse grid of Bi-PQN's low fidelity builds the correction of its own template."""
    inst = make_instance("spheres8_grid7x14", 1)
    cfg = L.config_for(inst, L.LCP_MIXED, self_quadrature=1, lowfi_n_theta=5, lowfi_n_phi=10, lowfi_tol=1e-6)
    ctx = L.lcp_setup(cfg, inst.centers, inst.axes)
    try:
        coarse = DenseMobility(inst.centers, 5, 10, a=inst.radius, self_quadrature=True)
        FT = np.random.default_rng(7).standard_normal(6 * inst.n_bodies)
        U = L.mobility_apply(ctx, FT, fidelity=L.LCP_LOW_BIE)
        assert rel(U, coarse.apply(FT)) <= 1e-5
    finally:
        L.lcp_destroy(ctx)


@pytest.mark.parametrize("precision,tol", [(L.LCP_FP64, 1e-12), (L.LCP_MIXED, 1e-5), (L.LCP_DF64, 1e-12)])
def test_plain_product_rule_operator_matches_the_plain_oracle(precision, tol):
    """self_quadrature = 0 (the product rule for the self-interaction, also the operator of
    the allocation-free entry) against the oracle without the correction, and one LCP solve."""
    inst = make_instance("spheres8_grid7x14", 1)
    mob = DenseMobility(inst.centers, inst.n_theta, inst.n_phi, a=inst.radius)
    ctx = L.lcp_setup(L.config_for(inst, self_quadrature=0), inst.centers, inst.axes)
    try:
        phi = np.random.default_rng(4).standard_normal(mob.x.shape[0] * 3)
        out = torch.empty(phi.size, dtype=torch.float64, device=DEV)
        L.lcp_stokes_apply_dev(ctx, torch.tensor(phi, device=DEV), out, precision)
        assert rel(out.cpu().numpy(), (mob.K + mob.P) @ phi) <= tol
        if precision == L.LCP_FP64:
            pairs, normals, gaps = detect_contacts(inst.centers, inst.contact_radius, inst.delta)
            D = contact_matrix(inst.n_bodies, pairs, normals)
            A, b = lcp_data(D, mob.matrix(), mob.apply(np.zeros(6 * inst.n_bodies), axes=inst.axes), gaps,
                            inst.dt)
            x, st, _ = L.lcp_solve(ctx, L.LCP_MONO_PQN, inst.tol)
            g = A @ x + b
            eps_op, _ = kkt_bound(inst.tol, x, g, L.lcp_apply_A(ctx, x) + L.lcp_get_b(ctx), b, st["hi_mvps"])
            assert kkt_abs(x, g) <= inst.tol + eps_op
    finally:
        L.lcp_destroy(ctx)
