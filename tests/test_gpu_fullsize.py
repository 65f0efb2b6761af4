"""Parity at the benchmark's full size: 216 spheres, 11 x 22 nodes (52 272 nodes).

The dense oracle does not fit at this size; the plain-C matrix-free oracle
checks every output of one operator application, the slip-driven velocities
U_nc (a full FP64 GMRES solve) and, for the mixed Bi-PQN solution computed in
the bench's configuration, the KKT error with the oracle's own MVP A x.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2604_10089_gb300 as L  # noqa: E402
from oracle.contacts import contact_matrix, detect_contacts  # noqa: E402
from oracle.lcp import kkt_abs  # noqa: E402
from oracle.mf import MatrixFreeMobility  # noqa: E402
from workloads import make_instance  # noqa: E402

from .cases import MISMATCH_REL, SELF_QUADRATURE, kkt_bound  # noqa: E402


def rel(a, b):
    return float(np.abs(a - b).max() / np.abs(b).max())


@pytest.fixture(scope="module")
def big():
    inst = make_instance("spheres216_grid11x22", 0)
    mf = MatrixFreeMobility(inst.centers, inst.n_theta, inst.n_phi, a=inst.radius, self_quadrature=SELF_QUADRATURE)
    ctx = L.lcp_setup(L.config_for(inst, L.LCP_MIXED), inst.centers, inst.axes)
    yield inst, mf, ctx
    L.lcp_destroy(ctx)


@pytest.mark.parametrize("precision,tol", [(L.LCP_FP64, 1e-12), (L.LCP_DF64, 1e-12), (L.LCP_MIXED, 1e-4)])
def test_fullsize_operator(big, precision, tol):
    inst, mf, ctx = big
    assert L.lcp_kernel_variant(ctx) in ("sym_p8rc", "sym_p8rc5")   # the symmetric FP32 sum at this size
    phi = np.random.default_rng(21).standard_normal(3 * mf.x.shape[0])
    ref = mf.apply_operator(phi)
    out = torch.empty(phi.size, dtype=torch.float64, device="cuda")
    L.lcp_stokes_apply_dev(ctx, torch.tensor(phi, device="cuda"), out, precision)
    assert rel(out.cpu().numpy(), ref) <= tol


def test_fullsize_slip_velocities_and_lcp_solution(big):
    inst, mf, ctx = big
    U_nc = mf.apply(np.zeros(6 * inst.n_bodies), axes=inst.axes)
    assert rel(L.lcp_get_unc(ctx), U_nc) <= 1e-9
    pairs, normals, gaps = detect_contacts(inst.centers, inst.contact_radius, inst.delta)
    gp, gn, gg = L.lcp_get_contacts(ctx)
    np.testing.assert_array_equal(gp, pairs)
    D = contact_matrix(inst.n_bodies, pairs, normals)
    b = gaps / inst.dt + D.T @ U_nc
    x, st, _ = L.lcp_solve(ctx, L.LCP_BI_PQN, inst.tol)
    assert st["converged"] == 1
    Ax = D.T @ mf.apply(D @ x)          # the oracle's MVP at the GPU's solution
    g_gpu = L.lcp_apply_A(ctx, x, L.LCP_HIGH) + L.lcp_get_b(ctx)
    eps_op, mismatch = kkt_bound(inst.tol, x, Ax + b, g_gpu, b, st["hi_mvps"])
    assert mismatch <= MISMATCH_REL * max(1.0, np.linalg.norm(b)), (eps_op, mismatch)
    assert kkt_abs(x, Ax + b) <= inst.tol + eps_op
    assert np.count_nonzero(x) >= 0.1 * x.size     # a non-trivial LCP


@pytest.mark.parametrize("method", [L.LCP_MONO_PQN, L.LCP_BI_PQN])
@pytest.mark.parametrize("precision", [L.LCP_FP64, L.LCP_MIXED])
def test_c2_solves_against_the_oracle(method, precision):
    """64 spheres (the Mono vs Bi, FP64 vs mixed comparison): each solution's KKT error with
    the matrix-free oracle's MVP and b stays within tol + eps_op."""
    inst = make_instance("spheres64_grid9x18", 0)
    mf = MatrixFreeMobility(inst.centers, inst.n_theta, inst.n_phi, a=inst.radius, self_quadrature=SELF_QUADRATURE)
    pairs, normals, gaps = detect_contacts(inst.centers, inst.contact_radius, inst.delta)
    D = contact_matrix(inst.n_bodies, pairs, normals)
    b_or = gaps / inst.dt + D.T @ mf.apply(np.zeros(6 * inst.n_bodies), axes=inst.axes)
    ctx = L.lcp_setup(L.config_for(inst, precision), inst.centers, inst.axes)
    try:
        x, st, _ = L.lcp_solve(ctx, method, inst.tol)
        assert st["converged"] == 1
        g_gpu = L.lcp_apply_A(ctx, x, L.LCP_HIGH) + L.lcp_get_b(ctx)
    finally:
        L.lcp_destroy(ctx)
    g = D.T @ mf.apply(D @ x) + b_or
    eps_op, mismatch = kkt_bound(inst.tol, x, g, g_gpu, b_or, st["hi_mvps"])
    assert mismatch <= MISMATCH_REL * max(1.0, np.linalg.norm(b_or)), mismatch
    assert kkt_abs(x, g) <= inst.tol + eps_op
