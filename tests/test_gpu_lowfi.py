"""The coarse-grid boundary-integral low-fidelity operator (Sec. 5.1: fidelity
by the coarseness of the discretisation) against the oracle, and Bi-PQN with
it: the solution must be the high-fidelity one (the low fidelity only changes
the path, Algorithm 4).

Tolerances: the low-fidelity mobility is solved with FP32 sums to a relative
GMRES residual lowfi_tol = 1e-6 (the paper's low-fidelity eps_gmres), so its
MVP matches the oracle's coarse-grid operator to ~1e-6 relative (checked at
1e-5); the LCP solution is checked like every other solve (same active set as
the oracle, KKT with the oracle's A at most 10 tol).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2604_10089_gb300 as L  # noqa: E402
from oracle.bie import DenseMobility  # noqa: E402
from oracle.contacts import contact_matrix, detect_contacts  # noqa: E402
from oracle.lcp import kkt_abs  # noqa: E402
from oracle.mf import MatrixFreeMobility  # noqa: E402
from workloads import make_instance  # noqa: E402

from .cases import MISMATCH_REL, SELF_QUADRATURE, active_set, dense_case, kkt_bound  # noqa: E402


def rel(a, b):
    return float(np.abs(np.asarray(a) - np.asarray(b)).max() / max(np.abs(np.asarray(b)).max(), 1e-300))


@pytest.mark.parametrize("grid", [(5, 10), (6, 12)])
def test_lowfi_mvp_matches_coarse_grid_oracle(grid):
    case = dense_case("spheres8_grid7x14", 1)
    inst = case["inst"]
    coarse = DenseMobility(inst.centers, grid[0], grid[1], a=inst.radius, mu=inst.viscosity, self_quadrature=SELF_QUADRATURE)
    A_lo = case["D"].T @ coarse.matrix() @ case["D"]
    cfg = L.config_for(inst, L.LCP_MIXED, lowfi_n_theta=grid[0], lowfi_n_phi=grid[1], lowfi_tol=1e-6)
    ctx = L.lcp_setup(cfg, inst.centers, inst.axes)
    try:
        x = np.abs(np.random.default_rng(2).standard_normal(case["b"].size))
        assert rel(L.lcp_apply_A(ctx, x, L.LCP_LOW_BIE), A_lo @ x) <= 1e-5
        # the RPY operator stays available beside it
        assert rel(L.lcp_apply_A(ctx, x, L.LCP_LOW_RPY), case["Ahat"] @ x) <= 1e-12
        # mobility of the coarse grid, U = M F
        FT = np.random.default_rng(3).standard_normal(6 * inst.n_bodies)
        assert rel(L.mobility_apply(ctx, FT, fidelity=L.LCP_LOW_BIE), coarse.apply(FT)) <= 1e-5
    finally:
        L.lcp_destroy(ctx)


@pytest.mark.parametrize("init_forcing", [0.0, 1e-3])
@pytest.mark.parametrize("index", [0, 1, 2])
def test_bi_pqn_with_coarse_grid_low_fidelity(index, init_forcing):
    case = dense_case("spheres8_grid7x14", index)
    inst = case["inst"]
    A, b, xs = case["A"], case["b"], case["x"]
    cfg = L.config_for(inst, L.LCP_MIXED, lowfi_n_theta=5, lowfi_n_phi=10, init_forcing=init_forcing)
    ctx = L.lcp_setup(cfg, inst.centers, inst.axes)
    try:
        x, st, status = L.lcp_solve(ctx, L.LCP_BI_PQN, inst.tol)
        assert status == L.LCP_OK and st["converged"] == 1 and st["lo_mvps"] >= 1
        g = A @ x + b
        g_gpu = L.lcp_apply_A(ctx, x, L.LCP_HIGH) + L.lcp_get_b(ctx)
        eps_op, mismatch = kkt_bound(inst.tol, x, g, g_gpu, b, st["hi_mvps"])
        assert mismatch <= MISMATCH_REL * max(1.0, np.linalg.norm(b)), mismatch
        assert kkt_abs(x, g) <= inst.tol + eps_op
        act, amb = active_set(x, g)
        act_ref, amb_ref = active_set(xs, A @ xs + b)
        assert act - amb_ref == act_ref - amb
    finally:
        L.lcp_destroy(ctx)


def test_bi_pqn_coarse_low_fidelity_64_spheres():
    """Fewer high-fidelity MVPs than with RPY, same solution (oracle MVP at the result)."""
    inst = make_instance("spheres64_grid9x18", 0)
    mf = MatrixFreeMobility(inst.centers, inst.n_theta, inst.n_phi, a=inst.radius, self_quadrature=SELF_QUADRATURE)
    pairs, normals, gaps = detect_contacts(inst.centers, inst.contact_radius, inst.delta)
    D = contact_matrix(inst.n_bodies, pairs, normals)
    res = {}
    for name, kw in (("rpy", {}), ("bie", dict(lowfi_n_theta=6, lowfi_n_phi=12))):
        ctx = L.lcp_setup(L.config_for(inst, L.LCP_MIXED, **kw), inst.centers, inst.axes)
        try:
            x, st, _ = L.lcp_solve(ctx, L.LCP_BI_PQN, inst.tol)
            assert st["converged"] == 1
            b = L.lcp_get_b(ctx)
            res[name] = (x, st, L.lcp_apply_A(ctx, x, L.LCP_HIGH) + b)
        finally:
            L.lcp_destroy(ctx)
    x, st, g_gpu = res["bie"]
    b_or = gaps / inst.dt + D.T @ mf.apply(np.zeros(6 * inst.n_bodies), axes=inst.axes)
    g = D.T @ mf.apply(D @ x) + b_or
    eps_op, mismatch = kkt_bound(inst.tol, x, g, g_gpu, b_or, st["hi_mvps"])
    assert mismatch <= MISMATCH_REL * max(1.0, np.linalg.norm(b_or)), mismatch
    assert kkt_abs(x, g) <= inst.tol + eps_op
    assert res["bie"][1]["hi_mvps"] < res["rpy"][1]["hi_mvps"]


def test_lowfi_errors_and_footprint():
    case = dense_case("spheres8_grid7x14", 2)
    inst = case["inst"]
    with pytest.raises(L.LcpError):
        L.lcp_setup(L.config_for(inst, L.LCP_MIXED, lowfi_n_theta=5, lowfi_n_phi=9), inst.centers, inst.axes)
    ctx = L.lcp_setup(L.config_for(inst, L.LCP_MIXED), inst.centers, inst.axes)
    try:
        with pytest.raises(L.LcpError):
            L.lcp_apply_A(ctx, np.ones(case["b"].size), L.LCP_LOW_BIE)
    finally:
        L.lcp_destroy(ctx)
    cfg = L.config_for(inst, L.LCP_MIXED, lowfi_n_theta=6, lowfi_n_phi=12)
    ctx = L.lcp_setup(cfg, inst.centers, inst.axes)
    try:
        L.lcp_solve(ctx, L.LCP_BI_PQN, inst.tol)
        est = L.lcp_footprint_estimate(cfg, inst.n_bodies, L.lcp_sizes(ctx)[2])
        foot = L.lcp_footprint(ctx)
        assert foot <= est
        plain = L.lcp_setup(L.config_for(inst, L.LCP_MIXED), inst.centers, inst.axes)
        try:
            assert foot > L.lcp_footprint(plain)      # the coarse-grid context is counted
        finally:
            L.lcp_destroy(plain)
    finally:
        L.lcp_destroy(ctx)


def test_coarse_child_keeps_parent_shared_memory_limits():
    """A coarse-grid child context set up after its parent needs less shared
    memory per pair kernel; the parent's launches must still be allowed theirs
    (11 x 22 parent: the symmetric double-float kernel takes 105 KB, the 8 x 16
    child 61 KB)."""
    inst = make_instance("spheres8_grid7x14", 0)
    cfg = L.config_for(inst, L.LCP_MIXED, n_theta=11, n_phi=22, lowfi_n_theta=8, lowfi_n_phi=16)
    ctx = L.lcp_setup(cfg, inst.centers, inst.axes)
    try:
        n = 3 * L.lcp_sizes(ctx)[1]
        phi = torch.tensor(np.random.default_rng(4).standard_normal(n), device="cuda")
        ref = torch.empty_like(phi)
        L.lcp_stokes_apply_dev(ctx, phi, ref, L.LCP_FP64)
        out = torch.empty_like(phi)
        for v in ("sym_a4", "sym_p8rc", "t2c8"):
            L.lcp_select_kernel_variant(ctx, v)
            L.lcp_stokes_apply_dev(ctx, phi, out, L.LCP_DF64)
            assert rel(out.cpu().numpy(), ref.cpu().numpy()) <= 1e-12, v
            L.lcp_stokes_apply_dev(ctx, phi, out, L.LCP_MIXED)
            assert rel(out.cpu().numpy(), ref.cpu().numpy()) <= 1e-5, v
    finally:
        L.lcp_destroy(ctx)
