"""GPU parity: every step of the hot path through the C ABI against the FP64 oracle.

Tolerances (relative, max-norm over the compared vector):
  FP64 stresslet apply             1e-12   (rounding order only)
  double-FP32 stresslet apply      1e-12   (~2^-44 per operation)
  FP32 stresslet apply (unrefined) 1e-4    (the mixed-mode bound of the spec; measured ~1e-6)
  mobility solve, FP64 and mixed   1e-9    (GMRES tol 1e-12 on a well-conditioned second-kind system)
  RPY, D, D^T, b                   1e-12 / 1e-9
  LCP solutions: same active set as the oracle and ||min(x, A x + b)||_2 <= tol + eps_op with
  the oracle's A and b, eps_op = the measured gap between the oracle's gradient and a fresh GPU
  MVP at x plus the bounded drift of the GPU's updated gradient (cases.kkt_bound); the measured
  gap itself must stay below 1e-10 ||b||_2.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2604_10089_gb300 as L  # noqa: E402
from oracle.bie import DenseMobility  # noqa: E402
from oracle.lcp import brute_force, kkt_abs  # noqa: E402
from oracle.mf import MatrixFreeMobility  # noqa: E402
from oracle.rpy import rpy_matrix  # noqa: E402
from workloads import make_instance  # noqa: E402

from .cases import MISMATCH_REL, SELF_QUADRATURE, active_set, dense_case, kkt_bound, rhs_oracle  # noqa: E402

DEV = "cuda"


def rel(a, b):
    return float(np.abs(np.asarray(a) - np.asarray(b)).max() / max(np.abs(np.asarray(b)).max(), 1e-300))


@pytest.fixture(scope="module")
def c1():
    case = dense_case("spheres8_grid7x14", 1)
    inst = case["inst"]
    ctx = L.lcp_setup(L.config_for(inst), inst.centers, inst.axes)
    yield case, ctx
    L.lcp_destroy(ctx)


def test_contacts_and_b_match_oracle(c1):
    case, ctx = c1
    pairs, normals, gaps = L.lcp_get_contacts(ctx)
    np.testing.assert_array_equal(pairs, case["pairs"])
    np.testing.assert_allclose(normals, case["normals"], atol=1e-15)
    np.testing.assert_allclose(gaps, case["gaps"], atol=1e-14)
    assert rel(L.lcp_get_unc(ctx), case["U_nc"]) <= 1e-9
    assert rel(L.lcp_get_b(ctx), case["b"]) <= 1e-9


@pytest.mark.parametrize("precision,tol", [(L.LCP_FP64, 1e-12), (L.LCP_MIXED, 1e-4), (L.LCP_DF64, 1e-12)])
def test_stresslet_apply(c1, precision, tol):
    case, ctx = c1
    mob = case["mob"]
    phi = np.random.default_rng(3).standard_normal(mob.x.shape[0] * 3)
    ref = (mob.K + mob.P) @ phi
    dphi = torch.tensor(phi, device=DEV)
    out = torch.empty_like(dphi)
    L.lcp_stokes_apply_dev(ctx, dphi, out, precision)
    err = rel(out.cpu().numpy(), ref)
    assert err <= tol, err


@pytest.mark.parametrize("name,index", [("spheres64_grid9x18", 0)])
@pytest.mark.parametrize("precision,tol", [(L.LCP_FP64, 1e-12), (L.LCP_MIXED, 1e-4), (L.LCP_DF64, 1e-12)])
def test_stresslet_apply_many_tiles(name, index, precision, tol):
    """10 368 nodes: 41 target blocks with a ragged tail and several source splits."""
    inst = make_instance(name, index)
    ctx = L.lcp_setup(L.config_for(inst), inst.centers, None)
    try:
        mf = MatrixFreeMobility(inst.centers, inst.n_theta, inst.n_phi, a=inst.radius, self_quadrature=SELF_QUADRATURE)
        phi = np.random.default_rng(5).standard_normal(mf.x.shape[0] * 3)
        ref = mf.apply_operator(phi)
        dphi = torch.tensor(phi, device=DEV)
        out = torch.empty_like(dphi)
        L.lcp_stokes_apply_dev(ctx, dphi, out, precision)
        assert rel(out.cpu().numpy(), ref) <= tol
    finally:
        L.lcp_destroy(ctx)


@pytest.mark.parametrize("precision", [L.LCP_FP64, L.LCP_MIXED])
def test_rhs_and_rigid_velocity(c1, precision):
    """The GMRES right-hand side: FP64 kernel in FP64 mode, double-FP32 kernel in mixed mode."""
    case, ctx64 = c1
    mob, inst = case["mob"], case["inst"]
    ctx = ctx64 if precision == L.LCP_FP64 else L.lcp_setup(L.config_for(inst, precision), inst.centers,
                                                              inst.axes)
    try:
        FT = np.random.default_rng(4).standard_normal(6 * inst.n_bodies)
        dFT = torch.tensor(FT, device=DEV)
        rhs = torch.empty(mob.x.shape[0] * 3, dtype=torch.float64, device=DEV)
        L.lcp_stokes_rhs_dev(ctx, dFT, True, rhs)
        assert rel(rhs.cpu().numpy(), rhs_oracle(mob, FT, inst.axes)) <= 1e-13
        L.lcp_stokes_rhs_dev(ctx, dFT, False, rhs)
        assert rel(rhs.cpu().numpy(), rhs_oracle(mob, FT)) <= 1e-13
    finally:
        if ctx is not ctx64:
            L.lcp_destroy(ctx)
    ctx = ctx64
    phi = np.random.default_rng(6).standard_normal(mob.x.shape[0] * 3)
    UO = torch.empty(6 * inst.n_bodies, dtype=torch.float64, device=DEV)
    L.lcp_rigid_velocity_dev(ctx, torch.tensor(phi, device=DEV), UO)
    from oracle.bie import rigid_velocities
    assert rel(UO.cpu().numpy(), rigid_velocities(phi, mob.parts)) <= 1e-13


@pytest.mark.parametrize("precision,residual", [(L.LCP_FP64, L.LCP_FP64), (L.LCP_MIXED, L.LCP_DF64),
                                                (L.LCP_MIXED, L.LCP_FP64)])
def test_mobility_matches_dense_lu(c1, precision, residual):
    case, _ = c1
    inst, mob = case["inst"], case["mob"]
    ctx = L.lcp_setup(L.config_for(inst, precision, residual_precision=residual), inst.centers, inst.axes)
    try:
        FT = np.random.default_rng(7).standard_normal(6 * inst.n_bodies)
        U = L.mobility_apply(ctx, FT, include_slip=False)
        assert rel(U, case["Mob"] @ FT) <= 1e-9
        Us = L.mobility_apply(ctx, np.zeros(6 * inst.n_bodies), include_slip=True)
        assert rel(Us, case["U_nc"]) <= 1e-9
    finally:
        L.lcp_destroy(ctx)


def test_single_sphere_drag_and_torque():
    cfg = L.lcp_default_config(n_theta=7, n_phi=14, radius=0.9, viscosity=1.7)
    ctx = L.lcp_setup(cfg, [[0.1, 0.2, -0.3]])
    try:
        U = L.mobility_apply(ctx, [1.0, -2.0, 0.5, 0.3, 0.0, -1.0])
        a, mu = 0.9, 1.7
        expect = np.array([1.0, -2.0, 0.5]) / (6 * np.pi * mu * a)
        np.testing.assert_allclose(U[:3], expect, rtol=1e-10)
        np.testing.assert_allclose(U[3:], np.array([0.3, 0.0, -1.0]) / (8 * np.pi * mu * a ** 3), rtol=1e-10, atol=1e-14)
        assert L.lcp_sizes(ctx)[2] == 0
    finally:
        L.lcp_destroy(ctx)


def test_rpy_and_apply_A(c1):
    case, ctx = c1
    inst = case["inst"]
    FT = np.random.default_rng(8).standard_normal(6 * inst.n_bodies)
    U = L.mobility_apply(ctx, FT, fidelity=L.LCP_LOW_RPY)
    assert rel(U, rpy_matrix(inst.centers, a=inst.radius) @ FT) <= 1e-13
    x = np.abs(np.random.default_rng(9).standard_normal(case["b"].size))
    assert rel(L.lcp_apply_A(ctx, x, L.LCP_HIGH), case["A"] @ x) <= 1e-9
    assert rel(L.lcp_apply_A(ctx, x, L.LCP_LOW_RPY), case["Ahat"] @ x) <= 1e-12


def check_solution(case, x, tol, ctx, hi_mvps):
    A, b, xs = case["A"], case["b"], case["x"]
    g = A @ x + b
    g_gpu = L.lcp_apply_A(ctx, x, L.LCP_HIGH) + L.lcp_get_b(ctx)
    eps_op, mismatch = kkt_bound(tol, x, g, g_gpu, b, hi_mvps)
    assert mismatch <= MISMATCH_REL * max(1.0, np.linalg.norm(b)), mismatch
    assert kkt_abs(x, g) <= tol + eps_op, (kkt_abs(x, g), eps_op)
    act, amb = active_set(x, g)
    act_ref, amb_ref = active_set(xs, A @ xs + b)
    assert act - amb_ref == act_ref - amb, (sorted(act), sorted(act_ref))
    assert np.abs(x - xs).max() <= 1e-5 * max(1.0, np.abs(xs).max())


def test_c1_thirty_two_seeds_plain_fp64_mono_pqn():
    """The 8-sphere configuration's run: plain FP64 Mono-PQN on 32 seeded instances (9-11
    contacts each), each against its dense oracle: same active set, KKT error within
    tol + eps_op, x within 1e-5 of the projected Gauss-Seidel solution, and that solution
    equal to the brute-force enumeration of active sets."""
    for index in range(32):
        case = dense_case("spheres8_grid7x14", index)
        inst = case["inst"]
        xbf = brute_force(case["A"], case["b"])
        assert np.abs(xbf - case["x"]).max() <= 1e-9 * max(1.0, np.abs(xbf).max()), index
        ctx = L.lcp_setup(L.config_for(inst, L.LCP_FP64), inst.centers, inst.axes)
        try:
            assert L.lcp_sizes(ctx)[2] == case["b"].size, index
            x, st, status = L.lcp_solve(ctx, L.LCP_MONO_PQN, inst.tol)
            assert status == L.LCP_OK and st["converged"] == 1, index
            check_solution(case, x, inst.tol, ctx, st["hi_mvps"])
        finally:
            L.lcp_destroy(ctx)


@pytest.mark.parametrize("index", [0, 1, 2, 3])
@pytest.mark.parametrize("method", [L.LCP_MONO_PQN, L.LCP_BI_PQN])
@pytest.mark.parametrize("precision", [L.LCP_FP64, L.LCP_MIXED])
def test_lcp_solve_matches_oracle(index, method, precision):
    case = dense_case("spheres8_grid7x14", index)
    inst = case["inst"]
    ctx = L.lcp_setup(L.config_for(inst, precision), inst.centers, inst.axes)
    try:
        x, st, status = L.lcp_solve(ctx, method, inst.tol)
        assert status == L.LCP_OK and st["converged"] == 1
        check_solution(case, x, inst.tol, ctx, st["hi_mvps"])
        assert st["hi_mvps"] >= 1
        if method == L.LCP_BI_PQN:
            assert st["lo_mvps"] >= 1
    finally:
        L.lcp_destroy(ctx)


def test_lcp_solve_device_pointers_and_warm_start():
    case = dense_case("spheres8_grid7x14", 2)
    inst = case["inst"]
    ctx = L.lcp_setup(L.config_for(inst), inst.centers, inst.axes)
    try:
        n = case["b"].size
        x = torch.empty(n, dtype=torch.float64, device=DEV)
        st, _ = L.lcp_solve_dev(ctx, L.LCP_MONO_PQN, inst.tol, None, x)
        check_solution(case, x.cpu().numpy(), inst.tol, ctx, st["hi_mvps"])
        # warm start at the solution: one MVP, no iteration
        x2 = torch.empty_like(x)
        st2, _ = L.lcp_solve_dev(ctx, L.LCP_MONO_PQN, inst.tol, x, x2)
        assert st2["hi_mvps"] == 1 and st2["iterations"] == 0
    finally:
        L.lcp_destroy(ctx)


def test_caller_contacts_in_caller_order():
    case = dense_case("spheres8_grid7x14", 3)
    inst = case["inst"]
    perm = np.random.default_rng(1).permutation(case["b"].size)
    contacts = [(case["pairs"][l][0], case["pairs"][l][1], case["normals"][l], case["gaps"][l]) for l in perm]
    ctx = L.lcp_setup(L.config_for(inst), inst.centers, inst.axes, contacts=contacts)
    try:
        assert rel(L.lcp_get_b(ctx), case["b"][perm]) <= 1e-9
        x, st, _ = L.lcp_solve(ctx, L.LCP_MONO_PQN, inst.tol)
        np.testing.assert_allclose(x, case["x"][perm], atol=1e-5 * max(1, case["x"].max()))
    finally:
        L.lcp_destroy(ctx)


def test_no_contacts_and_trivial_lcp():
    inst = make_instance("spheres8_grid7x14", 0)
    ctx = L.lcp_setup(L.config_for(inst, delta=-1.0), inst.centers, inst.axes)
    try:
        assert L.lcp_sizes(ctx)[2] == 0
        x, st, _ = L.lcp_solve(ctx, L.LCP_BI_PQN, 1e-8)
        assert x.size == 0 and st["converged"] == 1
    finally:
        L.lcp_destroy(ctx)
    # no slip: b = gap / dt > 0, so x = 0 after the first MVP
    ctx = L.lcp_setup(L.config_for(inst), inst.centers, None)
    try:
        x, st, _ = L.lcp_solve(ctx, L.LCP_MONO_PQN, 1e-8)
        assert np.all(x == 0.0) and st["hi_mvps"] == 1
    finally:
        L.lcp_destroy(ctx)


def test_invalid_arguments_are_rejected():
    with pytest.raises(L.LcpError):
        L.lcp_setup(L.lcp_default_config(n_phi=13), [[0, 0, 0]])
    with pytest.raises(L.LcpError):
        L.lcp_setup(L.lcp_default_config(contact_radius=0.5), [[0, 0, 0]])


def _rotate(e, w, dt):
    th = np.linalg.norm(w) * dt
    if th == 0.0:
        return e
    k = w / np.linalg.norm(w)
    out = e * np.cos(th) + np.cross(k, e) * np.sin(th) + k * (k @ e) * (1 - np.cos(th))
    return out / np.linalg.norm(out)


@pytest.mark.parametrize("method", [L.LCP_MONO_PQN, L.LCP_BI_PQN])
def test_time_step_matches_oracle(method):
    """Eq. (dvi): c += dt (U_nc + M D x); the next configuration's b matches the oracle's."""
    case = dense_case("spheres8_grid7x14", 4)
    inst = case["inst"]
    ctx = L.lcp_setup(L.config_for(inst), inst.centers, inst.axes)
    try:
        x, _, _ = L.lcp_solve(ctx, method, inst.tol)
        c_new, a_new = L.lcp_step(ctx, inst.dt)
        U = (case["U_nc"] + case["Mob"] @ (case["D"] @ x)).reshape(-1, 6)
        c_ref = inst.centers + inst.dt * U[:, :3]
        a_ref = np.array([_rotate(inst.axes[i], U[i, 3:], inst.dt) for i in range(inst.n_bodies)])
        np.testing.assert_allclose(c_new, c_ref, atol=1e-12 + 1e-9 * inst.dt * np.abs(U[:, :3]).max())
        np.testing.assert_allclose(a_new, a_ref, atol=1e-10)
        # the context now holds the next LCP
        from oracle.contacts import contact_matrix, detect_contacts
        from oracle.lcp import lcp_data
        mob = DenseMobility(c_ref, inst.n_theta, inst.n_phi, a=inst.radius, self_quadrature=SELF_QUADRATURE)
        pairs, normals, gaps = detect_contacts(c_ref, inst.contact_radius, inst.delta)
        D = contact_matrix(inst.n_bodies, pairs, normals)
        _, b_next = lcp_data(D, np.eye(6 * inst.n_bodies), mob.apply(np.zeros(6 * inst.n_bodies), axes=a_ref),
                             gaps, inst.dt)
        assert rel(L.lcp_get_b(ctx), b_next) <= 1e-8
        with pytest.raises(L.LcpError):
            L.lcp_step(ctx, inst.dt)          # no solve since the last step
    finally:
        L.lcp_destroy(ctx)


def test_short_trajectory_mixed_bi_pqn():
    inst = make_instance("spheres8_grid7x14", 2)
    ctx = L.lcp_setup(L.config_for(inst, L.LCP_MIXED), inst.centers, inst.axes)
    try:
        for _ in range(5):
            x, st, _ = L.lcp_solve(ctx, L.LCP_BI_PQN, inst.tol)
            assert st["converged"] == 1
            c, a = L.lcp_step(ctx, inst.dt)
        d = np.linalg.norm(c[:, None] - c[None], axis=2) + np.eye(len(c)) * 10
        assert d.min() - 2 * inst.contact_radius > -1e-3      # contacts resolved: no deep overlap
        np.testing.assert_allclose(np.linalg.norm(a, axis=1), 1.0, rtol=1e-12)
    finally:
        L.lcp_destroy(ctx)


@pytest.mark.parametrize("index", [0, 1, 3])
def test_bb_pgd_baseline_matches_oracle(index):
    """The BB-PGD comparison method of Sec. 6 on the GPU: same solution, same MVP count as the oracle's."""
    from oracle.pgd import bb_pgd
    case = dense_case("spheres8_grid7x14", index)
    inst = case["inst"]
    ctx = L.lcp_setup(L.config_for(inst), inst.centers, inst.axes)
    try:
        x, st, _ = L.lcp_solve(ctx, L.LCP_BB_PGD, inst.tol)
        check_solution(case, x, inst.tol, ctx, st["hi_mvps"])
        _, _, it, mvps, ok = bb_pgd(lambda v: case["A"] @ v, case["b"], np.zeros(case["b"].size),
                                    tau0=3 * np.pi * inst.viscosity * inst.radius, tol=inst.tol)
        assert ok and abs(st["hi_mvps"] - mvps) <= 1
    finally:
        L.lcp_destroy(ctx)


@pytest.mark.parametrize("method", [L.LCP_MONO_PQN, L.LCP_BI_PQN, L.LCP_BB_PGD])
def test_duplicated_contact_degenerate_lcp(method):
    """A contact listed twice gives A two equal columns (semidefinite, not definite): the
    split of the force between the two copies is not unique, their sum is.  The solvers
    must still converge, the KKT error with the oracle's A stays within tol + eps_op, and
    the pair's total force equals the single-contact solution's."""
    case = dense_case("spheres8_grid7x14", 1)
    inst, A, b, xs = case["inst"], case["A"], case["b"], case["x"]
    l0 = int(np.argmax(xs))                       # an active contact
    order = list(range(xs.size)) + [l0]
    contacts = [(case["pairs"][l][0], case["pairs"][l][1], case["normals"][l], case["gaps"][l]) for l in order]
    ctx = L.lcp_setup(L.config_for(inst), inst.centers, inst.axes, contacts=contacts)
    try:
        x, st, status = L.lcp_solve(ctx, method, inst.tol)
        assert status == L.LCP_OK and st["converged"] == 1
        g_gpu = L.lcp_apply_A(ctx, x, L.LCP_HIGH) + L.lcp_get_b(ctx)
    finally:
        L.lcp_destroy(ctx)
    idx = np.array(order)
    A2, b2 = A[np.ix_(idx, idx)], b[idx]
    g = A2 @ x + b2
    eps_op, mismatch = kkt_bound(inst.tol, x, g, g_gpu, b2, st["hi_mvps"])
    assert mismatch <= MISMATCH_REL * max(1.0, np.linalg.norm(b2)), mismatch
    assert kkt_abs(x, g) <= inst.tol + eps_op
    merged = x[:xs.size].copy()
    merged[l0] += x[-1]
    assert np.abs(merged - xs).max() <= 1e-5 * max(1.0, np.abs(xs).max())
    assert x.min() >= 0.0


def test_update_grows_the_contact_buffers():
    """A context set up with two caller contacts, then updated to the full collisional set
    (more contacts than its first allocation): the solve still matches the oracle."""
    case = dense_case("spheres8_grid7x14", 3)
    inst = case["inst"]
    few = [(case["pairs"][l][0], case["pairs"][l][1], case["normals"][l], case["gaps"][l]) for l in range(2)]
    ctx = L.lcp_setup(L.config_for(inst), inst.centers, inst.axes, contacts=few)
    try:
        assert L.lcp_sizes(ctx)[2] == 2
        L.lcp_solve(ctx, L.LCP_MONO_PQN, inst.tol)
        L.lcp_update(ctx, inst.centers, inst.axes)          # detect: the full set
        assert L.lcp_sizes(ctx)[2] == case["b"].size > 2
        assert rel(L.lcp_get_b(ctx), case["b"]) <= 1e-9
        x, st, _ = L.lcp_solve(ctx, L.LCP_BI_PQN, inst.tol)
        check_solution(case, x, inst.tol, ctx, st["hi_mvps"])
    finally:
        L.lcp_destroy(ctx)


@pytest.mark.parametrize("precision", [L.LCP_FP64, L.LCP_MIXED])
@pytest.mark.parametrize("R", [2.5, 4.0])
def test_two_sphere_resistances_match_exact_stokes_flow(precision, R):
    """The GPU mobility of two spheres on the workloads' 11 x 22 grid against exact Stokes
    flow (not only against the oracle): moving together along their line of centres
    (Stimson & Jeffery), approaching each other (Brenner) and rotating about that line in
    the same or opposite senses (Jeffery), at the steric-shell distance 2.5 radii and at 4."""
    from .exact_stokes import brenner_approach, jeffery_rotation, stimson_jeffery
    cfg = L.lcp_default_config(n_theta=11, n_phi=22, radius=1.0, contact_radius=1.25, precision=precision)
    centers = np.array([[0.0, 0.0, -R / 2], [0.0, 0.0, R / 2]])
    ctx = L.lcp_setup(cfg, centers)
    try:
        for sign, exact, bound in ((1.0, stimson_jeffery(R), 1e-5), (-1.0, brenner_approach(R), 6e-4)):
            FT = np.zeros(12)
            FT[2], FT[8] = 1.0, sign
            U = L.mobility_apply(ctx, FT)
            assert abs(U[8] - sign * U[2]) <= 1e-9 * abs(U[2])
            lam = 1.0 / (6.0 * np.pi * U[2])
            assert abs(lam - exact) <= bound * exact, (sign, lam, exact)
        # rotation about the line of centres, in the same and in opposite senses (Jeffery)
        for sign in (1.0, -1.0):
            exact = jeffery_rotation(R, same_sense=sign > 0)
            FT = np.zeros(12)
            FT[5], FT[11] = 1.0, sign
            U = L.mobility_apply(ctx, FT)
            assert abs(U[11] - sign * U[5]) <= 1e-9 * abs(U[5])
            zeta = 1.0 / (8.0 * np.pi * U[5])
            assert abs(zeta - exact) <= 3e-5 * exact, (sign, zeta, exact)
    finally:
        L.lcp_destroy(ctx)
