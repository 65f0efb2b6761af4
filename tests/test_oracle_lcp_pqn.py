"""Pins for the oracle's LCP solvers and its Mono-/Bi-PQN restatement.

Closed forms (n = 1, diagonal A), brute-force enumeration of active sets, the
exact 1-D minimiser behind Algorithm 2, the brute-force weighted prox behind
Proposition 1, the inverse relation between the two-loop H and the unrolled
B, the reduction of Mono-PQN to conjugate gradients when no constraint is
active (Sec. 3.3), monotone decrease (Appendix B) and the Bi-PQN secant
identity B^(k+1) S_low = Y_low (Sec. 5.2).
"""
import numpy as np
import pytest

from oracle import pqn as P
from oracle.bie import DenseMobility
from oracle.contacts import contact_matrix, detect_contacts
from oracle.lcp import brute_force, kkt_abs, lcp_data, objective, pgs
from oracle.rpy import rpy_matrix
from workloads import make_instance


def random_spd(n, rng, cond=10.0):
    Q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    return Q @ np.diag(np.linspace(1.0, cond, n)) @ Q.T


def test_lcp_closed_forms():
    A = np.array([[2.5]])
    for bb in (-3.0, 0.0, 4.0):
        b = np.array([bb])
        x = pgs(A, b)
        np.testing.assert_allclose(x, [max(0.0, -bb / 2.5)])
    d = np.array([1.0, 2.0, 3.0, 0.5])
    b = np.array([-1.0, 2.0, -6.0, 0.0])
    np.testing.assert_allclose(pgs(np.diag(d), b), np.maximum(0, -b / d))
    np.testing.assert_allclose(brute_force(np.diag(d), b), np.maximum(0, -b / d))


@pytest.mark.parametrize("seed", range(8))
def test_pgs_matches_brute_force(seed):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(2, 10))
    A = random_spd(n, rng)
    b = rng.standard_normal(n) * 3
    x1, x2 = pgs(A, b), brute_force(A, b)
    np.testing.assert_allclose(x1, x2, atol=1e-12)
    assert kkt_abs(x1, A @ x1 + b, ord=np.inf) <= 1e-12
    assert (x1 >= 0).all() and ((A @ x1 + b) >= -1e-12).all()


@pytest.mark.parametrize("seed", range(6))
def test_step_size_is_exact_constrained_minimiser(seed):
    rng = np.random.default_rng(100 + seed)
    n = 12
    A = random_spd(n, rng)
    b = rng.standard_normal(n)
    x = np.maximum(rng.standard_normal(n), 0.0)
    g = A @ x + b
    p = np.maximum(x - 0.5 * g + 0.3 * rng.standard_normal(n), 0.0) - x
    if p @ g >= 0:
        p = np.maximum(x - g, 0.0) - x
    eta, blk = P.step_size(x, p, g, A @ p)
    # feasible interval [0, eta_max]; the quadratic's minimiser over it
    neg = p < 0
    eta_max = np.min(-x[neg] / p[neg]) if neg.any() else np.inf
    grid = np.linspace(0.0, min(eta_max, 10.0), 200001)
    f = np.array([objective(A, b, x + e * p) for e in grid[::100]])
    e_best = grid[::100][np.argmin(f)]
    assert abs(eta - e_best) <= 2 * (grid[100] - grid[0])
    assert (x + eta * p >= -1e-14).all()
    assert objective(A, b, x + eta * p) <= f.min() + 1e-12


def bfgs_model(n, r, rng, d=None):
    A = random_spd(n, rng, cond=30)
    m = P.QNModel(np.ones(n) if d is None else d, r_max=64)
    for _ in range(r):
        s = rng.standard_normal(n)
        m.update(s, A @ s)
    return m


@pytest.mark.parametrize("seed", range(10))
def test_weighted_prox_matches_brute_force(seed):
    rng = np.random.default_rng(200 + seed)
    n = int(rng.integers(3, 11))
    r = int(rng.integers(1, 5))
    d = rng.uniform(0.5, 2.0, n)
    m = bfgs_model(n, r, rng, d)
    U, V = m._Umat()
    B = np.diag(d) + U @ U.T - V @ V.T
    xt = rng.standard_normal(n) * 2
    z, it, ok = P.prox_ssn(d, U, V, xt)
    assert ok
    z_ref = brute_force(B, -B @ xt)   # prox = LCP  B z - B xt >= 0 perp z >= 0
    np.testing.assert_allclose(z, z_ref, atol=1e-10)


def test_two_loop_inverts_unrolled_bfgs():
    rng = np.random.default_rng(7)
    n = 9
    m = bfgs_model(n, 5, rng, d=rng.uniform(0.5, 2, n))
    U, V = m._Umat()
    B = np.diag(m.d) + U @ U.T - V @ V.T
    g = rng.standard_normal(n)
    np.testing.assert_allclose(m.H(g), np.linalg.solve(B, g), rtol=1e-10, atol=1e-12)
    # the newest pair satisfies the secant condition exactly
    np.testing.assert_allclose(B @ m.S[-1], m.Y[-1], rtol=1e-10, atol=1e-12)


def _dense_bfgs(d, pairs):
    """Textbook BFGS recursion on dense matrices (Nocedal-Wright Eq. 6.19):
    B+ = B - B s s^T B / (s^T B s) + y y^T / (y^T s), from B_0 = diag(d)."""
    B = np.diag(d).astype(float)
    for s, y in pairs:
        Bs = B @ s
        B = B - np.outer(Bs, Bs) / (s @ Bs) + np.outer(y, y) / (y @ s)
    return B


def test_full_memory_keeps_every_pair():
    """Sec. 6 keeps every secant pair: with the default (no bound) the model
    after 20 updates equals the dense BFGS recursion over all 20 pairs."""
    rng = np.random.default_rng(11)
    n = 12
    A = random_spd(n, rng, cond=30)
    d = rng.uniform(0.5, 2.0, n)
    m = P.QNModel(d)
    pairs = []
    for _ in range(20):
        s = rng.standard_normal(n)
        pairs.append((s, A @ s))
        assert m.update(s, A @ s)
    assert m.r == 20
    U, V = m._Umat()
    B = np.diag(d) + U @ U.T - V @ V.T
    np.testing.assert_allclose(B, _dense_bfgs(d, pairs), rtol=1e-9, atol=1e-9)
    g = rng.standard_normal(n)
    np.testing.assert_allclose(m.H(g), np.linalg.solve(B, g), rtol=1e-8, atol=1e-10)


def test_bounded_memory_drops_the_oldest_quarter():
    """With a storage bound r_max = 8, the ninth pair drops the two oldest pairs
    at once; the rebuilt unrolled B must be the BFGS matrix of exactly the kept
    (most recent) pairs in order, the two-loop H must invert it, and the newest
    pair must satisfy the secant condition."""
    rng = np.random.default_rng(12)
    n = 12
    A = random_spd(n, rng, cond=30)
    d = rng.uniform(0.5, 2.0, n)
    m = P.QNModel(d, r_max=8)
    pairs = []
    counts = []
    for _ in range(13):
        s = rng.standard_normal(n)
        pairs.append((s, A @ s))
        assert m.update(s, A @ s)
        counts.append(m.r)
    # 1..8 kept, 9th -> 7 (drop 2), 10th -> 8, 11th -> 7, 12th -> 8, 13th -> 7
    assert counts == [1, 2, 3, 4, 5, 6, 7, 8, 7, 8, 7, 8, 7]
    kept = pairs[-7:]
    for (s_m, y_m), (s_k, y_k) in zip(zip(m.S, m.Y), kept):
        np.testing.assert_array_equal(s_m, s_k)
        np.testing.assert_array_equal(y_m, y_k)
    U, V = m._Umat()
    B = np.diag(d) + U @ U.T - V @ V.T
    np.testing.assert_allclose(B, _dense_bfgs(d, kept), rtol=1e-9, atol=1e-9)
    g = rng.standard_normal(n)
    np.testing.assert_allclose(m.H(g), np.linalg.solve(B, g), rtol=1e-8, atol=1e-10)
    np.testing.assert_allclose(B @ m.S[-1], m.Y[-1], rtol=1e-9, atol=1e-10)


def test_mono_pqn_reduces_to_cg_without_active_constraints():
    rng = np.random.default_rng(11)
    n = 8
    A = random_spd(n, rng, cond=20)
    xstar = rng.uniform(50.0, 60.0, n)
    b = -A @ xstar
    x0 = xstar + rng.uniform(-1, 1, n)
    res = P.mono_pqn(lambda v: A @ v, b, x0, tol=1e-11, kmax=50)
    # conjugate gradients from the same start
    x = x0.copy()
    r = -(A @ x + b)
    p = r.copy()
    cg = [x.copy()]
    for _ in range(n):
        if np.linalg.norm(r) < 1e-12:
            break
        al = (r @ r) / (p @ A @ p)
        x = x + al * p
        rn = r - al * (A @ p)
        p = rn + (rn @ rn) / (r @ r) * p
        r = rn
        cg.append(x.copy())
    assert res.converged and res.iterations <= n
    np.testing.assert_allclose(res.x, xstar, rtol=1e-10)
    # replay: the first few iterates coincide with CG's, with B_0 = I and with B_0 = delta I
    for scale0 in (False, True):
        replay = P.mono_pqn(lambda v: A @ v, b, x0, tol=0.0, kmax=3, scale0=scale0)
        np.testing.assert_allclose(replay.x, cg[3], rtol=1e-9)


def dense_instance(name, index):
    inst = make_instance(name, index)
    mob = DenseMobility(inst.centers, inst.n_theta, inst.n_phi, a=inst.radius)
    pairs, normals, gaps = detect_contacts(inst.centers, inst.contact_radius, inst.delta)
    D = contact_matrix(inst.n_bodies, pairs, normals)
    U_nc = mob.apply(np.zeros(6 * inst.n_bodies), axes=inst.axes)
    A, b = lcp_data(D, mob.matrix(), U_nc, gaps, inst.dt)
    Ahat = D.T @ rpy_matrix(inst.centers, a=inst.radius) @ D
    return inst, A, b, Ahat


@pytest.mark.parametrize("index", range(4))
def test_pqn_on_packings(index):
    inst, A, b, Ahat = dense_instance("spheres8_grid7x14", index)
    n = b.size
    xs = pgs(A, b)
    xb = brute_force(A, b)
    np.testing.assert_allclose(xs, xb, atol=1e-12)
    assert np.count_nonzero(xs) >= 1          # the instance is not trivial
    mono = P.mono_pqn(lambda v: A @ v, b, np.zeros(n), tol=inst.tol)
    assert mono.converged
    np.testing.assert_allclose(mono.x, xs, atol=1e-6)
    # MVP reuse drift: g tracks A x + b
    assert np.abs(mono.g - (A @ mono.x + b)).max() <= 1e-12 * (1 + np.abs(mono.g).max()) * 10
    bi = P.bi_pqn(lambda v: A @ v, lambda v: Ahat @ v, b, np.zeros(n), tol=inst.tol)
    assert bi.converged
    np.testing.assert_allclose(bi.x, xs, atol=1e-6)
    assert set(np.nonzero(bi.x > 1e-9)[0]) == set(np.nonzero(xs > 1e-9)[0])


def test_mono_pqn_objective_decreases_monotonically():
    """Appendix B: the optimal over-relaxation gives sufficient decrease on the QP.

    The discrete A is symmetric only up to quadrature error, so the QP
    objective is taken with its symmetric part.
    """
    inst, A, b, _ = dense_instance("spheres8_grid7x14", 4)
    A = 0.5 * (A + A.T)
    vals = []
    x = np.zeros(b.size)
    for k in range(1, 12):
        r = P.mono_pqn(lambda v: A @ v, b, x, tol=0.0, kmax=k)
        vals.append(objective(A, b, r.x))
    assert all(v1 <= v0 + 1e-13 for v0, v1 in zip(vals, vals[1:]))


def test_bi_pqn_exact_low_fidelity_needs_one_high_fidelity_mvp():
    inst, A, b, _ = dense_instance("spheres8_grid7x14", 1)
    bi = P.bi_pqn(lambda v: A @ v, lambda v: A @ v, b, np.zeros(b.size), tol=inst.tol)
    assert bi.converged and bi.hi_mvps == 1


def test_bi_pqn_approximate_initialisation():
    """Sec. 5.2 solves the low-fidelity initialisation only approximately: with
    init_forcing the init stops at a relative KKT decrease; the outer loop still
    reaches the LCP solution, and with an exact low fidelity it needs at most the
    gradient MVP plus two corrections (each subproblem is then the exact problem,
    solved to the forcing tolerance)."""
    inst, A, b, Ahat = dense_instance("spheres8_grid7x14", 1)
    xs = pgs(A, b)
    exact = P.bi_pqn(lambda v: A @ v, lambda v: A @ v, b, np.zeros(b.size), tol=inst.tol, init_forcing=1e-3)
    assert exact.converged and 1 <= exact.hi_mvps <= 3
    np.testing.assert_allclose(exact.x, xs, atol=1e-6)
    full = P.bi_pqn(lambda v: A @ v, lambda v: Ahat @ v, b, np.zeros(b.size), tol=inst.tol)
    approx = P.bi_pqn(lambda v: A @ v, lambda v: Ahat @ v, b, np.zeros(b.size), tol=inst.tol, init_forcing=1e-3)
    assert approx.converged
    np.testing.assert_allclose(approx.x, xs, atol=1e-6)
    assert approx.lo_mvps <= full.lo_mvps
    # the init stops at the relative decrease: its KKT history ends at <= 1e-3 of its start
    init = P.mono_pqn(lambda v: Ahat @ v, b, np.zeros(b.size), tol=inst.tol, tol_rel=1e-3)
    assert init.history[-1] <= max(inst.tol, 1e-3 * init.history[0])
    assert len(init.history) < len(P.mono_pqn(lambda v: Ahat @ v, b, np.zeros(b.size), tol=inst.tol).history)


def _secant_trace(sign):
    """Run Bi-PQN's outer loop and report max |B^(k+1) S_low - Y_low|.

    sign=+1 is the carry-over the oracle uses; sign=-1 is the printed sign,
    planted here to show the identity test detects it.
    """
    inst, A, b, Ahat = dense_instance("spheres8_grid7x14", 4)
    n = b.size
    init = P.mono_pqn(lambda v: Ahat @ v, b, np.zeros(n), tol=1e-10)
    S_low, Y_low = list(init.model.S), list(init.model.Y)
    Uh, Vh = [], []
    x = init.x
    g = A @ x + b
    worst = 0.0
    for k in range(3):
        Bmat = Ahat + sum(np.outer(u, u) - np.outer(v, v) for u, v in zip(Uh, Vh)) if Uh else Ahat.copy()
        sub = P.mono_pqn(lambda v: (Bmat @ v, Ahat @ v), b, x, tol=1e-12, pairs=list(zip(S_low, Y_low)),
                         g0=g, extra_mvp=True)
        p = sub.x - x
        if not np.any(p):
            break
        Ap = A @ p
        eta, _ = P.step_size(x, p, g, Ap)
        s, y = eta * p, eta * Ap
        Bs = Bmat @ s
        u, v = y / np.sqrt(y @ s), Bs / np.sqrt(s @ Bs)
        Uh.append(u)
        Vh.append(v)
        x = x + eta * p
        g = g + eta * Ap
        S_low = list(sub.model.S)
        Y_low = [yy + sign * (u * (u @ ss) - v * (v @ ss)) for ss, yy in zip(S_low, sub.model.Y)]
        Bnew = Bmat + np.outer(u, u) - np.outer(v, v)
        for ss, yy in zip(S_low, Y_low):
            worst = max(worst, np.abs(Bnew @ ss - yy).max() / (1 + np.abs(yy).max()))
    return worst


def test_bi_pqn_secant_carry_over_identity():
    assert _secant_trace(+1) <= 1e-10
    assert _secant_trace(-1) > 1e-6      # the printed sign breaks the identity


@pytest.mark.parametrize("index", range(3))
def test_bb_pgd_converges_to_the_lcp_solution(index):
    from oracle.pgd import bb_pgd
    inst, A, b, _ = dense_instance("spheres8_grid7x14", index)
    xs = pgs(A, b)
    x, g, it, mvps, ok = bb_pgd(lambda v: A @ v, b, np.zeros(b.size), tau0=3 * np.pi, tol=inst.tol)
    assert ok and mvps == it + 1
    np.testing.assert_allclose(x, xs, atol=1e-6)
    np.testing.assert_allclose(g, A @ x + b, atol=1e-12)


def test_bb_step_is_the_inverse_rayleigh_quotient_on_a_quadratic():
    """With no active constraint the second step uses tau = s^T s / s^T A s."""
    from oracle.pgd import bb_pgd
    rng = np.random.default_rng(5)
    A = random_spd(6, rng)
    xstar = rng.uniform(20, 30, 6)
    b = -A @ xstar
    x0 = xstar + rng.uniform(-1, 1, 6)
    x1, g1, *_ = bb_pgd(lambda v: A @ v, b, x0, tau0=0.1, tol=0.0, kmax=1)
    s = x1 - x0
    tau = (s @ s) / (s @ A @ s)
    x2, *_ = bb_pgd(lambda v: A @ v, b, x0, tau0=0.1, tol=0.0, kmax=2)
    np.testing.assert_allclose(x2, x1 - tau * (A @ x1 + b), rtol=1e-12)


def test_contact_matrix_gives_the_rate_of_change_of_the_gaps():
    """(D^T U)_l is the time derivative of gap l when the bodies move with U (Sec. 3:
    D^T = grad Phi G): checked by finite differences of the gaps under random body
    velocities (a swapped normal or body index flips the sign)."""
    inst = make_instance("spheres8_grid7x14", 1)
    a = inst.contact_radius
    pairs, normals, gaps = detect_contacts(inst.centers, a, inst.delta)
    D = contact_matrix(inst.n_bodies, pairs, normals)
    U = np.random.default_rng(5).standard_normal((inst.n_bodies, 6))
    eps = 1e-6
    moved = inst.centers + eps * U[:, :3]
    gaps_eps = np.array([np.linalg.norm(moved[j] - moved[i]) - 2 * a for i, j in pairs])
    np.testing.assert_allclose((gaps_eps - gaps) / eps, D.T @ U.reshape(-1), atol=1e-5)


def test_contact_forces_conserve_momentum_and_angular_momentum():
    """A unit contact force is a pair of equal and opposite forces along the line of
    centres: the total force and the total torque about the origin vanish."""
    inst = make_instance("spheres8_grid7x14", 2)
    pairs, normals, _ = detect_contacts(inst.centers, inst.contact_radius, inst.delta)
    D = contact_matrix(inst.n_bodies, pairs, normals)
    FT = (D @ np.random.default_rng(6).uniform(0, 1, len(pairs))).reshape(-1, 6)
    np.testing.assert_allclose(FT[:, :3].sum(0), 0.0, atol=1e-12)
    np.testing.assert_allclose(np.cross(inst.centers, FT[:, :3]).sum(0), 0.0, atol=1e-11)
    np.testing.assert_array_equal(FT[:, 3:], 0.0)


def test_collisional_set_threshold():
    """Eq. (collisional-set): a pair enters when its gap is at most delta."""
    a, delta = 1.25, 0.05
    c = np.array([[0.0, 0.0, 0.0], [2 * a + 0.03, 0.0, 0.0], [0.0, 2 * a + delta + 1e-9, 0.0],
                  [0.0, 0.0, 2 * a + delta]])
    pairs, normals, gaps = detect_contacts(c, a, delta)
    assert [tuple(p) for p in pairs] == [(0, 1), (0, 3)]
    np.testing.assert_allclose(gaps, [0.03, delta], atol=1e-14)
    np.testing.assert_allclose(normals, [[1.0, 0, 0], [0, 0, 1.0]], atol=1e-15)


def test_rpy_mobility_is_symmetric_positive_definite():
    """The RPY tensor of non-overlapping equal spheres is a symmetric positive definite
    mobility (a property of the Rotne-Prager-Yamakawa construction for r >= 2a)."""
    for k in range(3):
        inst = make_instance("spheres64_grid9x18", k)
        R = rpy_matrix(inst.centers, a=inst.radius)
        np.testing.assert_allclose(R, R.T, atol=1e-15)
        assert np.linalg.eigvalsh(R).min() > 0.0
