"""Batched solves, the continuous-batching server and the kernel autotuner (GPU).

Each result must be the same alone and in the mix: contexts share nothing and
every reduction has a fixed order, so the check is bitwise.
"""
import time

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2604_10089_gb300 as L  # noqa: E402
from oracle.contacts import contact_matrix, detect_contacts  # noqa: E402
from oracle.lcp import kkt_abs  # noqa: E402
from oracle.mf import MatrixFreeMobility  # noqa: E402
from workloads import batched_instances  # noqa: E402

from .cases import MISMATCH_REL, SELF_QUADRATURE, kkt_bound  # noqa: E402


def check_against_oracle(inst, x, g_gpu, hi_mvps):
    """KKT error of x with the matrix-free FP64 oracle's MVP and b: <= tol + eps_op."""
    mf = MatrixFreeMobility(inst.centers, inst.n_theta, inst.n_phi, a=inst.radius, mu=inst.viscosity,
                            self_quadrature=SELF_QUADRATURE)
    pairs, normals, gaps = detect_contacts(inst.centers, inst.contact_radius, inst.delta)
    D = contact_matrix(inst.n_bodies, pairs, normals)
    b = gaps / inst.dt + D.T @ mf.apply(np.zeros(6 * inst.n_bodies), axes=inst.axes)
    g = D.T @ mf.apply(D @ x) + b
    eps_op, mismatch = kkt_bound(inst.tol, x, g, g_gpu, b, hi_mvps)
    assert mismatch <= MISMATCH_REL * max(1.0, np.linalg.norm(b)), mismatch
    assert kkt_abs(x, g) <= inst.tol + eps_op


@pytest.fixture(scope="module")
def small_batch():
    insts = [i for i in batched_instances(64, seed=4100) if i.n_bodies <= 40][:10]
    assert len(insts) >= 6
    return insts


VARIANTS = ("sym_a4", "sym_a4m4", "sym_a8m2", "sym_a2", "sym", "sym_t8b2", "sym_t8b4", "sym_p8rc", "sym_p4rc", "sym_p8rc5",
            "t2c8", "t1c8", "t2c16", "t2c4", "t1c16")


def make_ctxs(insts, **kw):
    return [L.lcp_setup(L.config_for(i, L.LCP_MIXED, own_stream=1, **kw), i.centers, i.axes) for i in insts]


def solve_alone(ctxs, insts):
    out = []
    for c, i in zip(ctxs, insts):
        x, st, _ = L.lcp_solve(c, L.LCP_BI_PQN, i.tol)
        assert st["converged"] == 1
        out.append(x)
    return out


# Bi-PQN's low fidelity in the batched and served solves: the RPY mobility, or the
# boundary-integral mobility on a coarse 6 x 12 grid (the bench's choice where it resolves
# neighbouring spheres)
LOWFI = {"rpy": {}, "coarse": dict(lowfi_n_theta=6, lowfi_n_phi=12, lowfi_tol=1e-4, init_forcing=1e-3)}


@pytest.mark.parametrize("lowfi", ["rpy", "coarse"])
def test_batch_equals_alone(small_batch, lowfi):
    ctxs = make_ctxs(small_batch, **LOWFI[lowfi])
    try:
        alone = solve_alone(ctxs, small_batch)
        xs = [torch.empty(L.lcp_sizes(c)[2], dtype=torch.float64, device="cuda") for c in ctxs]
        statuses, stats = L.lcp_batch_solve(ctxs, L.LCP_BI_PQN, 1e-8, xs, workers=6)
        torch.cuda.synchronize()
        assert all(s == L.LCP_OK for s in statuses)
        for a, x in zip(alone, xs):
            assert np.array_equal(a, x.cpu().numpy())
        # and every batched result against the oracle
        for c, i, x, st in zip(ctxs, small_batch, xs, stats):
            xh = x.cpu().numpy()
            check_against_oracle(i, xh, L.lcp_apply_A(c, xh, L.LCP_HIGH) + L.lcp_get_b(c), st["hi_mvps"])
    finally:
        for c in ctxs:
            L.lcp_destroy(c)


def test_server_continuous_batching_and_admission(small_batch):
    ctxs = make_ctxs(small_batch)
    try:
        alone = solve_alone(ctxs, small_batch)
        foot = [L.lcp_footprint(c) for c in ctxs]
        budget = sum(sorted(foot)[:3]) + max(foot)      # not everything fits at once
        srv = L.lcp_server_create(3, budget)
        try:
            waiting = list(range(len(ctxs)))
            running = {}
            results = {}
            t_end = time.time() + 120
            while (waiting or running) and time.time() < t_end:
                for k in list(waiting):                      # admit and submit while memory allows
                    if L.lcp_server_admit(srv, ctxs[k]) == L.LCP_OK:
                        running[k] = L.lcp_server_submit(srv, ctxs[k], L.LCP_BI_PQN, 1e-8)
                        waiting.remove(k)
                for k, t in list(running.items()):
                    status, x, st = L.lcp_server_poll(srv, t, L.lcp_sizes(ctxs[k])[2], 1000)
                    if status == L.LCP_ERR_TIMEOUT:
                        continue
                    assert status == L.LCP_OK and st["converged"] == 1
                    results[k] = x
                    del running[k]
                    L.lcp_server_release(srv, ctxs[k])
                resident, _, _ = L.lcp_server_stats(srv)
                assert resident <= budget
            assert len(results) == len(ctxs)
            for k in range(len(ctxs)):
                assert np.array_equal(results[k], alone[k])
            # a ticket that does not exist times out quickly
            status, _, _ = L.lcp_server_poll(srv, 10 ** 9, 1, 1000)
            assert status == L.LCP_ERR_TIMEOUT
            # a context that was not admitted is rejected
            with pytest.raises(L.LcpError):
                L.lcp_server_submit(srv, ctxs[0], L.LCP_BI_PQN, 1e-8)
        finally:
            L.lcp_server_destroy(srv)
    finally:
        for c in ctxs:
            L.lcp_destroy(c)


@pytest.mark.parametrize("lowfi", ["rpy", "coarse"])
def test_server_simulations_held_admission(small_batch, lowfi):
    """Server-owned simulations: each request carries its problem, the server creates the
    context only when its estimated footprint fits the budget (holding the request until
    then), keeps it resident across time steps and frees it on close.  Results equal solving
    alone (two steps each), the first solves are checked against the oracle, and the budget
    is never exceeded."""
    insts = small_batch[:6]
    cfgs = [L.config_for(i, L.LCP_MIXED, **LOWFI[lowfi]) for i in insts]
    est = [L.lcp_footprint_estimate(c, i.n_bodies, 6 * i.n_bodies) for c, i in zip(cfgs, insts)]
    budget = sum(sorted(est)[:2]) + max(est)          # at most three at once, often two
    # alone: solve, step, solve on a context of its own
    alone = []
    for c, i in zip(cfgs, insts):
        ctx = L.lcp_setup(c, i.centers, i.axes)
        try:
            x1, _, _ = L.lcp_solve(ctx, L.LCP_BI_PQN, i.tol)
            L.lcp_step(ctx, i.dt)
            x2, _, _ = L.lcp_solve(ctx, L.LCP_BI_PQN, i.tol)
            alone.append((x1, x2, L.lcp_sizes(ctx)[2]))
        finally:
            L.lcp_destroy(ctx)
    srv = L.lcp_server_create(3, budget)
    try:
        sims = [L.lcp_server_open(srv, c, i.centers, i.axes) for c, i in zip(cfgs, insts)]
        tickets = {k: L.lcp_server_request(srv, sims[k], L.LCP_BI_PQN, insts[k].tol, insts[k].dt)
                   for k in range(len(sims))}
        results = {k: [] for k in range(len(sims))}
        saw_held = False
        t_end = time.time() + 180
        while tickets and time.time() < t_end:
            resident, queued, _ = L.lcp_server_stats(srv)
            assert resident <= budget
            saw_held = saw_held or queued > 0
            for k, t in list(tickets.items()):
                n = alone[k][0].size if not results[k] else alone[k][2]
                status, x, st = L.lcp_server_poll(srv, t, n, 1000)
                if status == L.LCP_ERR_TIMEOUT:
                    continue
                assert status == L.LCP_OK and st["converged"] == 1
                results[k].append((x, st))
                if len(results[k]) == 1:        # next step: solve only
                    tickets[k] = L.lcp_server_request(srv, sims[k], L.LCP_BI_PQN, insts[k].tol, 0.0)
                else:
                    del tickets[k]
                    L.lcp_server_close(srv, sims[k])
        assert not tickets and saw_held
        for k in range(len(sims)):
            assert np.array_equal(results[k][0][0], alone[k][0])
            assert np.array_equal(results[k][1][0], alone[k][1])
        # the first solves against the oracle (the GPU gradient from a context of its own)
        for k, i in enumerate(insts[:3]):
            ctx = L.lcp_setup(cfgs[k], i.centers, i.axes)
            try:
                x = results[k][0][0]
                g_gpu = L.lcp_apply_A(ctx, x, L.LCP_HIGH) + L.lcp_get_b(ctx)
            finally:
                L.lcp_destroy(ctx)
            check_against_oracle(i, x, g_gpu, results[k][0][1]["hi_mvps"])
        assert L.lcp_server_stats(srv)[0] == 0
        # a simulation that can never fit is rejected at once
        big = L.lcp_server_open(srv, cfgs[0], np.arange(3 * 2000, dtype=float).reshape(-1, 3) * 3.0)
        with pytest.raises(L.LcpError) as err:
            L.lcp_server_request(srv, big, L.LCP_BI_PQN, 1e-8)
        assert err.value.status == L.LCP_ERR_REJECTED
        L.lcp_server_close(srv, big)
    finally:
        L.lcp_server_destroy(srv)


def test_autotuned_kernel_gives_the_same_solution(small_batch):
    inst = small_batch[0]
    a = L.lcp_setup(L.config_for(inst, L.LCP_MIXED), inst.centers, inst.axes)
    b = L.lcp_setup(L.config_for(inst, L.LCP_MIXED, autotune=1), inst.centers, inst.axes)
    try:
        assert L.lcp_kernel_variant(a) == "t2c8"    # few units per CTA: the plain kernel
        assert L.lcp_kernel_variant(b) in VARIANTS
        xa, _, _ = L.lcp_solve(a, L.LCP_BI_PQN, inst.tol)
        xb, _, _ = L.lcp_solve(b, L.LCP_BI_PQN, inst.tol)
        np.testing.assert_allclose(xb, xa, atol=1e-7 * max(1.0, np.abs(xa).max()))
    finally:
        L.lcp_destroy(a)
        L.lcp_destroy(b)


def test_footprint_estimate_covers_context(small_batch):
    """Admission by estimate is safe: the estimate bounds the bytes a solved context holds."""
    for inst in small_batch[:4]:
        ctx = L.lcp_setup(L.config_for(inst, L.LCP_MIXED), inst.centers, inst.axes)
        try:
            _, st, _ = L.lcp_solve(ctx, L.LCP_BI_PQN, inst.tol)
            assert st["converged"] == 1
            n = L.lcp_sizes(ctx)[2]
            est = L.lcp_footprint_estimate(L.config_for(inst, L.LCP_MIXED), inst.n_bodies, n)
            assert L.lcp_footprint(ctx) <= est
        finally:
            L.lcp_destroy(ctx)


@pytest.mark.parametrize("name,index", [("spheres8_grid7x14", 2), ("spheres64_grid9x18", 1), ("grid16x32", 0)])
def test_every_kernel_variant_applies_the_same_operator(name, index):
    """Each FP32 variant (symmetric or plain, any tile shape) against the double-FP32 apply;
    grid16x32 is the largest sphere grid (512 nodes, padded to 515 for five-source batches)."""
    from workloads import make_instance
    if name == "grid16x32":
        idx = np.stack(np.meshgrid(*[np.arange(k) for k in (4, 4, 2)], indexing="ij"), -1).reshape(-1, 3)
        centers = idx * 2.7 + np.random.default_rng(3).uniform(-0.05, 0.05, (32, 3))
        cfg = L.lcp_default_config(n_theta=16, n_phi=32, precision=L.LCP_MIXED)
        ctx = L.lcp_setup(cfg, centers)
    else:
        inst = make_instance(name, index)
        ctx = L.lcp_setup(L.config_for(inst, L.LCP_MIXED), inst.centers, inst.axes)
    try:
        n = 3 * L.lcp_sizes(ctx)[1]
        phi = torch.tensor(np.random.default_rng(9).standard_normal(n), device="cuda")
        ref = torch.empty_like(phi)
        L.lcp_stokes_apply_dev(ctx, phi, ref, L.LCP_DF64)
        out = torch.empty_like(phi)
        ref64 = torch.empty_like(phi)
        L.lcp_stokes_apply_dev(ctx, phi, ref64, L.LCP_FP64)
        for v in VARIANTS:
            try:
                L.lcp_select_kernel_variant(ctx, v)
            except L.LcpError:
                assert name == "grid16x32" and not v.startswith("sym_p")   # may not fit the largest grid
                continue
            assert L.lcp_kernel_variant(ctx) == v
            L.lcp_stokes_apply_dev(ctx, phi, out, L.LCP_MIXED)
            err = float((out - ref).abs().max() / ref.abs().max())
            assert err <= 1e-5, (v, err)
            # the double-float residual sum follows the choice (symmetric or plain): FP64 accuracy
            L.lcp_stokes_apply_dev(ctx, phi, out, L.LCP_DF64)
            err = float((out - ref64).abs().max() / ref64.abs().max())
            assert err <= 1e-12, (v, "df", err)
        with pytest.raises(L.LcpError):
            L.lcp_select_kernel_variant(ctx, "no_such_kernel")
    finally:
        L.lcp_destroy(ctx)


def test_captured_arnoldi_graphs_match_direct_launches(small_batch):
    """Contexts on their own stream replay each GMRES Arnoldi step as a captured
    CUDA graph; on the legacy stream the same kernels are launched directly.  The
    arithmetic is identical, so the results are bitwise equal, also on replay."""
    inst = small_batch[1]
    direct = L.lcp_setup(L.config_for(inst, L.LCP_MIXED), inst.centers, inst.axes)
    graphed = L.lcp_setup(L.config_for(inst, L.LCP_MIXED, own_stream=1), inst.centers, inst.axes)
    try:
        xa, sa, _ = L.lcp_solve(direct, L.LCP_BI_PQN, inst.tol)
        n0 = L.lcp_launch_count(graphed)
        xb, sb, _ = L.lcp_solve(graphed, L.LCP_BI_PQN, inst.tol)
        n1 = L.lcp_launch_count(graphed)
        xc, sc, _ = L.lcp_solve(graphed, L.LCP_BI_PQN, inst.tol)
        n2 = L.lcp_launch_count(graphed)
        assert np.array_equal(xa, xb) and np.array_equal(xb, xc)
        assert sa["gmres_iterations"] == sb["gmres_iterations"] == sc["gmres_iterations"]
        assert sa["fp32_applies"] == sb["fp32_applies"]
        assert n2 - n1 == n1 - n0 > 0      # replayed kernels are counted like launched ones
    finally:
        L.lcp_destroy(direct)
        L.lcp_destroy(graphed)


def test_kernel_timing_inside_graph_replays(small_batch):
    """With kernel timing on, the GMRES steps still replay as graphs (their own
    recorded events are read after each replay): the same bitwise result, one timed
    launch per FP32 apply of the fine grid, positive durations; timing off again
    returns to the untimed graphs."""
    inst = small_batch[1]
    ctx = L.lcp_setup(L.config_for(inst, L.LCP_MIXED, own_stream=1), inst.centers, inst.axes)
    try:
        xa, sa, _ = L.lcp_solve(ctx, L.LCP_BI_PQN, inst.tol)
        L.lcp_profile(ctx, True)
        xb, sb, _ = L.lcp_solve(ctx, L.LCP_BI_PQN, inst.tol)
        xc, sc, _ = L.lcp_solve(ctx, L.LCP_BI_PQN, inst.tol)
        count, ms = L.lcp_profile_read(ctx, 0)
        L.lcp_profile(ctx, False)
        xd, _, _ = L.lcp_solve(ctx, L.LCP_BI_PQN, inst.tol)
        assert np.array_equal(xa, xb) and np.array_equal(xa, xc) and np.array_equal(xa, xd)
        assert count == sb["fp32_applies"] + sc["fp32_applies"] > 0
        assert ms > 0.0
    finally:
        L.lcp_destroy(ctx)
