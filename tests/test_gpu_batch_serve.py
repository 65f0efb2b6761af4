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
from workloads import batched_instances  # noqa: E402


@pytest.fixture(scope="module")
def small_batch():
    insts = [i for i in batched_instances(64, seed=4100) if i.n_bodies <= 40][:10]
    assert len(insts) >= 6
    return insts


VARIANTS = ("sym_a4", "sym_a4m4", "sym_a8m2", "sym_a2", "sym", "sym_t8b2", "sym_t8b4", "sym_p8rc", "sym_p4rc",
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


def test_batch_equals_alone(small_batch):
    ctxs = make_ctxs(small_batch)
    try:
        alone = solve_alone(ctxs, small_batch)
        xs = [torch.empty(L.lcp_sizes(c)[2], dtype=torch.float64, device="cuda") for c in ctxs]
        statuses, stats = L.lcp_batch_solve(ctxs, L.LCP_BI_PQN, 1e-8, xs, workers=6)
        torch.cuda.synchronize()
        assert all(s == L.LCP_OK for s in statuses)
        for a, x in zip(alone, xs):
            assert np.array_equal(a, x.cpu().numpy())
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


@pytest.mark.parametrize("name,index", [("spheres8_grid7x14", 2), ("spheres64_grid9x18", 1)])
def test_every_kernel_variant_applies_the_same_operator(name, index):
    """Each FP32 variant (symmetric or plain, any tile shape) against the double-FP32 apply."""
    from workloads import make_instance
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
            L.lcp_select_kernel_variant(ctx, v)
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
