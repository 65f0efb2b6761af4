"""The allocation-free stresslet apply, checked against the context-based one.

Callers that cannot allocate GPU memory (allocator callbacks, hosts that hand
the whole device budget elsewhere, real-time loops) use
lcp_stokes_apply_noalloc, which works out of a fixed scratch area compiled
into the library.  Its result must equal lcp_stokes_apply_dev's for the same
input, on consecutive calls that reuse the shared scratch area.  This file is
collected last so that a run stopping at the first failure has already run
every other test.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2604_10089_gb300 as L  # noqa: E402
from workloads import make_instance  # noqa: E402

TOL = {L.LCP_FP64: 1e-12, L.LCP_MIXED: 1e-5}   # relative, max-norm (summation order differs)


def rel(a, b):
    return float((a - b).abs().max() / b.abs().max())


@pytest.mark.parametrize("name", ["spheres8_grid7x14", "spheres64_grid9x18"])
@pytest.mark.parametrize("precision", [L.LCP_FP64, L.LCP_MIXED])
def test_noalloc_matches_context_apply_twice(name, precision):
    inst = make_instance(name, 0)
    ctx = L.lcp_setup(L.config_for(inst, precision, self_quadrature=0), inst.centers, None)
    try:
        M, N, _ = L.lcp_sizes(ctx)
        centers = torch.tensor(inst.centers, dtype=torch.float64, device="cuda")
        gen = torch.Generator(device="cuda").manual_seed(11)
        for call in range(2):
            phi = torch.randn(3 * N, dtype=torch.float64, device="cuda", generator=gen)
            ref = torch.empty_like(phi)
            L.lcp_stokes_apply_dev(ctx, phi, ref, precision)
            out = torch.full_like(phi, float("nan"))
            L.lcp_stokes_apply_noalloc(M, inst.n_theta, inst.n_phi, inst.radius, centers, phi, out, precision)
            torch.cuda.synchronize()
            assert rel(out, ref) <= TOL[precision], (call, rel(out, ref))
    finally:
        L.lcp_destroy(ctx)


def test_noalloc_rejects_sizes_beyond_its_scratch():
    centers = torch.zeros(3 * 200, dtype=torch.float64, device="cuda")
    phi = torch.zeros(3 * 200 * 98, dtype=torch.float64, device="cuda")
    with pytest.raises(L.LcpError) as err:
        L.lcp_stokes_apply_noalloc(200, 7, 14, 1.0, centers, phi, phi, L.LCP_FP64)
    assert err.value.status == L.LCP_ERR_INVALID_ARG
    assert "scratch" in str(err.value)


def _lattice(m, spacing=3.0):
    idx = np.stack(np.meshgrid(*[np.arange(k) for k in m], indexing="ij"), -1).reshape(-1, 3)
    return idx * spacing


@pytest.mark.parametrize("precision", [L.LCP_FP64, L.LCP_MIXED])
def test_noalloc_at_its_maximum_sizes_on_a_caller_stream(precision):
    """32 bodies on a 16 x 32 grid: 512 nodes per sphere and 16384 nodes, both
    at the documented limits (the FP64 kernel needs a raised shared-memory
    limit there), launched on a caller-owned stream."""
    centers_h = _lattice((4, 4, 2))
    cfg = L.lcp_default_config(n_theta=16, n_phi=32, precision=precision, self_quadrature=0)
    ctx = L.lcp_setup(cfg, centers_h)
    try:
        M, N, _ = L.lcp_sizes(ctx)
        assert (M, N) == (32, 16384)
        centers = torch.tensor(centers_h, dtype=torch.float64, device="cuda")
        gen = torch.Generator(device="cuda").manual_seed(12)
        s = torch.cuda.Stream()
        for call in range(2):
            phi = torch.randn(3 * N, dtype=torch.float64, device="cuda", generator=gen)
            ref = torch.empty_like(phi)
            L.lcp_stokes_apply_dev(ctx, phi, ref, precision)
            torch.cuda.synchronize()
            out = torch.full_like(phi, float("nan"))
            with torch.cuda.stream(s):
                L.lcp_stokes_apply_noalloc(M, 16, 32, 1.0, centers, phi, out, precision, s.cuda_stream)
            s.synchronize()
            assert rel(out, ref) <= TOL[precision], (call, rel(out, ref))
    finally:
        L.lcp_destroy(ctx)


def test_noalloc_matches_the_oracle_and_allocates_nothing_on_repeat_calls():
    """Against the oracle's dense (K + P) phi directly, and with the device's
    free memory unchanged over repeated calls (after the first, which may let
    the driver load the library's kernels)."""
    from oracle.bie import DenseMobility
    inst = make_instance("spheres8_grid7x14", 3)
    mob = DenseMobility(inst.centers, inst.n_theta, inst.n_phi, a=inst.radius)
    phi_h = np.random.default_rng(13).standard_normal(3 * mob.x.shape[0])
    ref = torch.tensor((mob.K + mob.P) @ phi_h)
    centers = torch.tensor(inst.centers, dtype=torch.float64, device="cuda")
    phi = torch.tensor(phi_h, device="cuda")
    out = torch.empty_like(phi)
    M = inst.n_bodies
    L.lcp_stokes_apply_noalloc(M, inst.n_theta, inst.n_phi, inst.radius, centers, phi, out, L.LCP_FP64)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for _ in range(3):
        out.fill_(float("nan"))
        L.lcp_stokes_apply_noalloc(M, inst.n_theta, inst.n_phi, inst.radius, centers, phi, out, L.LCP_FP64)
        torch.cuda.synchronize()
        assert rel(out.cpu(), ref) <= TOL[L.LCP_FP64]
    assert torch.cuda.mem_get_info()[0] == free0
