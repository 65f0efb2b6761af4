"""Host-side choices of the bench (no GPU): the low-fidelity operator for a
workload grid and the kernel names it reports."""
import bench


def test_lowfi_auto_picks_coarse_grid_or_rpy():
    # 11 x 22 workload: the 8 x 16 boundary-integral grid, loose FP32 solves, approximate init
    assert bench.lowfi_overrides("auto", 11) == {"lowfi_n_theta": 8, "lowfi_n_phi": 16, "lowfi_tol": 1e-4,
                                                 "init_forcing": 1e-3}
    assert bench.lowfi_overrides("auto", 9) == {"lowfi_n_theta": 6, "lowfi_n_phi": 12, "lowfi_tol": 1e-4,
                                                "init_forcing": 1e-3}
    # grids coarser than 6 x 12 would not resolve neighbouring spheres: RPY
    assert bench.lowfi_overrides("auto", 8) == {}
    assert bench.lowfi_overrides("auto", 7) == {}


def test_lowfi_explicit_specs():
    assert bench.lowfi_overrides("rpy", 11) == {}
    assert bench.lowfi_overrides("6x12") == {"lowfi_n_theta": 6, "lowfi_n_phi": 12}
    assert bench.lowfi_overrides("8X16") == {"lowfi_n_theta": 8, "lowfi_n_phi": 16}


def test_kernel_names_and_traffic_guard():
    assert bench.pair32_kernel_name("t2c8") == "k_pair32"
    assert bench.pair32_kernel_name("sym_a4") == "k_pair32_sym_a4"
    # every recorded traffic figure names a kernel whose device code can be hashed (the bench
    # reports the figure only while that hash is unchanged)
    for kname, info in bench.PAIR32_TRAFFIC.items():
        assert info["bytes_per_launch"] > 0
        h = bench.source_sha1(kname)
        assert len(h) == 40 and int(h, 16) >= 0, kname


def test_batched_and_serving_low_fidelity_per_instance():
    """Batched and serving modes: the coarse grid for instances of at least --lowfi-min-bodies
    spheres where it resolves neighbours (9 x 18 -> 6 x 12), RPY for 7 x 14 spheres and below
    the threshold; the description says which."""
    import argparse

    from workloads import make_instance
    big = make_instance("spheres64_grid9x18", 0)          # 9 x 18 nodes
    small = make_instance("spheres8_grid7x14", 0)         # 7 x 14 nodes
    args = argparse.Namespace(lowfi="auto", lowfi_min_bodies=8)
    assert bench.instance_lowfi(args, big)["lowfi_n_theta"] == 6
    assert bench.instance_lowfi(args, small) == {}
    assert "coarse grid" in bench.batch_lowfi_description(args)
    args.lowfi_min_bodies = 100
    assert bench.instance_lowfi(args, big) == {}
    args.lowfi_min_bodies = 10 ** 9
    assert bench.batch_lowfi_description(args) == "rpy"
    args = argparse.Namespace(lowfi="rpy", lowfi_min_bodies=8)
    assert bench.instance_lowfi(args, big) == {} and bench.batch_lowfi_description(args) == "rpy"


def test_host_cpu_names_the_processor():
    name = bench.host_cpu()
    assert isinstance(name, str) and name.strip()
