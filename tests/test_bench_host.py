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
