"""Host-side arithmetic of bench.py (no GPU): the roofline numerator, the launch
bookkeeping and the committed profile summaries it reads."""
import glob
import json
import os
import re

import bench

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_algorithmic_bytes_of_the_full_size_duct():
    """2 Q s per fluid node, one flag byte per padded node, 4 B per boundary
    record and 4 B per wall link: the 618,132,744 bytes of the FP32 duct line,
    from its node and link counts."""
    nfluid, nb, nwall = 4015427, 162162, 736222
    np_ = bench.padded_nodes((256, 128, 128))
    assert np_ == 256 * 128 * 128
    b = bench.algorithmic_bytes(nfluid, np_, nb, nwall, 19, 4, 4, False)
    assert b == nfluid * 152 + np_ + 4 * nb + 4 * nwall == 618132744
    # FP16: half the population bytes; a moving wall link adds u_w at t and t+1
    assert bench.algorithmic_bytes(nfluid, np_, nb, nwall, 19, 2, 4, False) == b - nfluid * 76
    assert bench.algorithmic_bytes(1, 1, 1, 1, 19, 4, 4, True) - bench.algorithmic_bytes(1, 1, 1, 1, 19, 4, 4, False) == 24
    assert bench.padded_nodes((48, 48, 48)) == 64 * 48 * 48  # rows padded to a multiple of 32


def test_job_throughput_of_replicas():
    # two ranks of 1000 fluid nodes, 10 steps, the slower rank took 20 ms
    assert abs(bench.job_mlups(2, 1000, 10, 20.0) - 1.0) < 1e-12


def test_launch_bookkeeping():
    for v in (9, 10):
        t = {"bx": 32, "by": 4, "variant": v, "tiles": 2}
        assert bench.is_split(t)
        assert bench.profile_name(t, "f16", "sphere_duct") == "k_lattice_k_boundary_d3q19_f16_sphere_duct"
        assert "k_lattice" in bench.step_kernels(t)
    for v in (0, 3, 4, 8, 11, 12):
        t = {"bx": 32, "by": 4, "variant": v, "tiles": 1}
        assert not bench.is_split(t)
        assert bench.profile_name(t, "f32", "porous_moving") == "k_step_d3q19_f32_porous_moving"
    # a downscaled lattice narrows the block to its rows, at the same threads per block;
    # node pairs (variants 5-8) need rows of two block widths, the others one
    assert bench.clip_launch({"bx": 256, "by": 1, "variant": 12, "tiles": 1}, 64) == (64, 4, 12, 1)
    assert bench.clip_launch({"bx": 128, "by": 1, "variant": 8, "tiles": 1}, 64) == (32, 4, 8, 1)
    assert bench.clip_launch({"bx": 64, "by": 2, "variant": 9, "tiles": 2}, 64) == (64, 2, 9, 2)


def test_committed_profile_summaries():
    """Every profiles/*.json names its kernel, launch, command and DRAM bytes and
    carries the kernel-source hash bench.py compares; each has a summary beside
    it, and no summary names anything but a kernel and a workload."""
    files = sorted(glob.glob(os.path.join(ROOT, "profiles", "*.json")))
    assert files
    for f in files:
        d = json.load(open(f))
        for k in ("kernel", "launch", "command", "dram_bytes_read", "dram_bytes_write",
                  "dram_bytes_per_launch_full_size", "kernel_source_hash"):
            assert k in d, (f, k)
        assert re.fullmatch(r"[0-9a-f]{16}", d["kernel_source_hash"])
        assert d["dram_bytes_per_launch_full_size"] >= d["dram_bytes_read"] + d["dram_bytes_write"] - 1
        assert "--clock-control none" in d["command"]
        name = os.path.basename(f)[:-5]
        assert re.fullmatch(r"k_[a-z_]+_d3q19_(f32|f16|bf16)_[a-z_]+", name), name
    for f in glob.glob(os.path.join(ROOT, "profiles", "*.md")):
        txt = open(f).read()
        assert "--clock-control none" in txt
    assert bench.profiled_traffic("no_such_profile") is None
