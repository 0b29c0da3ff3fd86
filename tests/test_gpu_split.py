"""The split step (launch variants 9 and 10), and the combined step kernel at 48
and 40 registers (variants 11 and 12), against the combined kernel at 64.

The split step runs the lattice tiles and the boundary-record tiles as two
kernels side by side, each with its own register budget; every node runs the
same per-node code as in the one-node combined kernel (variants 0..3), so the
stored populations must agree bit for bit with variant 3. The saved states are
compared byte for byte after direct launches and graph replays, on geometries
that reach every part of the step: inlet, outlet and walls of a duct; random
q, moving walls, open links and a body force; the sheared x wrap; a moving
body (its records are rebuilt every step and stay in the boundary kernel); a
thin shell (its nodes are relaxed by the boundary kernel); D3Q27 with TRT. The
oracle comparison at these launches is in test_gpu_timed_launch.py and
test_gpu_trt_unified.py.
"""
import numpy as np
import pytest

from paper_2009_04604_gb300 import build, lbm
from paper_2009_04604_gb300 import workloads as W

pytestmark = pytest.mark.gpu

HEADER = 128  # bytes of the lbm_save header before the raw populations


@pytest.fixture(scope="module", autouse=True)
def _lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()
    lbm.load()


def _make(case, dtype, stream=None):
    if case == "duct":
        wl = W.sphere_duct_small()
        s = lbm.Simulation(wl["lattice"], wl["dims"], wl["tau"], dtype, stream=stream)
        s.set_options(lbm.BC_ELIBB_FQ, 1.0, (0, 0, 0), 0)
        s.build_geometry(wl["base"], wl["base_u"], wl["shapes"])
        s.init(1.0)
    elif case in ("random3d", "random2d_shear", "random27_trt"):
        lat, dims, xshift = {"random3d": (lbm.D3Q19, (64, 13, 11), 0),
                             "random2d_shear": (lbm.D2Q9, (96, 19, 1), 7),
                             "random27_trt": (lbm.D3Q27, (32, 12, 10), 0)}[case]
        Q = {lbm.D2Q9: 9, lbm.D3Q19: 19, lbm.D3Q27: 27}[lat]
        flags, q, uw, uw1, tag = W.random_geometry(dims, seed=31, Q=Q)
        if lat == lbm.D2Q9:
            uw[..., 2] = 0.0
            uw1[..., 2] = 0.0
        s = lbm.Simulation(lat, dims, 0.9, dtype, stream=stream)
        s.set_options(lbm.BC_ELIBB_FQ if case != "random2d_shear" else lbm.BC_ELIBB_F, 1.0,
                      (1e-5, 2e-5, 0.0), xshift)
        if case == "random27_trt":
            s.set_collision(lbm.COLL_TRT)
        s.set_geometry(flags, q, uw, uw1, tag)
        s.init(1.0, (0.01, -0.005, 0.0))
    elif case == "porous":
        wl = W.porous_with_moving_sphere(n=48, rmin=3.0, rmax=5.0, moving_radius=4.0, amplitude=3.0,
                                         period=300, seed=5, g=1e-5)
        s = lbm.Simulation(lbm.D3Q19, wl["dims"], wl["tau"], dtype, stream=stream)
        s.set_options(lbm.BC_ELIBB_F, 1.0, wl["force"], 0)
        s.build_geometry(None, None, wl["shapes"])
        s.set_moving_body(wl["body"], wl["traj"], 0)
        s.init(1.0)
    else:  # thin shell beside a solid sphere
        s = lbm.Simulation(lbm.D3Q19, (64, 24, 20), 0.7, dtype, stream=stream)
        s.set_options(lbm.BC_ELIBB_F, 1.0, (1e-5, 0.0, -1e-5), 0)
        s.build_geometry(None, None, [
            dict(type="shell", tag=2, c=(30.4, 11.7, 9.6), r=(7.3, 0, 0), v=(4e-3, 0, 0),
                 om=(1e-3, -2e-3, 3e-3), v1=(4e-3, 0, 0), om1=(1e-3, -2e-3, 3.2e-3)),
            dict(type="sphere", tag=3, c=(52.3, 5.1, 14.2), r=(3.1, 0, 0))])
        s.init(1.0)
    return s


CASES = ["duct", "random3d", "random2d_shear", "random27_trt", "porous", "shell"]


@pytest.mark.parametrize("dtype", [lbm.F32, lbm.F16, lbm.BF16])
@pytest.mark.parametrize("case", CASES)
def test_split_step_is_bitwise_the_combined_step(case, dtype):
    ref = _make(case, dtype)
    ref.set_launch(32, 8, 3, 2)
    runs = [_make(case, dtype) for _ in range(4)]
    runs[0].set_launch(32, 8, 9, 1)
    runs[1].set_launch(32, 4, 10, 2)
    runs[2].set_launch(32, 8, 11, 1)  # the combined kernel at 48 and 40 registers
    runs[3].set_launch(32, 8, 12, 2)
    for n in (3, 40):  # direct launches, then a graph replay
        for s in [ref] + runs:
            s.step(n)
    want = ref.save()[HEADER:]
    Fw = ref.wall_force(-1)
    for s in runs:
        assert s.save()[HEADER:] == want, s.get_launch()
        assert np.array_equal(s.wall_force(-1), Fw)
        s.close()
    assert np.isfinite(ref.get_populations()).all()
    ref.close()


def test_split_step_limits():
    s = _make("duct", lbm.F32)
    s.set_launch(64, 4, 9, 1)
    s.set_launch(32, 8, 10, 4)
    with pytest.raises(lbm.LBMError):
        s.set_launch(32, 8, 13, 1)
    s.set_options(lbm.BC_BFL, 1.0, (0, 0, 0), 0)  # one node per thread: BFL keeps the variant
    assert s.get_launch()[2] == 10
    s.step(4)
    s.close()
    d = lbm.Simulation(lbm.D3Q19, (32, 8, 8), 0.8, lbm.F64)
    with pytest.raises(lbm.LBMError):
        d.set_launch(32, 8, 9, 1)
    d.close()


def test_batch_of_split_and_pair_simulations():
    """A batch takes its own one-node launch whatever its simulations are set to
    alone: its tiles follow the batch's block width and variant."""
    import torch
    st = torch.cuda.Stream()
    sims = [_make(c, lbm.F32, st) for c in ("duct", "random3d")]
    sims[0].set_launch(32, 8, 9, 1)
    sims[1].set_launch(32, 4, 8, 1)
    alone = [_make(c, lbm.F32) for c in ("duct", "random3d")]
    for s in alone:
        s.set_launch(32, 4, 3, 1)
    b = lbm.Batch(sims)
    b.set_launch(32, 4, 3, 1)
    b.step(34)
    for s in alone:
        s.step(34)
    for s, t in zip(sims, alone):
        assert s.save()[HEADER:] == t.save()[HEADER:]
    b.close()
    for s in sims + alone:
        s.close()
