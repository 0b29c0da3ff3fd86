"""Checkpoint and resume (lbm_save / lbm_load): k steps, save, load into a fresh
handle built the same way, m more steps, must equal k + m steps run straight
bit for bit. Covered: FP32 and FP16 storage on the sphere duct, BFL (whose link
values hold a partial value) in FP64 on a random geometry, a thin shell, and a
moving body, which resumes at its saved pose. A state is refused by a handle
with another geometry or size."""
import numpy as np
import pytest

from paper_2009_04604_gb300 import build, lbm
from paper_2009_04604_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()
    lbm.load()


def _moving_traj(n=300):
    t = np.arange(n)
    traj = np.zeros((n, 9))
    traj[:, 0] = 24.3 + 4 * np.sin(2 * np.pi * t / n)
    traj[:, 1], traj[:, 2] = 18.1, 17.7
    traj[:, 3] = 4 * 2 * np.pi / n * np.cos(2 * np.pi * t / n)
    return traj


def _make(case, dtype):
    if case == "duct":
        wl = W.sphere_duct_small()
        s = lbm.Simulation(wl["lattice"], wl["dims"], wl["tau"], dtype)
        s.set_options(lbm.BC_ELIBB_F, 1.0, (0, 0, 0), 0)
        s.build_geometry(wl["base"], wl["base_u"], wl["shapes"])
        s.set_launch(32, 4, 3, 2)
        s.init(1.0)
    elif case == "bfl_random":
        flags, q, uw, uw1, tag = W.random_geometry((37, 11, 9), seed=41)
        s = lbm.Simulation(lbm.D3Q19, (37, 11, 9), 0.8, dtype)
        s.set_options(lbm.BC_BFL, 1.0, (1e-4, 0, -1e-4), 0)
        s.set_geometry(flags, q, uw, uw1, tag)
        s.init(1.0, (0.01, 0.005, 0.0))
    elif case == "shell":
        s = lbm.Simulation(lbm.D2Q9, (48, 40, 1), 0.8, dtype)
        s.set_options(lbm.BC_ELIBB_FQ, 1.0, (2e-5, 0, 0), 0)
        s.build_geometry(None, None, [dict(type="shell", tag=1, c=(23.4, 19.7, 0), r=(12.7, 0, 0),
                                           om=(0, 0, 0.002), om1=(0, 0, 0.002))])
        s.init(1.0)
    else:  # moving body
        s = lbm.Simulation(lbm.D3Q19, (48, 36, 36), 0.8, dtype)
        s.set_options(lbm.BC_ELIBB_F, 1.0, (1e-5, 0, 0), 0)
        s.build_geometry(None, None, [dict(type="sphere", tag=0, c=(6.2, 5.1, 5.3), r=(3.5, 0, 0))])
        s.set_moving_body(dict(type="sphere", tag=1, r=(5.2, 0, 0)), _moving_traj(), 0)
        s.init(1.0)
    return s


@pytest.mark.parametrize("case,dtype", [("duct", lbm.F32), ("duct", lbm.F16), ("bfl_random", lbm.F64),
                                        ("shell", lbm.F64), ("moving", lbm.F32)])
def test_resume_is_bitwise(case, dtype):
    k, m = 37, 45  # an odd k leaves the state in the second buffer
    a = _make(case, dtype)
    a.step(k)
    blob = a.save()
    a.step(m)
    b = _make(case, dtype)
    b.load(blob)
    b.step(m)
    fa, fb = a.get_populations(), b.get_populations()
    assert np.array_equal(fa, fb), np.abs(fa - fb).max()
    assert np.array_equal(a.get_geometry()[0], b.get_geometry()[0])
    if case == "moving":
        assert np.array_equal(a.wall_force(1), b.wall_force(1))
    a.close()
    b.close()


def test_load_refuses_another_geometry():
    a = _make("duct", lbm.F32)
    a.step(3)
    blob = a.save()
    wl = W.sphere_duct_small()
    other = lbm.Simulation(wl["lattice"], wl["dims"], wl["tau"], lbm.F32)
    other.set_options(lbm.BC_ELIBB_F, 1.0, (0, 0, 0), 0)
    shapes = [dict(s, c=(17.0, 16.0, 16.0)) for s in wl["shapes"]]  # the sphere moved by one node
    other.build_geometry(wl["base"], wl["base_u"], shapes)
    with pytest.raises(lbm.LBMError):
        other.load(blob)
    small = lbm.Simulation(lbm.D3Q19, (32, 32, 32), 0.7, lbm.F32)
    small.set_geometry(np.zeros(32 ** 3, np.uint8))
    with pytest.raises(lbm.LBMError):
        small.load(blob)
    with pytest.raises(lbm.LBMError):
        a.load(blob[:100])  # truncated
    a.load(blob)  # its own state loads back
    a.close()
    other.close()
    small.close()
