"""The two-nodes-per-thread step kernel (launch variants 5..8) gives the
populations of the one-node-per-thread kernel (variant 0). The per-node
arithmetic is the same; only the loads (vector loads plus warp shuffles for the
x-shifted planes) and the stores differ. The compiler may still fuse
multiply-adds differently in the two kernels, so results agree to a few units
in the last place of the storage type."""
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


def _make(case, dtype):
    if case == "duct":
        wl = W.sphere_duct_small()
        s = lbm.Simulation(wl["lattice"], wl["dims"], wl["tau"], dtype)
        s.set_options(lbm.BC_ELIBB_FQ, 1.0, (0, 0, 0), 0)
        s.build_geometry(wl["base"], wl["base_u"], wl["shapes"])
        s.init(1.0)
    elif case in ("random3d", "random2d_shear"):
        # odd row lengths: the last pair of a row holds one node and one pad
        lat, dims, xshift = ((lbm.D3Q19, (47, 13, 11), 0) if case == "random3d"
                             else (lbm.D2Q9, (61, 19, 1), 7))
        Q = {lbm.D2Q9: 9, lbm.D3Q19: 19, lbm.D3Q27: 27}[lat]
        flags, q, uw, uw1, tag = W.random_geometry(dims, seed=23, Q=Q)
        if lat == lbm.D2Q9:
            uw[..., 2] = 0.0
            uw1[..., 2] = 0.0
        s = lbm.Simulation(lat, dims, 0.9, dtype)
        s.set_options(lbm.BC_ELIBB_FQ if case == "random3d" else lbm.BC_ELIBB_F, 1.0,
                      (1e-5, 2e-5, 0.0), xshift)
        s.set_geometry(flags, q, uw, uw1, tag)
        s.init(1.0, (0.01, -0.005, 0.0))
    elif case == "periodic":  # all fluid: every x wrap goes through the pair path
        s = lbm.Simulation(lbm.D3Q19, (64, 9, 7), 0.7, dtype)
        s.set_options(lbm.BC_ELIBB_F, 1.0, (2e-5, 0, 1e-5), 0)
        s.set_geometry(np.zeros(64 * 9 * 7, np.uint8))
        s.init(1.0, (0.02, -0.01, 0.01))
        f = s.get_populations()
        rng = np.random.default_rng(5)
        s.set_populations(f * (1.0 + 0.02 * rng.standard_normal(f.shape)))
    else:  # moving body in a periodic box with a static sphere
        s = lbm.Simulation(lbm.D3Q19, (48, 36, 36), 0.8, dtype)
        s.set_options(lbm.BC_ELIBB_F, 1.0, (1e-5, 0, 0), 0)
        s.build_geometry(None, None, [dict(type="sphere", tag=0, c=(6.2, 5.1, 5.3), r=(3.5, 0, 0))])
        traj = np.zeros((300, 9))
        t = np.arange(300)
        traj[:, 0] = 24.3 + 4 * np.sin(2 * np.pi * t / 300)
        traj[:, 1], traj[:, 2] = 18.1, 17.7
        traj[:, 3] = 4 * 2 * np.pi / 300 * np.cos(2 * np.pi * t / 300)
        s.set_moving_body(dict(type="sphere", tag=1, r=(5.2, 0, 0)), traj, 0)
        s.init(1.0)
    return s


VARIANT = {"duct": 5, "random3d": 6, "random2d_shear": 7, "periodic": 8, "moving": 8}


@pytest.mark.parametrize("dtype", [lbm.F32, lbm.F16, lbm.BF16])
@pytest.mark.parametrize("case", list(VARIANT))
def test_pair_variant_matches_register_variant(case, dtype):
    a, b = _make(case, dtype), _make(case, dtype)
    a.set_launch(32, 8, 0, 1)
    b.set_launch(32, 4, VARIANT[case], 2)  # 64 nodes of a row per warp, 128 threads a block
    for n in (3, 40):  # direct launches, then a graph replay
        a.step(n)
        b.step(n)
    fa, fb = a.get_populations(), b.get_populations()
    assert np.isfinite(fb).all()
    rel = {lbm.F32: 2e-6, lbm.F16: 4e-3, lbm.BF16: 3e-2}[dtype]
    scale = np.abs(fa).max()
    assert np.abs(fa - fb).max() <= rel * scale, np.abs(fa - fb).max()
    if case == "moving":
        Fa, Fb = a.wall_force(1), b.wall_force(1)
        assert np.abs(Fa - Fb).max() <= 10 * rel * np.abs(Fa).max()
    a.close()
    b.close()


def test_pair_variant_limits():
    s = _make("random3d", lbm.F32)  # padded row of 64 nodes
    with pytest.raises(lbm.LBMError):  # a block row must cover whole pairs of the padded row
        s.set_launch(64, 4, 5, 1)
    with pytest.raises(lbm.LBMError):  # variant 8 is compiled for blocks of 128 threads
        s.set_launch(32, 8, 8, 1)
    s.set_launch(32, 4, 8, 1)
    s.set_launch(32, 8, 6, 1)
    s.set_options(lbm.BC_BFL, 1.0, (0, 0, 0), 0)  # BFL moves the launch back to variant 0
    assert s.get_launch()[2] == 0
    with pytest.raises(lbm.LBMError):
        s.set_launch(32, 8, 5, 1)
    s.step(2)
    s.close()
    d = lbm.Simulation(lbm.D3Q19, (32, 8, 8), 0.8, lbm.F64)
    with pytest.raises(lbm.LBMError):
        d.set_launch(32, 8, 5, 1)
    d.close()
