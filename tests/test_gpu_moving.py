"""Moving body: per-step link geometry on the device and refill of fresh nodes,
against the oracle rebuilding its whole geometry every step (FP64, 1e-12)."""
import math

import numpy as np
import pytest

import oracle
from paper_2009_04604_gb300 import build, lbm

from gpu_helpers import oracle_shapes, perm, rel_l2, to_oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()
    oracle.build()
    lbm.load()


DIMS = (48, 36, 36)
STATIC = [dict(type="sphere", tag=0, c=(6.2, 5.1, 5.3), r=(3.5, 0, 0)),
          dict(type="sphere", tag=0, c=(42.1, 30.4, 29.8), r=(3.5, 0, 0))]


def trajectory(n, c0=(24.3, 18.1, 17.7), amp=4.0, period=300.0):
    """Sinusoidal path along x; peak speed amp * 2 pi / period = 0.084 (Mach 0.15),
    and over the 50 tested steps the body sweeps about 3.5 nodes."""
    w = 2 * math.pi / period
    t = np.arange(n)
    traj = np.zeros((n, 9))
    traj[:, 0] = c0[0] + amp * np.sin(w * t)
    traj[:, 1] = c0[1]
    traj[:, 2] = c0[2]
    traj[:, 3] = amp * w * np.cos(w * t)
    return traj


def moving_shape(body, traj, k):
    n = len(traj)
    p, p1 = traj[k % n], traj[(k + 1) % n]
    return dict(body, c=tuple(p[:3]), v=tuple(p[3:6]), om=tuple(p[6:9]), v1=tuple(p1[3:6]), om1=tuple(p1[6:9]))


@pytest.mark.parametrize("body,bc", [
    (dict(type="sphere", tag=1, r=(5.2, 0, 0)), lbm.BC_ELIBB_F),
    (dict(type="ellipsoid", tag=1, r=(5.6, 4.1, 3.7)), lbm.BC_ELIBB_FQ),
])
def test_moving_body_f64_parity(body, bc):
    steps = 50
    traj = trajectory(300)
    force = (1e-5, 0.0, 0.0)
    wl = dict(lattice=lbm.D3Q19, dims=DIMS, tau=0.8, xshift=0, force=force, rho0=1.0)
    obc = {lbm.BC_ELIBB_F: oracle.BC_ELIBB_F, lbm.BC_ELIBB_FQ: oracle.BC_ELIBB_FQ}[bc]
    p = oracle.params(lbm.D3Q19, DIMS, 0.8, bc=obc, force=force)
    P = perm(lbm.D3Q19)
    # oracle
    flags, *_ = oracle.geometry(p, None, None, oracle_shapes(STATIC + [moving_shape(body, traj, 0)]))
    f = oracle.init_eq(p, flags)
    flink = None
    for t in range(steps):
        fl_t, q, uw, uw1, tag = oracle.geometry(p, None, None, oracle_shapes(STATIC + [moving_shape(body, traj, t)]))
        f, flink = oracle.step(p, fl_t, f, q, uw, uw1, want_force=True)
        fl_n, *_ = oracle.geometry(p, None, None, oracle_shapes(STATIC + [moving_shape(body, traj, t + 1)]))
        un = np.tile(traj[(t + 1) % len(traj), 3:6], (fl_n.size, 1))
        oracle.refill(p, fl_t, fl_n, un, f)
        flags = fl_n
    # GPU
    s = lbm.Simulation(lbm.D3Q19, DIMS, 0.8, lbm.F64)
    s.set_options(bc, 1.0, force, 0)
    s.build_geometry(None, None, STATIC)
    s.set_moving_body(body, traj, 0)
    s.init(1.0)
    s.step(steps)
    gflags = s.get_geometry()[0]
    assert np.array_equal(gflags, flags)
    fl = flags == 0
    g = to_oracle(s.get_populations(), P)
    assert rel_l2(g[fl], f[fl]) < 1e-12
    ref = flink[tag == 1].sum(0)
    got = s.wall_force(1)
    assert np.abs(got - ref).max() <= 1e-10 * np.abs(ref).max(), (got, ref)
    s.close()


def test_moving_body_f32_runs_and_rejects_bad_regions():
    traj = trajectory(300)
    body = dict(type="sphere", tag=1, r=(5.2, 0, 0))
    s = lbm.Simulation(lbm.D3Q19, DIMS, 0.8, lbm.F32)
    s.set_options(lbm.BC_ELIBB_F, 1.0, (1e-5, 0, 0), 0)
    s.build_geometry(None, None, STATIC)
    s.set_moving_body(body, traj, 0)
    s.init(1.0)
    s.step(80)  # graph path with the per-step body geometry
    _, u = s.macros()
    assert bool(np.isfinite(u.cpu().numpy()).all())
    with pytest.raises(lbm.LBMError):
        s.set_options(lbm.BC_BFL, 1.0, (0, 0, 0), 0)
    s.close()
    # a region that overlaps a static solid is refused
    s = lbm.Simulation(lbm.D3Q19, DIMS, 0.8, lbm.F32)
    s.build_geometry(None, None, [dict(type="sphere", tag=0, c=(24.0, 18.0, 26.5), r=(3.0, 0, 0))])
    with pytest.raises(lbm.LBMError):
        s.set_moving_body(body, traj, 0)
    s.close()


@pytest.mark.parametrize("dtype,bound", [(lbm.F64, 1e-12), (lbm.F32, 1e-5), (lbm.F16, 1e-3)])
def test_porous_moving_sphere_downscale(dtype, bound):
    """Porous medium with a moving sphere (downscale of the 384^3 configuration):
    static spheres from random sequential addition, a sphere on a sinusoidal path,
    body force; velocity against the FP64 oracle."""
    from paper_2009_04604_gb300 import workloads as W
    wl = W.porous_with_moving_sphere(n=48, rmin=3.0, rmax=5.0, moving_radius=4.0, amplitude=3.0,
                                     period=300, seed=5, g=1e-5)
    steps = 20
    traj, body = wl["traj"], wl["body"]
    p = oracle.params(lbm.D3Q19, wl["dims"], wl["tau"], bc=oracle.BC_ELIBB_F, force=wl["force"])
    stat = oracle_shapes(wl["shapes"])
    flags, *_ = oracle.geometry(p, None, None, stat + oracle_shapes([moving_shape(body, traj, 0)]))
    f = oracle.init_eq(p, flags)
    for t in range(steps):
        fl_t, q, uw, uw1, tag = oracle.geometry(p, None, None, stat + oracle_shapes([moving_shape(body, traj, t)]))
        f = oracle.step(p, fl_t, f, q, uw, uw1)
        fl_n, *_ = oracle.geometry(p, None, None, stat + oracle_shapes([moving_shape(body, traj, t + 1)]))
        oracle.refill(p, fl_t, fl_n, np.tile(traj[(t + 1) % len(traj), 3:6], (fl_n.size, 1)), f)
        flags = fl_n
    _, uo = oracle.macros(p, flags, f)
    s = lbm.Simulation(lbm.D3Q19, wl["dims"], wl["tau"], dtype)
    s.set_options(lbm.BC_ELIBB_F, 1.0, wl["force"], 0)
    s.build_geometry(None, None, wl["shapes"])
    s.set_moving_body(body, traj, 0)
    s.init(1.0)
    s.step(steps)
    assert np.array_equal(s.get_geometry()[0], flags)
    _, u = s.macros()
    fl = flags == 0
    err = rel_l2(u.cpu().numpy()[fl], uo[fl])
    assert err < bound, err
    s.close()
