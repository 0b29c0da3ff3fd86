"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

FP64 storage must match the oracle within 1e-12 relative L2. Integer link and
flag logic must match bit for bit. Reduced-precision storage must stay within
the per-dtype velocity bounds: 1e-5 for FP32, 1e-3 for FP16, BF16 reported.
"""
import numpy as np
import pytest

import oracle
from oracle import analytic as A
from paper_2009_04604_gb300 import build, lbm
from paper_2009_04604_gb300 import workloads as W

from gpu_helpers import gpu_sim, oracle_params, oracle_shapes, perm, rel_l2, to_lib, to_oracle

pytestmark = pytest.mark.gpu

TOL_F64 = 1e-12


@pytest.fixture(scope="module", autouse=True)
def _lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()
    oracle.build()
    lbm.load()


BCS = [lbm.BC_ELIBB_F, lbm.BC_ELIBB_FQ, lbm.BC_BFL, lbm.BC_HWBB]


def _random_case(lat, dims, seed, xshift=0, force=(0.0, 0.0, 0.0), tau=0.8):
    Q = {lbm.D2Q9: 9, lbm.D3Q19: 19, lbm.D3Q27: 27}[lat]
    N = int(np.prod(dims))
    flags, q, uw, uw1, tag = W.random_geometry(dims, seed=seed, Q=Q)
    if lat == lbm.D2Q9:
        uw[..., 2] = 0.0
        uw1[..., 2] = 0.0
    wl = dict(lattice=lat, dims=tuple(dims), tau=tau, xshift=xshift, force=force, rho0=1.0)
    rho, u, xi = W.random_fields(N, seed=seed + 1, Q=Q, two_d=lat == lbm.D2Q9)
    return wl, flags, q, uw, uw1, tag, rho, u, xi


@pytest.mark.parametrize("bc", BCS)
@pytest.mark.parametrize("lat,dims,xshift,force", [
    (lbm.D2Q9, (45, 23, 1), 0, (0.0, 0.0, 0.0)),
    (lbm.D2Q9, (64, 17, 1), 5, (1e-4, -2e-4, 0.0)),
    (lbm.D3Q19, (37, 11, 9), 0, (1e-4, 5e-5, -1e-4)),
    (lbm.D3Q19, (32, 8, 5), 0, (0.0, 0.0, 0.0)),
])
def test_random_geometry_f64_parity(bc, lat, dims, xshift, force):
    """Random walls, open nodes, q in (0,1] (including 1/2, 1 and below the FQ cutoff),
    moving walls, tags: populations, mass and per-tag force after 12 steps."""
    wl, flags, q, uw, uw1, tag, rho, u, xi = _random_case(lat, dims, 11 + bc, xshift, force)
    P = perm(lat)
    p = oracle_params(wl, bc)
    f0 = oracle.init_eq(p, flags, rho, u) * (1.0 + xi)
    f0[flags != 0] = 0.0
    s = gpu_sim(wl, lbm.F64, bc)
    s.set_geometry(flags, to_lib(q, P), to_lib(uw, P), to_lib(uw1, P), to_lib(tag, P))
    s.set_populations(to_lib(f0, P))
    # the state round-trips exactly
    assert np.abs(to_oracle(s.get_populations(), P)[flags == 0] - f0[flags == 0]).max() < 1e-15
    f = f0
    flink = None
    for k in range(12):
        f, flink = oracle.step(p, flags, f, q, uw, uw1, want_force=True)
    s.step(12)
    g = to_oracle(s.get_populations(), P)
    fl = flags == 0
    assert rel_l2(g[fl], f[fl]) < TOL_F64
    assert abs(s.mass() - oracle.mass(p, flags, f)) / oracle.mass(p, flags, f) < 1e-13
    for tg in (-1, 0, 3, 7):
        ref = flink.reshape(-1, 3) if tg < 0 else flink[tag == tg]
        ref = ref.sum(0)
        got = s.wall_force(tg)
        assert np.abs(got - ref).max() <= 1e-11 * max(1.0, np.abs(ref).max()), (tg, got, ref)
    s.close()


def _upstream(dims, c, xshift=0):
    """Brute-force index of node n - c_j for every node and direction."""
    nx, ny, nz = dims
    X = np.arange(nx * ny * nz)
    x, y, z = X % nx, (X // nx) % ny, X // (nx * ny)
    out = np.empty((X.size, len(c)), np.int64)
    for j in range(len(c)):
        xs, ys, zs = x - c[j, 0], y - c[j, 1], z - c[j, 2]
        ys = np.where(xs < 0, ys + xshift, np.where(xs >= nx, ys - xshift, ys))
        out[:, j] = (xs % nx) + nx * ((ys % ny) + ny * (zs % nz))
    return out


def test_geometry_roundtrip_and_counts():
    """Explicit geometry round-trips; wall links are exactly the fluid->solid links."""
    wl, flags, q, uw, uw1, tag, *_ = _random_case(lbm.D3Q19, (33, 7, 6), 3)
    P = perm(lbm.D3Q19)
    s = gpu_sim(wl, lbm.F64)
    s.set_geometry(flags, to_lib(q, P), to_lib(uw, P), to_lib(uw1, P), to_lib(tag, P))
    fl2, q2, uw2, uw12, tag2 = s.get_geometry()
    assert (fl2 == flags).all()
    c, _ = lbm.lattice_info(lbm.D3Q19)
    up = _upstream(wl["dims"], c)
    wall = (flags[:, None] == 0) & (flags[up] == 1)
    assert np.array_equal(q2 > 0, wall)
    ql = to_lib(q, P)
    assert np.array_equal(q2[wall], ql[wall])
    assert np.array_equal(uw2[wall], to_lib(uw, P)[wall])
    assert np.array_equal(uw12[wall], to_lib(uw1, P)[wall])
    assert np.array_equal(tag2[wall], to_lib(tag, P)[wall])
    nf, nb, nl = s.counts()
    assert nf == int((flags == 0).sum())
    assert nl == int(wall.sum())
    openl = (flags[:, None] == 0) & (flags[up] == 2)
    assert nb == int((wall | openl).any(1).sum())
    s.close()


SHAPE_CASES = {
    "inclined_channel": lambda: W.inclined_channel(),
    "cylinders64": lambda: W.circular_couette(64),
    "cylinders_offcentre": lambda: W.circular_couette(50, centre=24.37),
    "sphere_duct_small": lambda: W.sphere_duct_small(),
    "ellipsoids": lambda: dict(lattice=lbm.D3Q19, dims=(40, 30, 20), tau=0.7, xshift=0, force=(0, 0, 0),
                               base=None, base_u=None, rho0=1.0,
                               shapes=[dict(type="ellipsoid", tag=2, c=(12.3, 14.1, 9.7), r=(6.5, 4.2, 3.3),
                                            v=(0.01, 0.0, -0.003), om=(0.0, 0.001, 0.002),
                                            v1=(0.011, 0.0, -0.003), om1=(0.0, 0.001, 0.002)),
                                       dict(type="sphere", tag=3, c=(27.6, 13.2, 10.1), r=(5.9, 0, 0))]),
}


@pytest.mark.parametrize("case", sorted(SHAPE_CASES))
@pytest.mark.parametrize("dtype", [lbm.F64, lbm.F32])
def test_link_geometry_kernel_parity(case, dtype):
    """Device link geometry vs the oracle: flags bit for bit, q and u_w to rounding."""
    wl = SHAPE_CASES[case]()
    P = perm(wl["lattice"])
    p = oracle_params(wl)
    of, oq, ouw, ouw1, otag = oracle.geometry(p, wl["base"], wl["base_u"], oracle_shapes(wl["shapes"]))
    s = gpu_sim(wl, dtype)
    s.build_geometry(wl["base"], wl["base_u"], wl["shapes"])
    gf, gq, guw, guw1, gtag = s.get_geometry()
    assert np.array_equal(gf, of)
    # the library keeps wall links only (links into OPEN nodes carry no q)
    c, _, _ = oracle.lattice(wl["lattice"])
    up = _upstream(wl["dims"], c, wl.get("xshift", 0))
    oqw = np.where(of[up] == oracle.SOLID, oq, 0.0)
    gq_o = to_oracle(gq, P)
    assert np.array_equal(gq_o > 0, oqw > 0)
    tol = 0.0 if dtype == lbm.F64 else 6e-8
    assert np.abs(gq_o - oqw).max() <= tol
    wall = oqw > 0
    assert np.abs(to_oracle(guw, P)[wall] - ouw[wall]).max() <= (0.0 if dtype == lbm.F64 else 1e-9)
    assert np.abs(to_oracle(guw1, P)[wall] - ouw1[wall]).max() <= (0.0 if dtype == lbm.F64 else 1e-9)
    assert np.array_equal(to_oracle(gtag, P)[wall], otag[wall])
    s.close()


def _run_pair(wl, bc, dtype, steps, init_u=None):
    """Same workload on the oracle and the GPU from an equilibrium start."""
    P = perm(wl["lattice"])
    p = oracle_params(wl, bc)
    of, oq, ouw, ouw1, otag = oracle.geometry(p, wl["base"], wl["base_u"], oracle_shapes(wl["shapes"]))
    f = oracle.init_eq(p, of, None, init_u)
    s = gpu_sim(wl, dtype, bc)
    s.build_geometry(wl["base"], wl["base_u"], wl["shapes"])
    if init_u is None:
        s.init(wl.get("rho0", 1.0))
    else:
        s.set_populations(to_lib(f, P))
    for _ in range(steps):
        f = oracle.step(p, of, f, oq, ouw, ouw1)
    s.step(steps)
    return s, p, of, f, P


def test_inclined_channel_f64_parity_and_analytic():
    """Config 1: D2Q9 FP64, tau 0.8, g = 1e-6 along a 30 degree channel, 5000 steps."""
    wl = W.inclined_channel()
    s, p, of, f, P = _run_pair(wl, lbm.BC_ELIBB_F, lbm.F64, wl["steps"])
    g = to_oracle(s.get_populations(), P)
    fl = of == 0
    assert rel_l2(g[fl], f[fl]) < TOL_F64
    rho, u = s.macros()
    u = u.cpu().numpy()
    _, uo = oracle.macros(p, of, f)
    assert rel_l2(u[fl], uo[fl]) < TOL_F64
    # against the transient channel solution (walls at v = -20, +20)
    N = len(of)
    X = np.arange(N)
    x, y = X % 52, X // 52
    v = wl["channel_nrm"][0] * x + wl["channel_nrm"][1] * y - wl["channel_off"]
    v = v - wl["channel_period"] * np.floor(v / wl["channel_period"] + 0.5)
    d = np.array(wl["channel_dir"])
    nu = (wl["tau"] - 0.5) / 3.0
    uth = A.poiseuille_transient(v[fl] + 20.0, wl["steps"], 40.0, wl["g"], nu)
    assert A.rrse(u[fl] @ d, uth) < 2e-2
    s.close()


@pytest.mark.parametrize("dtype,bound", [(lbm.F64, 1e-3), (lbm.F32, 1e-3)])
def test_inclined_channel_steady_parabola(dtype, bound):
    """Config 1 to steady state on the GPU (30000 steps): the body-force
    parabola across the 30-degree channel on the sheared-periodic lattice, to
    the same second-order error as the oracle (relative RMS 4.7e-4), and no flow
    across the channel."""
    wl = W.inclined_channel()
    s = gpu_sim(wl, dtype, lbm.BC_ELIBB_F)
    s.build_geometry(wl["base"], wl["base_u"], wl["shapes"])
    s.init(wl["rho0"])
    s.step(30000)
    flags = s.get_geometry()[0]
    _, u = s.macros()
    u = u.cpu().numpy()
    s.close()
    X = np.arange(flags.size)
    x, y = X % 52, X // 52
    v = wl["channel_nrm"][0] * x + wl["channel_nrm"][1] * y - wl["channel_off"]
    v = v - wl["channel_period"] * np.floor(v / wl["channel_period"] + 0.5)
    fl = flags == 0
    sc = v[fl] + 20.0
    nu = (wl["tau"] - 0.5) / 3.0
    uth = wl["g"] / (2.0 * nu) * sc * (40.0 - sc)
    err = A.rrse(u[fl] @ np.array(wl["channel_dir"]), uth)
    print(f"inclined channel, steady: rRSE {err:.3e}")
    assert err < bound
    assert np.abs(u[fl] @ np.array(wl["channel_nrm"])).max() < 1e-3 * uth.max()


@pytest.mark.parametrize("bc", [lbm.BC_ELIBB_F, lbm.BC_ELIBB_FQ, lbm.BC_BFL])
def test_circular_couette_parity(bc):
    """Config 2 at L = 64: FP64 parity, and FP32 storage within 1e-5 of the FP64 oracle."""
    wl = W.circular_couette(64, tau=0.8)
    steps = 600
    s, p, of, f, P = _run_pair(wl, bc, lbm.F64, steps)
    fl = of == 0
    assert rel_l2(to_oracle(s.get_populations(), P)[fl], f[fl]) < TOL_F64
    s.close()
    s32 = gpu_sim(wl, lbm.F32, bc)
    s32.build_geometry(None, None, wl["shapes"])
    s32.init(1.0)
    s32.step(steps)
    _, u32 = s32.macros()
    _, uo = oracle.macros(p, of, f)
    assert rel_l2(u32.cpu().numpy()[fl], uo[fl]) < 1e-5
    s32.close()


@pytest.mark.parametrize("dtype,bound", [(lbm.F64, TOL_F64), (lbm.F32, 1e-5), (lbm.F16, 1e-3), (lbm.BF16, 2e-2)])
def test_sphere_duct_downscale(dtype, bound):
    """Config 3 downscale 64x32x32, sphere R = 4: velocity and drag vs the FP64 oracle."""
    wl = W.sphere_duct_small()
    steps = 300
    s, p, of, f, P = _run_pair(wl, lbm.BC_ELIBB_F, dtype, steps)
    fl = of == 0
    _, u = s.macros()
    _, uo = oracle.macros(p, of, f)
    err = rel_l2(u.cpu().numpy()[fl], uo[fl])
    assert err < bound, err
    of_, oq, ouw, ouw1, otag = oracle.geometry(p, wl["base"], wl["base_u"], oracle_shapes(wl["shapes"]))
    _, flink = oracle.step(p, of, f, oq, ouw, ouw1, want_force=True)
    s.step(1)
    drag = s.wall_force(1)
    ref = flink[otag == 1].sum(0)
    assert abs(drag[0] - ref[0]) / abs(ref[0]) < max(bound * 10, 1e-11)
    s.close()


def test_edge_cases():
    """1x1 periodic D2Q9, a fully solid box, a box with no boundary, nx = 1 channel."""
    for lat, dims in [(lbm.D2Q9, (1, 1, 1)), (lbm.D3Q19, (1, 1, 1)), (lbm.D3Q19, (3, 2, 1))]:
        wl = dict(lattice=lat, dims=dims, tau=0.9, xshift=0, force=(1e-5, 0, 0), rho0=1.0)
        N = int(np.prod(dims))
        flags = np.zeros(N, np.uint8)
        Q = {lbm.D2Q9: 9, lbm.D3Q19: 19, lbm.D3Q27: 27}[lat]
        rho, u, xi = W.random_fields(N, seed=5, Q=Q, two_d=lat == lbm.D2Q9)
        p = oracle_params(wl)
        f = oracle.init_eq(p, flags, rho, u) * (1 + xi)
        P = perm(lat)
        s = gpu_sim(wl, lbm.F64)
        s.set_geometry(flags)
        s.set_populations(to_lib(f, P))
        for _ in range(7):
            f = oracle.step(p, flags, f)
        s.step(7)
        assert rel_l2(to_oracle(s.get_populations(), P), f) < TOL_F64
        assert s.counts()[1] == 0
        s.close()
    # fully solid: stepping is a no-op, mass 0
    wl = dict(lattice=lbm.D3Q19, dims=(8, 4, 4), tau=0.7)
    s = gpu_sim(wl, lbm.F32)
    s.set_geometry(np.ones(128, np.uint8))
    s.init(1.0)
    s.step(3)
    assert s.mass() == 0.0
    assert s.counts() == (0, 0, 0)
    s.close()
    # bad q is rejected
    s = gpu_sim(dict(lattice=lbm.D2Q9, dims=(4, 4, 1), tau=0.7), lbm.F32)
    fl = np.zeros(16, np.uint8)
    fl[0] = 1
    with pytest.raises(lbm.LBMError):
        s.set_geometry(fl, np.full((16, 9), 1.5))
    with pytest.raises(lbm.LBMError):
        s.step(1)  # no geometry yet
    s.close()


def test_nonfinite_state_is_reported():
    """A NaN planted in a host copy of the state is found by the FP64 mass reduction
    and reported as LBM_ERR_NONFINITE; the context stays usable."""
    wl = W.sphere_duct_small()
    s = gpu_sim(wl, lbm.F32)
    s.build_geometry(wl["base"], wl["base_u"], wl["shapes"])
    s.init(1.0)
    s.step(3)
    f = s.get_populations()
    fl = s.get_geometry()[0] == 0
    f[np.nonzero(fl)[0][100], 7] = np.nan
    s.set_populations(f)
    with pytest.raises(lbm.LBMError) as e:
        s.mass()
    assert e.value.code == -4
    s.init(1.0)  # recover by re-initialising
    assert np.isfinite(s.mass())
    s.close()


def test_full_size_step_conserves_mass_in_closed_box():
    """Full-size launch shape of the benchmark (256 x 128 x 128, autotuned), closed box
    with static walls and a sphere: half-way walls at rest conserve mass exactly up
    to rounding, a property that holds at any size."""
    wl = W.sphere_duct()
    base = wl["base"].copy()
    base[base == 2] = 1                      # close the outlet
    s = gpu_sim(wl, lbm.F64, lbm.BC_HWBB)
    s.build_geometry(base, None, wl["shapes"])
    s.init(1.0, (0.01, 0.0, 0.0))
    m0 = s.mass()
    s.autotune(2)
    s.step(64)
    m1 = s.mass()
    assert abs(m1 - m0) / m0 < 1e-12, (m0, m1)
    s.close()
