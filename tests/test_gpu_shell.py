"""Thin shells with fluid on both sides on the GPU (the thin-shell cylinders of
Sec. III.B): link geometry, every boundary rule in FP64, the force counted on
the outer side, launch variants, the batched launch, and thin-shell circular
Couette flow at second order, against the FP64 oracle and the closed form."""
import numpy as np
import pytest

import oracle
from oracle import analytic as A
from paper_2009_04604_gb300 import build, lbm

from gpu_helpers import gpu_sim, oracle_params, perm, rel_l2, to_lib, to_oracle

pytestmark = pytest.mark.gpu

TOL_F64 = 1e-12
ORACLE_SHAPES_SHELL = {"shell": oracle.SHAPE_SHELL, "sphere": oracle.SHAPE_SPHERE}


@pytest.fixture(scope="module", autouse=True)
def _lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()
    oracle.build()
    lbm.load()


def _case(name):
    """A rotating and translating thin shell, a solid sphere beside it, a body force."""
    if name == "d2q9":
        wl = dict(lattice=lbm.D2Q9, dims=(48, 40, 1), tau=0.8, force=(1e-5, -2e-5, 0.0))
        shapes = [dict(type="shell", tag=2, c=(23.3, 19.6, 0.0), r=(12.7, 0, 0),
                       om=(0, 0, 2e-3), om1=(0, 0, 2.1e-3)),
                  dict(type="sphere", tag=3, c=(42.2, 6.3, 0.0), r=(3.1, 0, 0))]
    elif name == "d3q19":
        wl = dict(lattice=lbm.D3Q19, dims=(64, 24, 20), tau=0.7, force=(1e-5, 0.0, -1e-5))
        shapes = [dict(type="shell", tag=2, c=(30.4, 11.7, 9.6), r=(7.3, 0, 0), v=(4e-3, 0, 0),
                       om=(1e-3, -2e-3, 3e-3), v1=(4e-3, 0, 0), om1=(1e-3, -2e-3, 3.2e-3)),
                  dict(type="sphere", tag=3, c=(52.3, 5.1, 14.2), r=(3.1, 0, 0))]
    else:
        wl = dict(lattice=lbm.D3Q27, dims=(24, 20, 20), tau=0.9, force=(0.0, 1e-5, 0.0))
        shapes = [dict(type="shell", tag=2, c=(10.6, 9.7, 10.2), r=(5.6, 0, 0),
                       om=(2e-3, 0, -1e-3), om1=(2e-3, 0, -1e-3))]
    wl["shapes"] = shapes
    return wl


def _oracle_geometry(wl, bc=lbm.BC_ELIBB_F):
    p = oracle_params(wl, bc)
    shapes = []
    for s in wl["shapes"]:
        s = dict(s)
        s["type"] = ORACLE_SHAPES_SHELL[s["type"]]
        shapes.append(s)
    return (p,) + oracle.geometry(p, shapes=shapes, with_shell=True)


def _upstream(dims, c):
    nx, ny, nz = dims
    X = np.arange(nx * ny * nz)
    x, y, z = X % nx, (X // nx) % ny, X // (nx * ny)
    return np.stack([((x - c[j, 0]) % nx) + nx * (((y - c[j, 1]) % ny) + ny * ((z - c[j, 2]) % nz))
                     for j in range(len(c))], 1)


@pytest.mark.parametrize("dtype", [lbm.F64, lbm.F32])
@pytest.mark.parametrize("case", ["d2q9", "d3q19", "d3q27"])
def test_shell_link_geometry_parity(case, dtype):
    """Flags bit for bit, the same wall links (solid and across the shell), q and u_w
    to rounding, tags with the inner side's links at -1."""
    wl = _case(case)
    P = perm(wl["lattice"])
    p, of, oq, ouw, ouw1, otag, oshell = _oracle_geometry(wl)
    s = gpu_sim(wl, dtype)
    s.build_geometry(None, None, wl["shapes"])
    gf, gq, guw, guw1, gtag = s.get_geometry()
    assert np.array_equal(gf, of)
    c, _, _ = oracle.lattice(wl["lattice"])
    up = _upstream(wl["dims"], c)
    wall = (of[:, None] == oracle.FLUID) & ((of[up] == oracle.SOLID) | (oshell > 0))
    assert (oshell > 0).sum() > 100
    gq_o = to_oracle(gq, P)
    assert np.array_equal(gq_o > 0, wall)
    # FP32 link storage rounds the FP64 geometry to nearest: half an ulp, 2^-24 relative
    rel = 0.0 if dtype == lbm.F64 else 2.0 ** -24
    oqw = np.where(wall, oq, 0.0)
    assert (np.abs(gq_o - oqw) <= rel * np.abs(oqw)).all()
    assert (np.abs(to_oracle(guw, P)[wall] - ouw[wall]) <= rel * np.abs(ouw[wall])).all()
    assert (np.abs(to_oracle(guw1, P)[wall] - ouw1[wall]) <= rel * np.abs(ouw1[wall])).all()
    assert np.array_equal(to_oracle(gtag, P)[wall], otag[wall])
    assert (otag[oshell == 2] == -1).all() and (otag[oshell == 1] == 2).all()
    s.close()


ALL_BC = [lbm.BC_ELIBB_F, lbm.BC_ELIBB_FQ, lbm.BC_BFL, lbm.BC_HWBB, lbm.BC_ELIBB_U, lbm.BC_ELIBB_UQ]


def _random_state(p, of, lat, seed):
    c, w, _ = oracle.lattice(lat)
    rng = np.random.default_rng(seed)
    N = len(of)
    u = 0.02 * rng.standard_normal((N, 3))
    if lat == oracle.D2Q9:
        u[:, 2] = 0.0
    rho = 1.0 + 0.01 * rng.standard_normal(N)
    f = oracle.init_eq(p, of, rho, u) * (1.0 + 0.02 * rng.standard_normal((N, len(w))))
    f[of != oracle.FLUID] = 0.0
    return f


@pytest.mark.parametrize("bc", ALL_BC)
@pytest.mark.parametrize("case", ["d2q9", "d3q19", "d3q27"])
def test_shell_f64_parity(case, bc):
    """Populations, mass and per-tag force after 8 steps from a random state."""
    wl = _case(case)
    if bc == lbm.BC_ELIBB_UQ:
        wl["collision"] = lbm.COLL_TRT
    P = perm(wl["lattice"])
    p, of, oq, ouw, ouw1, otag, oshell = _oracle_geometry(wl, bc)
    f = _random_state(p, of, wl["lattice"], 5 + bc)
    s = gpu_sim(wl, lbm.F64, bc)
    s.build_geometry(None, None, wl["shapes"])
    s.set_populations(to_lib(f, P))
    flink = None
    for _ in range(8):
        f, flink = oracle.step(p, of, f, oq, ouw, ouw1, want_force=True, shell=oshell)
    s.step(8)
    g = to_oracle(s.get_populations(), P)
    fl = of == oracle.FLUID
    assert rel_l2(g[fl], f[fl]) < TOL_F64
    assert abs(s.mass() - oracle.mass(p, of, f)) / oracle.mass(p, of, f) < 1e-13
    for tg in (-1, 2, 3):
        ref = (flink.reshape(-1, 3) if tg < 0 else flink[otag == tg]).sum(0)
        got = s.wall_force(tg)
        assert np.abs(got - ref).max() <= 1e-11 * max(1.0, np.abs(ref).max()), (tg, got, ref)
    s.close()


def test_shell_regularized_f64_parity():
    """The regularized wall estimate across a shell, D3Q27, TRT."""
    wl = _case("d3q27")
    wl["collision"] = lbm.COLL_TRT
    wl["wall_neq"] = lbm.NEQ_REGULARIZED
    P = perm(wl["lattice"])
    p, of, oq, ouw, ouw1, otag, oshell = _oracle_geometry(wl, lbm.BC_ELIBB_FQ)
    f = _random_state(p, of, wl["lattice"], 21)
    s = gpu_sim(wl, lbm.F64, lbm.BC_ELIBB_FQ)
    s.build_geometry(None, None, wl["shapes"])
    s.set_populations(to_lib(f, P))
    for _ in range(6):
        f = oracle.step(p, of, f, oq, ouw, ouw1, shell=oshell)
    s.step(6)
    g = to_oracle(s.get_populations(), P)
    fl = of == oracle.FLUID
    assert rel_l2(g[fl], f[fl]) < TOL_F64
    s.close()


def test_shell_fp32_launch_variants():
    """FP32 storage: the one-node, TMA-staged and two-node launches agree with each
    other and with the oracle."""
    wl = _case("d3q19")
    wl["collision"] = lbm.COLL_TRT
    P = perm(wl["lattice"])
    p, of, oq, ouw, ouw1, otag, oshell = _oracle_geometry(wl, lbm.BC_ELIBB_FQ)
    f0 = _random_state(p, of, wl["lattice"], 9)
    out = {}
    for variant, (bx, by) in [(0, (32, 8)), (3, (32, 8)), (4, (64, 4)), (7, (32, 4))]:
        s = gpu_sim(wl, lbm.F32, lbm.BC_ELIBB_FQ)
        s.build_geometry(None, None, wl["shapes"])
        s.set_populations(to_lib(f0, P))
        s.set_launch(bx, by, variant, 1)
        s.step(3)
        s.step(40)  # direct launches, then a graph replay
        s.synchronize()
        out[variant] = (s.get_populations(), s.wall_force(2))
        s.close()
    f = f0
    for _ in range(43):
        f = oracle.step(p, of, f, oq, ouw, ouw1, shell=oshell)
    fl = of == oracle.FLUID
    g0 = out[0][0]
    assert np.array_equal(out[3][0], g0)
    scale = np.abs(g0).max()
    for v in (4, 7):
        assert np.abs(out[v][0] - g0).max() <= 2e-6 * scale, (v, np.abs(out[v][0] - g0).max())
        assert np.abs(out[v][1] - out[0][1]).max() <= 1e-4 * np.abs(out[0][1]).max()
    assert rel_l2(to_oracle(g0, P)[fl], f[fl]) < 1e-6
    rho, u = oracle.macros(p, of, f)
    s = gpu_sim(wl, lbm.F32, lbm.BC_ELIBB_FQ)
    s.build_geometry(None, None, wl["shapes"])
    s.set_populations(out[0][0])
    _, ug = s.macros()
    assert np.abs(ug.cpu().numpy()[fl] - u[fl]).max() < 1e-5
    s.close()


def test_shell_batch_equals_alone():
    """A thin-shell simulation batched with a plain one steps as it does alone."""
    import torch
    st_b, st_a = torch.cuda.Stream(), torch.cuda.Stream()
    sims = {}
    for key, st in (("batch", st_b), ("alone", st_a)):
        row = []
        for case, bc in (("d3q19", lbm.BC_ELIBB_F), ("d3q19_plain", lbm.BC_ELIBB_UQ)):
            wl = _case("d3q19")
            if case == "d3q19_plain":
                wl["shapes"] = [dict(wl["shapes"][1])]
            s = lbm.Simulation(wl["lattice"], wl["dims"], wl["tau"], lbm.F32, stream=st)
            s.set_options(bc, 1.0, wl["force"], 0)
            s.build_geometry(None, None, wl["shapes"])
            s.init(1.0, (0.01, 0.0, 0.0))
            row.append(s)
        sims[key] = row
    for s in sims["alone"]:
        s.set_launch(32, 4, 3, 2)
    b = lbm.Batch(sims["batch"])
    b.set_launch(32, 4, 3, 2)
    b.step(37)
    for s in sims["alone"]:
        s.step(37)
    for sb, sa in zip(sims["batch"], sims["alone"]):
        assert np.array_equal(sb.get_populations(), sa.get_populations())
    b.close()


def test_shell_rejections():
    s = lbm.Simulation(lbm.D2Q9, (24, 24, 1), 0.8, lbm.F64)
    with pytest.raises(lbm.LBMError):  # node (17, 12) lies on the circle
        s.build_geometry(None, None, [dict(type="shell", tag=0, c=(12, 12, 0), r=(5, 0, 0))])
    with pytest.raises(lbm.LBMError):
        s.build_geometry(None, None, [dict(type="shell", tag=0, c=(12.2, 12.1, 0), r=(0.5, 0, 0))])
    s.build_geometry(None, None, [dict(type="shell", tag=0, c=(12.2, 12.1, 0), r=(5.3, 0, 0))])
    traj = np.zeros((2, 9))
    traj[:, 0], traj[:, 1] = 4.0, 4.0
    with pytest.raises(lbm.LBMError):
        s.set_moving_body(dict(type="sphere", tag=1, r=(1.5, 0, 0)), traj, 0)
    s.close()


def _thin_shell_couette_gpu(L, speed):
    """Inner shell r1 = L/4 rotating (wall speed `speed`), outer shell r2 = 0.45 L at
    rest, fluid everywhere; D2Q9, FP64, ELIBB-FQ, TRT. Errors inside, in the gap and
    outside (the last scaled by the inner speeds)."""
    import torch
    R1, R2 = 0.25 * L, 0.45 * L
    cx = cy = L / 2.0 + 0.1
    om = speed / R1
    wl = dict(lattice=lbm.D2Q9, dims=(L, L, 1), tau=0.8, collision=lbm.COLL_TRT)
    s = gpu_sim(wl, lbm.F64, lbm.BC_ELIBB_FQ)
    s.build_geometry(None, None, [dict(type="shell", tag=1, c=(cx, cy, 0), r=(R1, 0, 0),
                                       om=(0, 0, om), om1=(0, 0, om)),
                                  dict(type="shell", tag=2, c=(cx, cy, 0), r=(R2, 0, 0))])
    X, Y = np.meshgrid(np.arange(L), np.arange(L))
    dx, dy = X.ravel() - cx, Y.ravel() - cy
    r = np.hypot(dx, dy)
    ut = np.where(r < R1, om * r, 0.0)
    gap = (r >= R1) & (r < R2)
    ut[gap] = A.cylindrical_couette(r[gap], R1, R2, om)
    uth = np.stack([-ut * dy / r, ut * dx / r], 1)
    p = oracle.params(oracle.D2Q9, (L, L, 1), 0.8)
    flags = np.zeros(L * L, np.uint8)
    P = perm(lbm.D2Q9)
    s.set_populations(to_lib(oracle.init_eq(p, flags, None, np.c_[uth, 0 * r]), P))
    prev = None
    for _ in range(400):
        s.step(500)
        u = s.macros()[1][:, :2].cpu().numpy()
        if prev is not None and np.sqrt(((u - prev) ** 2).sum() / (u ** 2).sum()) < 1e-11:
            break
        prev = u
    inner, outer = r < R1, r >= R2
    sc_in = (uth[inner] ** 2).sum()
    e_in = np.sqrt(((u[inner] - uth[inner]) ** 2).sum() / sc_in)
    e_gap = np.sqrt(((u[gap] - uth[gap]) ** 2).sum() / (uth[gap] ** 2).sum())
    e_out = np.sqrt((u[outer] ** 2).sum() / sc_in)
    s.close()
    return e_in, e_gap, e_out


def test_thin_shell_couette_second_order_gpu():
    """Diffusive scaling from wall speed 0.01 at L = 32: the inner region's error is a
    Mach-number effect at fixed speed."""
    res = [_thin_shell_couette_gpu(L, 0.01 * 32 / L) for L in (32, 64, 128)]
    for k in range(2):
        orders = [np.log2(res[j][k] / res[j + 1][k]) for j in range(2)]
        assert min(orders) > 1.8, (k, [e[k] for e in res])
    assert max(e[2] for e in res) < 1e-12
