"""D3Q27, the lattice of the paper's 3-D cylindrical Couette runs (Sec. III.B),
through the C ABI against the FP64 oracle: the device link geometry bit for bit,
FP64 populations within 1e-12 for every boundary rule (also under TRT and with
the regularized wall estimate), FP32 storage on the sphere-duct downscale for
each launch variant, and batched against stepped alone bit for bit."""
import numpy as np
import pytest

import oracle
from paper_2009_04604_gb300 import build, lbm
from paper_2009_04604_gb300 import workloads as W

from gpu_helpers import gpu_sim, oracle_params, oracle_shapes, perm, rel_l2, to_lib, to_oracle
from test_gpu_parity import TOL_F64, _random_case, _upstream

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()
    oracle.build()
    lbm.load()


def _duct(**kw):
    wl = W.sphere_duct_small()
    wl.update(lattice=lbm.D3Q27, **kw)
    return wl


@pytest.mark.parametrize("dtype", [lbm.F64, lbm.F32])
def test_link_geometry_kernel_parity(dtype):
    wl = _duct()
    wl["shapes"] = wl["shapes"] + [dict(type="ellipsoid", tag=2, c=(40.3, 14.1, 17.7), r=(6.5, 4.2, 3.3),
                                        v=(0.01, 0.0, -0.003), om=(0.0, 0.001, 0.002),
                                        v1=(0.011, 0.0, -0.003), om1=(0.0, 0.001, 0.002))]
    P = perm(lbm.D3Q27)
    p = oracle_params(wl)
    of, oq, ouw, ouw1, otag = oracle.geometry(p, wl["base"], wl["base_u"], oracle_shapes(wl["shapes"]))
    s = gpu_sim(wl, dtype)
    s.build_geometry(wl["base"], wl["base_u"], wl["shapes"])
    gf, gq, guw, guw1, gtag = s.get_geometry()
    assert np.array_equal(gf, of)
    c, _, _ = oracle.lattice(lbm.D3Q27)
    up = _upstream(wl["dims"], c)
    oqw = np.where(of[up] == oracle.SOLID, oq, 0.0)
    gq_o = to_oracle(gq, P)
    assert np.array_equal(gq_o > 0, oqw > 0)
    assert np.abs(gq_o - oqw).max() <= (0.0 if dtype == lbm.F64 else 6e-8)
    wall = oqw > 0
    assert np.abs(to_oracle(guw, P)[wall] - ouw[wall]).max() <= (0.0 if dtype == lbm.F64 else 1e-9)
    assert np.array_equal(to_oracle(gtag, P)[wall], otag[wall])
    s.close()


CASES = [(bc, lbm.COLL_BGK, 0) for bc in (lbm.BC_ELIBB_F, lbm.BC_ELIBB_FQ, lbm.BC_BFL, lbm.BC_HWBB,
                                           lbm.BC_ELIBB_U, lbm.BC_ELIBB_UQ)] + [
    (lbm.BC_ELIBB_F, lbm.COLL_TRT, 0), (lbm.BC_ELIBB_UQ, lbm.COLL_TRT, lbm.NEQ_REGULARIZED),
    (lbm.BC_ELIBB_FQ, lbm.COLL_BGK, lbm.NEQ_REGULARIZED)]


@pytest.mark.parametrize("bc,coll,neq", CASES)
def test_random_geometry_f64_parity(bc, coll, neq):
    wl, flags, q, uw, uw1, tag, rho, u, xi = _random_case(lbm.D3Q27, (33, 10, 9), 71 + bc, 0,
                                                          (1e-4, 5e-5, -1e-4), 0.9)
    wl.update(collision=coll, magic=3.0 / 16.0, wall_neq=neq)
    P = perm(lbm.D3Q27)
    p = oracle_params(wl, bc)
    f0 = oracle.init_eq(p, flags, rho, u) * (1.0 + xi)
    f0[flags != 0] = 0.0
    s = gpu_sim(wl, lbm.F64, bc)
    s.set_geometry(flags, to_lib(q, P), to_lib(uw, P), to_lib(uw1, P), to_lib(tag, P))
    s.set_populations(to_lib(f0, P))
    f, flink = f0, None
    for _ in range(10):
        f, flink = oracle.step(p, flags, f, q, uw, uw1, want_force=True)
    s.step(10)
    g = to_oracle(s.get_populations(), P)
    fl = flags == 0
    assert rel_l2(g[fl], f[fl]) < TOL_F64
    assert abs(s.mass() - oracle.mass(p, flags, f)) / oracle.mass(p, flags, f) < 1e-13
    ref = flink.reshape(-1, 3).sum(0)
    assert np.abs(s.wall_force(-1) - ref).max() <= 1e-11 * max(1.0, np.abs(ref).max())
    s.close()


def test_sphere_duct_downscale_f32_all_variants():
    wl = _duct(force=(1e-6, 0.0, 0.0))
    steps = 200
    p = oracle_params(wl, lbm.BC_ELIBB_F)
    of, oq, ouw, ouw1, _ = oracle.geometry(p, wl["base"], wl["base_u"], oracle_shapes(wl["shapes"]))
    f = oracle.init_eq(p, of)
    for _ in range(steps):
        f = oracle.step(p, of, f, oq, ouw, ouw1)
    _, uo = oracle.macros(p, of, f)
    fl = of == 0
    ref = None
    for variant in (0, 3, 4, 7):
        s = gpu_sim(wl, lbm.F32, lbm.BC_ELIBB_F)
        s.build_geometry(wl["base"], wl["base_u"], wl["shapes"])
        s.init(1.0)
        s.set_launch(32, 4, variant, 1)
        s.step(steps)
        _, u = s.macros()
        u = u.cpu().numpy()
        assert rel_l2(u[fl], uo[fl]) < 1e-5
        pops = s.get_populations()
        if ref is None:
            ref = pops
        elif variant in (3, 4):  # same arithmetic as variant 0
            assert np.array_equal(pops, ref)
        else:
            assert np.abs(pops - ref).max() <= 2e-6 * np.abs(ref).max()
        s.close()


@pytest.mark.parametrize("dtype", [lbm.F64, lbm.F32])
def test_batch_equals_alone(dtype):
    import torch
    wls = W.batched_ducts(n=3, lo=20, hi=40, target=None, seed=5, rmin=2.0, rmax=5.0)
    for w in wls:
        w["lattice"] = lbm.D3Q27
    variant = 0 if dtype == lbm.F64 else 3
    sims = []
    for st in (torch.cuda.Stream(), torch.cuda.Stream()):
        group = []
        for k, w in enumerate(wls):
            s = lbm.Simulation(lbm.D3Q27, w["dims"], w["tau"], dtype, stream=st)
            s.set_options(lbm.BC_ELIBB_FQ, 1.0, (1e-5 * k, 0, 0), 0)
            s.build_geometry(w["base"], w["base_u"], w["shapes"])
            s.init(1.0)
            s.set_launch(32, 4, variant, 2)
            group.append(s)
        sims.append(group)
    b = lbm.Batch(sims[0])
    b.set_launch(32, 4, variant, 2)
    b.step(37)
    for s in sims[1]:
        s.step(37)
    for sb, sa in zip(*sims):
        assert np.array_equal(sb.get_populations(), sa.get_populations())
    b.close()
