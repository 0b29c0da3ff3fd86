"""Parity with the FP64 oracle of the unified ELIBB rules (ELIBB-U, Eq.
unified_space_coordinates; ELIBB-UQ, Eq. elibbqu) and of the TRT collision
(Sec. II.A, Eq. magic-parameter) with every boundary rule, through the C ABI:

- FP64 storage on random geometry (walls, open nodes, q in (0, 1] including 1/2,
  1 and both cutoffs, moving walls, tags, body force, sheared wrap): populations
  within 1e-12 relative L2, mass, and wall force per tag;
- FP32 storage on the sphere-duct downscale: velocity within 1e-5 of the oracle,
  for every launch variant of the step kernel;
- TRT with Lambda = 3/16 and half-way bounce-back: the body-force channel is the
  exact parabola with the walls half-way, at tau = 3, on the GPU.
"""
import numpy as np
import pytest

import oracle
from paper_2009_04604_gb300 import build, lbm
from paper_2009_04604_gb300 import workloads as W

from gpu_helpers import gpu_sim, oracle_params, oracle_shapes, perm, rel_l2, to_lib, to_oracle
from test_gpu_parity import TOL_F64, _random_case

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()
    oracle.build()
    lbm.load()


CASES = [(lbm.BC_ELIBB_U, lbm.COLL_BGK), (lbm.BC_ELIBB_UQ, lbm.COLL_BGK)] + [
    (bc, lbm.COLL_TRT) for bc in (lbm.BC_ELIBB_F, lbm.BC_ELIBB_FQ, lbm.BC_BFL, lbm.BC_HWBB,
                                  lbm.BC_ELIBB_U, lbm.BC_ELIBB_UQ)]


@pytest.mark.parametrize("bc,coll", CASES)
@pytest.mark.parametrize("lat,dims,xshift,force,tau", [
    (lbm.D2Q9, (64, 17, 1), 5, (1e-4, -2e-4, 0.0), 0.8),
    (lbm.D3Q19, (37, 11, 9), 0, (1e-4, 5e-5, -1e-4), 1.3),
])
def test_random_geometry_f64_parity(bc, coll, lat, dims, xshift, force, tau):
    wl, flags, q, uw, uw1, tag, rho, u, xi = _random_case(lat, dims, 31 + bc, xshift, force, tau)
    wl.update(collision=coll, magic=3.0 / 16.0)
    P = perm(lat)
    p = oracle_params(wl, bc)
    f0 = oracle.init_eq(p, flags, rho, u) * (1.0 + xi)
    f0[flags != 0] = 0.0
    s = gpu_sim(wl, lbm.F64, bc)
    s.set_geometry(flags, to_lib(q, P), to_lib(uw, P), to_lib(uw1, P), to_lib(tag, P))
    s.set_populations(to_lib(f0, P))
    f, flink = f0, None
    for _ in range(12):
        f, flink = oracle.step(p, flags, f, q, uw, uw1, want_force=True)
    s.step(12)
    g = to_oracle(s.get_populations(), P)
    fl = flags == 0
    assert rel_l2(g[fl], f[fl]) < TOL_F64
    assert abs(s.mass() - oracle.mass(p, flags, f)) / oracle.mass(p, flags, f) < 1e-13
    for tg in (-1, 0, 5):
        ref = (flink.reshape(-1, 3) if tg < 0 else flink[tag == tg]).sum(0)
        got = s.wall_force(tg)
        assert np.abs(got - ref).max() <= 1e-11 * max(1.0, np.abs(ref).max()), (tg, got, ref)
    s.close()


@pytest.mark.parametrize("variant", [0, 3, 4, 7, 9, 10, 12])
@pytest.mark.parametrize("bc,coll", [(lbm.BC_ELIBB_UQ, lbm.COLL_BGK), (lbm.BC_ELIBB_FQ, lbm.COLL_TRT),
                                     (lbm.BC_ELIBB_U, lbm.COLL_TRT)])
def test_sphere_duct_downscale_f32(bc, coll, variant):
    wl = W.sphere_duct_small()
    wl.update(collision=coll, magic=3.0 / 16.0, force=(1e-6, 0.0, 0.0))
    steps = 300
    P = perm(wl["lattice"])
    p = oracle_params(wl, bc)
    of, oq, ouw, ouw1, otag = oracle.geometry(p, wl["base"], wl["base_u"], oracle_shapes(wl["shapes"]))
    f = oracle.init_eq(p, of)
    for _ in range(steps):
        f = oracle.step(p, of, f, oq, ouw, ouw1)
    s = gpu_sim(wl, lbm.F32, bc)
    s.build_geometry(wl["base"], wl["base_u"], wl["shapes"])
    s.init(1.0)
    s.set_launch(32, 8 if variant < 5 else 4, variant, 1)
    s.step(steps)
    _, u = s.macros()
    _, uo = oracle.macros(p, of, f)
    fl = of == 0
    err = rel_l2(u.cpu().numpy()[fl], uo[fl])
    assert err < 1e-5, err
    s.close()


def test_trt_magic_3_16_half_way_wall_on_gpu():
    H, g, tau = 12, 1e-6, 3.0
    ny = H + 2
    s = lbm.Simulation(lbm.D2Q9, (1, ny, 1), tau, lbm.F64)
    s.set_options(lbm.BC_HWBB, 1.0, (g, 0.0, 0.0), 0)
    s.set_collision(lbm.COLL_TRT, 3.0 / 16.0)
    flags = np.zeros(ny, np.uint8)
    flags[0] = flags[-1] = lbm.SOLID
    s.set_geometry(flags)
    s.init(1.0)
    nu = (tau - 0.5) / 3.0
    s.step(int(40 * H * H / (np.pi ** 2 * nu)) + 200)
    u = s.macros()[1].cpu().numpy()[1:H + 1, 0]
    y = np.arange(1, H + 1, dtype=float)
    uth = g / (2.0 * nu) * (y - 0.5) * (H + 0.5 - y)
    assert np.abs(u - uth).max() / uth.max() < 1e-9
    s.close()


def test_set_collision_arguments():
    s = lbm.Simulation(lbm.D2Q9, (8, 8, 1), 0.8, lbm.F32)
    with pytest.raises(lbm.LBMError):
        s.set_collision(7, 0.1875)
    with pytest.raises(lbm.LBMError):
        s.set_collision(lbm.COLL_TRT, 0.0)
    s.set_collision(lbm.COLL_TRT, 0.25)
    s.set_collision(lbm.COLL_BGK, 0.0)  # magic is ignored for BGK
    s.close()
