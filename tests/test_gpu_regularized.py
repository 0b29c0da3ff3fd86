"""Parity with the FP64 oracle of the regularized wall non-equilibrium estimate
(the appendix's Eq. fi_neq; lbm_set_wall_neq), through the C ABI: FP64 storage on
random geometry (moving walls, open nodes, every q branch, body force, sheared
wrap) for the ELIBB rules under BGK and TRT, and FP32 storage on the
sphere-duct downscale."""
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


@pytest.mark.parametrize("bc", [lbm.BC_ELIBB_F, lbm.BC_ELIBB_FQ, lbm.BC_ELIBB_U, lbm.BC_ELIBB_UQ])
@pytest.mark.parametrize("coll", [lbm.COLL_BGK, lbm.COLL_TRT])
@pytest.mark.parametrize("lat,dims,xshift,force,tau", [
    (lbm.D2Q9, (64, 17, 1), 5, (1e-4, -2e-4, 0.0), 0.8),
    (lbm.D3Q19, (37, 11, 9), 0, (1e-4, 5e-5, -1e-4), 1.3),
])
def test_random_geometry_f64_parity(bc, coll, lat, dims, xshift, force, tau):
    wl, flags, q, uw, uw1, tag, rho, u, xi = _random_case(lat, dims, 51 + bc, xshift, force, tau)
    wl.update(collision=coll, magic=3.0 / 16.0, wall_neq=lbm.NEQ_REGULARIZED)
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
    ref = flink.reshape(-1, 3).sum(0)
    got = s.wall_force(-1)
    assert np.abs(got - ref).max() <= 1e-11 * max(1.0, np.abs(ref).max())
    s.close()


@pytest.mark.parametrize("bc", [lbm.BC_ELIBB_F, lbm.BC_ELIBB_UQ])
def test_sphere_duct_downscale_f32(bc):
    wl = W.sphere_duct_small()
    wl.update(wall_neq=lbm.NEQ_REGULARIZED)
    steps = 300
    p = oracle_params(wl, bc)
    of, oq, ouw, ouw1, otag = oracle.geometry(p, wl["base"], wl["base_u"], oracle_shapes(wl["shapes"]))
    f = oracle.init_eq(p, of)
    for _ in range(steps):
        f = oracle.step(p, of, f, oq, ouw, ouw1)
    s = gpu_sim(wl, lbm.F32, bc)
    s.build_geometry(wl["base"], wl["base_u"], wl["shapes"])
    s.init(1.0)
    s.step(steps)
    _, u = s.macros()
    _, uo = oracle.macros(p, of, f)
    fl = of == 0
    err = rel_l2(u.cpu().numpy()[fl], uo[fl])
    assert err < 1e-5, err
    s.close()


def test_set_wall_neq_arguments():
    s = lbm.Simulation(lbm.D2Q9, (8, 8, 1), 0.8, lbm.F32)
    with pytest.raises(lbm.LBMError):
        s.set_wall_neq(5)
    s.set_wall_neq(lbm.NEQ_REGULARIZED)
    s.set_wall_neq(lbm.NEQ_BOUNCE_BACK)
    s.close()
