"""Batched stepping: each simulation of a batch gives exactly the results it gives
when stepped alone with the same launch variant (same per-node code, same
register budget), for uneven grids, mixed boundary rules, collision operators,
forces and buffer parities."""
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


def _make(wl, dtype, bc, stream, force=(0.0, 0.0, 0.0), coll=lbm.COLL_BGK):
    s = lbm.Simulation(wl["lattice"], wl["dims"], wl["tau"], dtype, stream=stream)
    s.set_options(bc, wl["rho0"], force, wl["xshift"])
    s.set_collision(coll, 3.0 / 16.0)
    s.build_geometry(wl["base"], wl["base_u"], wl["shapes"])
    s.init(wl["rho0"])
    return s


@pytest.mark.parametrize("dtype", [lbm.F64, lbm.F32, lbm.F16])
def test_batch_equals_alone(dtype):
    import torch
    wls = W.batched_ducts(n=5, lo=20, hi=44, target=None, seed=3, rmin=2.0, rmax=6.0)
    bcs = [lbm.BC_ELIBB_F, lbm.BC_ELIBB_FQ, lbm.BC_BFL, lbm.BC_ELIBB_U, lbm.BC_ELIBB_UQ]
    forces = [(0, 0, 0), (1e-5, 0, 0), (0, 0, 0), (0, -2e-5, 1e-5), (0, 0, 0)]
    colls = [lbm.COLL_BGK, lbm.COLL_TRT, lbm.COLL_BGK, lbm.COLL_TRT, lbm.COLL_TRT]
    st_b, st_a = torch.cuda.Stream(), torch.cuda.Stream()
    batched = [_make(w, dtype, bc, st_b, F, c) for w, bc, F, c in zip(wls, bcs, forces, colls)]
    alone = [_make(w, dtype, bc, st_a, F, c) for w, bc, F, c in zip(wls, bcs, forces, colls)]
    # give one pair an odd buffer parity before batching
    batched[2].step(3)
    alone[2].step(3)
    # the same register budget on both sides: the code generator may fuse multiplies
    # and adds differently under different launch bounds
    variant = 0 if dtype == lbm.F64 else 3
    for s in alone:
        s.set_launch(32, 4, variant, 2)
    b = lbm.Batch(batched)
    b.set_launch(32, 4, variant, 2)
    b.step(5)
    b.step(40)   # graph path (32 steps) + direct steps
    for s in alone:
        s.step(45)
    batched[1].step(2)  # a member stepped on its own in between
    alone[1].step(2)
    b.step(3)
    for k, s in enumerate(alone):
        s.step(3)
    for k, (sb, sa) in enumerate(zip(batched, alone)):
        fb, fa = sb.get_populations(), sa.get_populations()
        assert np.array_equal(fb, fa), (k, np.abs(fb - fa).max())
        assert np.isfinite(fb).all()
    b.close()


def test_batch_rejects_mixed_types():
    import torch
    wl = W.sphere_duct_small()
    st = torch.cuda.Stream()
    a = _make(wl, lbm.F32, lbm.BC_ELIBB_F, st)
    c = _make(wl, lbm.F16, lbm.BC_ELIBB_F, st)
    with pytest.raises(lbm.LBMError):
        lbm.Batch([a, c])
    with pytest.raises(lbm.LBMError):
        lbm.Batch([a, a])
