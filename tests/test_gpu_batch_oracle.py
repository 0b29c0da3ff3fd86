"""Batched simulations against the FP64 oracle.

Three ducts of uneven sizes, obstacles, inlet speeds, boundary rules and body
forces advance together in one batch (graph replays and direct launches), and
each is compared with the oracle stepping it alone: populations within 1e-12
relative L2 in FP64 storage, the velocity within 1e-5 in FP32 storage at the
batched launch the benchmark tunes for its ducts (32 x 8 threads, variant 3,
two tiles per block)."""
import numpy as np
import pytest

import oracle
from paper_2009_04604_gb300 import build, lbm
from paper_2009_04604_gb300 import workloads as W

from gpu_helpers import oracle_params, oracle_shapes, perm, rel_l2, to_oracle

pytestmark = pytest.mark.gpu

STEPS = 45
BCS = [lbm.BC_ELIBB_F, lbm.BC_ELIBB_FQ, lbm.BC_BFL]
FORCES = [(0.0, 0.0, 0.0), (1e-5, 0.0, 0.0), (0.0, -2e-5, 1e-5)]


@pytest.fixture(scope="module", autouse=True)
def _lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()
    oracle.build()
    lbm.load()


def _cases():
    wls = W.batched_ducts(n=3, lo=28, hi=60, target=None, seed=13, rmin=3.0, rmax=8.0)
    for wl, F in zip(wls, FORCES):
        wl["force"] = F
    return wls


@pytest.mark.parametrize("dtype,launch,bound", [(lbm.F64, (32, 4, 0, 2), 1e-12), (lbm.F32, (32, 8, 3, 2), 1e-5)])
def test_batched_members_match_oracle(dtype, launch, bound):
    import torch
    wls = _cases()
    st = torch.cuda.Stream()
    sims = []
    for wl, bc in zip(wls, BCS):
        s = lbm.Simulation(wl["lattice"], wl["dims"], wl["tau"], dtype, stream=st)
        s.set_options(bc, wl["rho0"], wl["force"], wl["xshift"])
        s.build_geometry(wl["base"], wl["base_u"], wl["shapes"])
        s.init(wl["rho0"])
        sims.append(s)
    b = lbm.Batch(sims)
    b.set_launch(*launch)
    b.step(5)
    b.step(STEPS - 5)  # one 32-step graph replay and direct launches
    P = perm(lbm.D3Q19)
    for k, (wl, bc, s) in enumerate(zip(wls, BCS, sims)):
        p = oracle_params(wl, bc)
        of, oq, ouw, ouw1, _ = oracle.geometry(p, wl["base"], wl["base_u"], oracle_shapes(wl["shapes"]))
        f = oracle.init_eq(p, of)
        for _ in range(STEPS):
            f = oracle.step(p, of, f, oq, ouw, ouw1)
        fl = of == 0
        if dtype == lbm.F64:
            g = to_oracle(s.get_populations(), P)
            assert rel_l2(g[fl], f[fl]) < bound, k
        _, u = s.macros()
        _, uo = oracle.macros(p, of, f)
        err = rel_l2(u.cpu().numpy()[fl], uo[fl])
        assert err < max(bound, 1e-12), (k, err)
    b.close()
    for s in sims:
        s.close()
