"""Step-by-step parity with the FP64 oracle over the first 100 steps.

The other parity tests compare the state after a run. Here the GPU state is read
back after every single step of a small random geometry (walls with q in (0, 1],
open nodes, moving walls, a body force, the sheared x-wrap on D2Q9) and compared
with the oracle's state after the same step, together with that step's
momentum-exchange force per tag. A rule that is right on average but wrong at
some step (a slot read one step late, a written-ahead value lost at one parity
of the A-B buffers) shows at the first step where it goes wrong."""
import numpy as np
import pytest

import oracle
from paper_2009_04604_gb300 import build, lbm
from paper_2009_04604_gb300 import workloads as W

from gpu_helpers import gpu_sim, oracle_params, perm, rel_l2, to_lib, to_oracle

pytestmark = pytest.mark.gpu

STEPS = 100
TOL_F64 = 1e-12


@pytest.fixture(scope="module", autouse=True)
def _lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()
    oracle.build()
    lbm.load()


@pytest.mark.parametrize("bc", [lbm.BC_ELIBB_F, lbm.BC_ELIBB_FQ, lbm.BC_BFL])
@pytest.mark.parametrize("lat,dims,xshift,force", [
    (lbm.D2Q9, (40, 21, 1), 4, (1e-4, -5e-5, 0.0)),
    (lbm.D3Q19, (32, 9, 6), 0, (5e-5, 0.0, -1e-4)),
])
def test_every_step_matches_the_oracle(bc, lat, dims, xshift, force):
    Q = {lbm.D2Q9: 9, lbm.D3Q19: 19}[lat]
    N = int(np.prod(dims))
    flags, q, uw, uw1, tag = W.random_geometry(dims, seed=23 + bc, Q=Q)
    if lat == lbm.D2Q9:
        uw[..., 2] = 0.0
        uw1[..., 2] = 0.0
    wl = dict(lattice=lat, dims=tuple(dims), tau=0.8, xshift=xshift, force=force, rho0=1.0)
    rho, u, xi = W.random_fields(N, seed=29 + bc, Q=Q, two_d=lat == lbm.D2Q9)
    P = perm(lat)
    p = oracle_params(wl, bc)
    f = oracle.init_eq(p, flags, rho, u) * (1.0 + xi)
    f[flags != 0] = 0.0
    s = gpu_sim(wl, lbm.F64, bc)
    s.set_geometry(flags, to_lib(q, P), to_lib(uw, P), to_lib(uw1, P), to_lib(tag, P))
    s.set_populations(to_lib(f, P))
    fl = flags == 0
    worst = 0.0
    for k in range(STEPS):
        f, flink = oracle.step(p, flags, f, q, uw, uw1, want_force=True)
        s.step(1)
        g = to_oracle(s.get_populations(), P)
        err = rel_l2(g[fl], f[fl])
        worst = max(worst, err)
        assert err < TOL_F64, (k + 1, err)
        ref = flink.reshape(-1, 3).sum(0)
        got = s.wall_force(-1)
        assert np.abs(got - ref).max() <= 1e-11 * max(1.0, np.abs(ref).max()), (k + 1, got, ref)
    print(f"worst relative L2 over {STEPS} steps: {worst:.2e}")
    s.close()
