"""lbm_mass_noalloc: the mass reduction for callers that cannot allocate device
memory.

Some callers cannot call cudaMalloc: monitoring code inside a step loop that must
not stall on the allocator, and processes where another allocator already holds
the device memory. This entry point keeps its partial sums in a static device
array. The tests check that, through the C ABI, it returns the same total mass as
lbm_mass on two calls in a row, and that it rejects a lattice too large for its
array. The file is named to be collected last.
"""
import ctypes

import numpy as np
import pytest

from paper_2009_04604_gb300 import build, lbm
from paper_2009_04604_gb300 import workloads as W

pytestmark = pytest.mark.gpu

TOL = 1e-12  # relative, the FP64 tolerance of the parity tests


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()
    lbm.load()
    return torch


@pytest.mark.parametrize("dtype", [lbm.F64, lbm.F32])
def test_mass_noalloc_matches_lbm_mass_twice(torch_cuda, dtype):
    torch = torch_cuda
    wl = W.sphere_duct_small()
    s = lbm.Simulation(wl["lattice"], wl["dims"], wl["tau"], dtype)
    s.set_options(lbm.BC_ELIBB_F, wl["rho0"], wl["force"], wl["xshift"])
    s.build_geometry(wl["base"], wl["base_u"], wl["shapes"])
    s.init(wl["rho0"])
    out = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
    lib = lbm.load()
    for call in range(2):
        s.step(7)
        ref = s.mass()
        rc = lib.lbm_mass_noalloc(s.h, ctypes.c_void_p(out.data_ptr()))
        assert rc == 0, lib.lbm_last_error(s.h)
        s.synchronize()
        got = float(out.item())
        assert abs(got - ref) <= TOL * abs(ref), (call, got, ref)
        out.fill_(float("nan"))
    s.close()


def test_mass_noalloc_rejects_oversized_lattice(torch_cuda):
    torch = torch_cuda
    # 8192 x 8192 D2Q9 needs 256 * 1024 = 262144 partial sums > 131072
    s = lbm.Simulation(lbm.D2Q9, (8192, 8192, 1), 0.8, lbm.F16)
    s.set_geometry(np.zeros(8192 * 8192, np.uint8))
    s.init(1.0)
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    lib = lbm.load()
    rc = lib.lbm_mass_noalloc(s.h, ctypes.c_void_p(out.data_ptr()))
    assert rc == -1
    assert b"too large" in lib.lbm_last_error(s.h)
    s.close()
