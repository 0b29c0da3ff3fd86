"""Failure detection of the TMA-staged step: a bounded mbarrier wait that runs
out sets the device error word, the block waits for its own copies in flight and
leaves, and the next lbm_synchronize reports LBM_ERR_TIMEOUT. The wait is made
to run out on an ordinary step by a poll limit of 0 (lbm_set_wait_limit): every
first wait gives up at once, while the copies it would have waited for complete
normally. Nothing hangs or faults. The handle stays usable: with the default
limit restored and the state re-initialised, it steps as the one-node-per-thread
kernel does (to the tolerance of the TMA-staged kernel's own test)."""
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


def _duct(dtype):
    wl = W.sphere_duct_small()
    s = lbm.Simulation(wl["lattice"], wl["dims"], wl["tau"], dtype)
    s.set_options(lbm.BC_ELIBB_F, 1.0, (0, 0, 0), 0)
    s.build_geometry(wl["base"], wl["base_u"], wl["shapes"])
    s.init(1.0)
    return s


@pytest.mark.parametrize("dtype", [lbm.F32, lbm.F16])
def test_wait_that_runs_out_is_reported_and_the_handle_recovers(dtype):
    s = _duct(dtype)
    s.set_launch(32, 8, 4, 1)  # the TMA-staged persistent kernel
    s.set_wait_limit(0)
    s.step(2)
    with pytest.raises(lbm.LBMError) as e:
        s.synchronize()
    assert e.value.code == -5  # LBM_ERR_TIMEOUT
    s.synchronize()  # the error word was cleared
    # recovery: default limit, fresh state, the same results as variant 0
    s.set_wait_limit(-1)
    s.init(1.0)
    ref = _duct(dtype)
    ref.set_launch(32, 8, 0, 1)
    for n in (3, 40):
        s.step(n)
        ref.step(n)
    s.synchronize()
    fa, fb = ref.get_populations(), s.get_populations()
    rel = {lbm.F32: 2e-6, lbm.F16: 4e-3}[dtype]  # as in the TMA-staged kernel's own test
    assert np.abs(fa - fb).max() <= rel * np.abs(fa).max()
    s.close()
    ref.close()
