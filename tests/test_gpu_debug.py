"""The bounds-checked build (LBM_DEBUG): every population index of the kernels is
checked against the buffer, and the first one out of range is reported by
lbm_synchronize as LBM_ERR_BOUNDS, without the access.

1. No false alarms: the checked build steps walls, open nodes, moving walls, a
   body force, BFL, a moving body and every launch kind (one node per thread,
   node pairs, the TMA-staged kernel) without a report, and gives the populations
   of the unchecked build bit for bit.
2. Detection: with the check's limit set to half the buffer (lbm_set_debug_limit)
   the accesses to the upper half, which are inside the real buffer, count as
   out of range. They are reported with an index at or above the limit, and the
   handle steps normally again once the limit is restored. Nothing outside the
   buffers is ever touched, so this exercises the checks without risking a fault.

The checked cases run in a child process that loads _build_debug/liblbm.so
(LBM_LIBRARY), since a process holds one build of the library."""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

from paper_2009_04604_gb300 import build, lbm
from paper_2009_04604_gb300 import workloads as W

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
LAUNCHES = [(32, 4, 0, 1), (32, 4, 3, 2), (32, 4, 7, 1), (32, 4, 8, 1), (32, 4, 4, 1)]


@pytest.fixture(scope="module", autouse=True)
def _lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()
    build.build(debug=True)
    lbm.load()


def _cases():
    """(name, builder) of the small workloads both builds run."""
    def random3d(dtype, bc):
        dims = (64, 9, 6)
        flags, q, uw, uw1, tag = W.random_geometry(dims, seed=41, Q=19)
        s = lbm.Simulation(lbm.D3Q19, dims, 0.8, dtype)
        s.set_options(bc, 1.0, (2e-5, 0.0, -1e-5), 0)
        s.set_geometry(flags, q, uw, uw1, tag)
        s.init(1.0, (0.01, -0.005, 0.002))
        return s

    def moving(dtype, bc):
        s = lbm.Simulation(lbm.D3Q19, (64, 24, 24), 0.8, dtype)
        s.set_options(bc, 1.0, (1e-5, 0, 0), 0)
        s.build_geometry(None, None, [dict(type="sphere", tag=0, c=(6.2, 5.1, 5.3), r=(3.5, 0, 0))])
        t = np.arange(200)
        traj = np.zeros((200, 9))
        traj[:, 0] = 32.3 + 3 * np.sin(2 * np.pi * t / 200)
        traj[:, 1], traj[:, 2] = 12.1, 11.7
        traj[:, 3] = 3 * 2 * np.pi / 200 * np.cos(2 * np.pi * t / 200)
        s.set_moving_body(dict(type="sphere", tag=1, r=(4.2, 0, 0)), traj, 0)
        s.init(1.0)
        return s
    return {"random3d": random3d, "moving": moving}


def _run_all(out_path):
    """Step every case with every launch; save the populations (both builds call this)."""
    res = {}
    for name, make in _cases().items():
        for bc in (lbm.BC_ELIBB_F, lbm.BC_BFL):
            if name == "moving" and bc == lbm.BC_BFL:
                continue  # BFL takes no moving body
            for L in LAUNCHES:
                if bc == lbm.BC_BFL and L[2] >= 5:
                    continue  # the pair kernels have no BFL path
                s = make(lbm.F32, bc)
                s.set_launch(*L)
                s.step(3)
                s.step(37)  # direct launches, then graph replays
                s.synchronize()
                res[f"{name}_{bc}_{'_'.join(map(str, L))}"] = s.get_populations()
                s.close()
    np.savez(out_path, **res)


CHILD = r"""
import json, sys
sys.path.insert(0, {root!r}); sys.path.insert(0, {tests!r})
import numpy as np
from paper_2009_04604_gb300 import lbm
import test_gpu_debug as T
lbm.load()
assert lbm.is_debug_build()
T._run_all({out!r})
# detection: a limit of half the buffer, then the default again
s = T._cases()["random3d"](lbm.F32, lbm.BC_ELIBB_F)
Q, N = 19, s.get_populations().shape[0]
s.set_launch(32, 4, 3, 1)
half = Q * 64 * 9 * 6 // 2
s.set_debug_limit(half)
s.step(2)
try:
    s.synchronize()
    caught = None
except lbm.LBMError as e:
    caught = (e.code, str(e))
s.set_debug_limit(-1)
s.init(1.0, (0.01, -0.005, 0.002))
s.step(5)
s.synchronize()
ok_after = bool(np.isfinite(s.get_populations()).all())
s.close()
print(json.dumps(dict(caught=caught, half=half, ok_after=ok_after)))
"""


def test_checked_build_runs_clean_matches_and_reports_out_of_range(tmp_path):
    out = str(tmp_path / "debug.npz")
    env = dict(os.environ, LBM_LIBRARY=build.DEBUG_LIB)
    code = CHILD.format(root=ROOT, tests=os.path.join(ROOT, "tests"), out=out)
    r = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stderr[-3000:]
    info = json.loads(r.stdout.strip().splitlines()[-1])
    # detection, with the index and the source line of the access
    assert info["caught"] is not None, "no report with a limit of half the buffer"
    code_, msg = info["caught"]
    assert code_ == -7 and "out of range" in msg, msg
    idx = int(msg.split("population index ")[1].split(" ")[0])
    assert info["half"] <= idx < 2 * info["half"] + 19, msg
    assert info["ok_after"]
    # no false alarms, and the same populations as the unchecked build
    assert not lbm.is_debug_build()
    ref = str(tmp_path / "release.npz")
    _run_all(ref)
    a, b = np.load(ref), np.load(out)
    assert sorted(a.files) == sorted(b.files) and len(a.files) >= 12
    for k in a.files:
        assert np.array_equal(a[k], b[k]), k
