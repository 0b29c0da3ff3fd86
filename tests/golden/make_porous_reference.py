"""Write the FP64 oracle's reference for the porous-medium downscale with a moving
sphere at the configured weak body force: D3Q19 BGK tau = 0.65, 48^3 periodic box
of static spheres (random sequential addition, radii U[3, 5], seed 5), one sphere
of radius 4 on a sinusoidal path (amplitude 3, period 300), body force g = 1e-6
along x, ELIBB-F, 1500 steps from rest. Stored: the node kinds at the end and the
velocity of every fluid node. The oracle rebuilds the geometry every step from
the static spheres (once) and the moving sphere at its pose (its region of the
box holds no static sphere, so no link is cut by both), and refills nodes the
sphere uncovers with f^eq(rho0, u_body). Calls only oracle/ and the seeded
workload builder. The GPU runs in FP32 and FP16 storage are compared with this
file (tests, and the accuracy figures bench.py prints beside the porous-medium
throughput).

    python tests/golden/make_porous_reference.py
"""
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_2009_04604_gb300 import workloads as W  # noqa: E402

STEPS = 1500
OUT = os.path.join(HERE, "porous_48_g1e-6_t1500.npz")
ARGS = dict(n=48, rmin=3.0, rmax=5.0, moving_radius=4.0, amplitude=3.0, period=300, seed=5, g=1e-6)


def body_at(body, traj, k):
    n = len(traj)
    p, p1 = traj[k % n], traj[(k + 1) % n]
    return dict(body, type=oracle.SHAPE_SPHERE, c=tuple(p[:3]), v=tuple(p[3:6]), om=tuple(p[6:9]),
                v1=tuple(p1[3:6]), om1=tuple(p1[6:9]))


def main():
    oracle.build()
    wl = W.porous_with_moving_sphere(**ARGS)
    p = oracle.params(wl["lattice"], wl["dims"], wl["tau"], bc=oracle.BC_ELIBB_F, rho0=wl["rho0"],
                      force=wl["force"])
    stat = [dict(s, type=oracle.SHAPE_SPHERE) for s in wl["shapes"]]
    fs, qs, uws, uw1s, tags = oracle.geometry(p, None, None, stat)
    traj, body = wl["traj"], wl["body"]

    def geo(k):
        fm, qm, uwm, uw1m, tagm = oracle.geometry(p, None, None, [body_at(body, traj, k)])
        flags = np.where(fm == oracle.SOLID, oracle.SOLID, fs).astype(np.uint8)
        return flags, qs + qm, uws + uwm, uw1s + uw1m

    flags, q, uw, uw1 = geo(0)
    f = oracle.init_eq(p, flags)
    t0 = time.time()
    for t in range(STEPS):
        f = oracle.step(p, flags, f, q, uw, uw1)
        fn, qn, uwn, uw1n = geo(t + 1)
        un = np.tile(traj[(t + 1) % len(traj), 3:6], (fn.size, 1))
        oracle.refill(p, flags, fn, un, f)
        flags, q, uw, uw1 = fn, qn, uwn, uw1n
    _, u = oracle.macros(p, flags, f)
    fl = flags == 0
    np.savez_compressed(OUT, flags=flags, u=u[fl].astype(np.float32), steps=STEPS,
                        note="FP64 oracle, porous 48^3 + moving sphere, g = 1e-6, ELIBB-F, BGK tau 0.65, "
                             "from rest; u of the fluid nodes in node order (float32)")
    print(f"{OUT}: {STEPS} steps in {time.time() - t0:.0f} s, |u|max {np.abs(u).max():.3e}, "
          f"mean u_x {u[fl, 0].mean():.3e}")


if __name__ == "__main__":
    main()
