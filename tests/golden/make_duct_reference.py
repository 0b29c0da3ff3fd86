"""Write the FP64 oracle's reference for the sphere-duct downscale (64 x 32 x 32,
sphere R = 4, D3Q19 BGK tau = 0.7, inlet u = 0.02, pressure outlet, ELIBB-F) after
20000 steps from rest: the velocity of every fluid node and the drag on the
sphere (momentum exchange of the last step, Sec. II.F). Calls only oracle/ and
the seeded workload builder. The GPU runs of every storage type are compared
with this file (tests, and the accuracy figures bench.py prints beside each
throughput).

    python tests/golden/make_duct_reference.py
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

STEPS = 20000
OUT = os.path.join(HERE, "sphere_duct_64x32x32_t20000.npz")
KINDS = {"sphere": oracle.SHAPE_SPHERE, "sphere_out": oracle.SHAPE_SPHERE_OUT,
         "ellipsoid": oracle.SHAPE_ELLIPSOID, "strip": oracle.SHAPE_STRIP}


def main():
    oracle.build()
    wl = W.sphere_duct_small()
    p = oracle.params(wl["lattice"], wl["dims"], wl["tau"], bc=oracle.BC_ELIBB_F, rho0=wl["rho0"])
    shapes = [dict(s, type=KINDS[s["type"]]) for s in wl["shapes"]]
    flags, q, uw, uw1, tag = oracle.geometry(p, wl["base"], wl["base_u"], shapes)
    f = oracle.init_eq(p, flags)
    t0 = time.time()
    for _ in range(STEPS - 1):
        f = oracle.step(p, flags, f, q, uw, uw1)
    f, flink = oracle.step(p, flags, f, q, uw, uw1, want_force=True)
    drag = flink[tag == 1].sum(0)
    _, u = oracle.macros(p, flags, f)
    fl = flags == 0
    np.savez_compressed(OUT, flags=flags, u=u[fl].astype(np.float32), drag=drag, steps=STEPS,
                        note="FP64 oracle, ELIBB-F, BGK tau 0.7, u_in 0.02, from rest; u of the fluid "
                             "nodes in node order (float32), drag = sphere wall force of the last step")
    print(f"{OUT}: {STEPS} steps in {time.time() - t0:.0f} s, drag {drag}, |u|max {np.abs(u).max():.5f}")


if __name__ == "__main__":
    main()
