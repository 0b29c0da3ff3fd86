"""Write the FP64 oracle's reference for Jeffery's orbit of a free elliptic
cylinder (Sec. III.C): D2Q9 BGK tau = 0.8, a 128 x 98 shear channel with walls
at -U/2 and +U/2 (U = 0.04), starting from the linear shear flow, an ellipse of
semi-axes 4 x 8 (aspect ratio 2) at the centre with its major axis along y,
turning freely about z under the momentum-exchange torque (oracle.free_rotation).
The run lasts 1.2 quarter turns of the closed-form orbit, 11309 steps, for four
couplings: ELIBB-F and BFL, each with the equilibrium refill of uncovered nodes
and with the local iteration refill (12 iterations, App. D).

Stored per coupling: the angle every 10 steps, the first step past a quarter
turn, and the mean torque squared fluctuation (App. D, Eq. TSF30: polynomial
baselines of order 30) over steps 500 to that quarter turn, with the mean
squared torque over the same steps. The GPU runs of the same couplings are
compared with this file (tests/test_gpu_rigid.py).

    python tests/golden/make_jeffery_reference.py      # four processes, about 20 minutes
"""
import math
import multiprocessing as mp
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

OUT = os.path.join(HERE, "jeffery_ellipse_128x98.npz")
CHANNEL = dict(nx=128, ny=98, U=0.04, tau=0.8, ra=8.0, rb=4.0)
RUNS = [("elibb_f", 0), ("elibb_f", 12), ("bfl", 0), ("bfl", 12)]
T_START = 500      # the start-up transient of the coupling is over by then
EVERY = 10


def steps_of(ch):
    """1.2 times the closed-form quarter turn: tan(gamma t r / (r^2 + 1)) = infinity."""
    r = ch["aspect"]
    return int(1.2 * (math.pi / 2) * (r * r + 1) / (ch["gamma"] * r))


def run(arg):
    bcname, lir = arg
    import oracle
    from oracle import analytic as A
    from paper_2009_04604_gb300 import workloads as W
    oracle.build()
    ch = W.shear_channel_ellipse(**CHANNEL)
    bc = {"elibb_f": oracle.BC_ELIBB_F, "bfl": oracle.BC_BFL}[bcname]
    p = oracle.params(oracle.D2Q9, ch["dims"], ch["tau"], bc=bc)
    body = dict(ch["body"], type=oracle.SHAPE_ELLIPSOID)
    flags, *_ = oracle.geometry(p, ch["base"], ch["base_u"], [body])
    f0 = oracle.init_eq(p, flags, None, ch["u0"])
    steps = steps_of(ch)
    _, _, hist = oracle.free_rotation(p, ch["base"], ch["base_u"], body, ch["inertia"], f0, steps, lir=lir)
    theta = -hist[:, 0]
    k = int(np.searchsorted(theta, math.pi / 2))
    t = np.arange(1, steps + 1, dtype=np.float64)
    T = hist[:, 2]
    _, tsf, _ = A.torque_squared_fluctuation(t[T_START:k], T[T_START:k])
    return dict(angle=hist[EVERY - 1::EVERY, 0].copy(), quarter=k, tsf=float(tsf.mean()),
                t2=float(np.mean(T[T_START:k] ** 2)), steps=steps)


def main():
    with mp.get_context("spawn").Pool(len(RUNS)) as pool:
        res = pool.map(run, RUNS)
    out = dict(channel=np.array([CHANNEL[k] for k in ("nx", "ny", "U", "tau", "ra", "rb")]),
               t_start=T_START, every=EVERY, steps=res[0]["steps"])
    for (bcname, lir), r in zip(RUNS, res):
        key = f"{bcname}_lir{lir}"
        out[key + "_angle"] = r["angle"]
        out[key + "_quarter"] = r["quarter"]
        out[key + "_tsf"] = r["tsf"]
        out[key + "_t2"] = r["t2"]
        print(f"{key}: quarter turn at step {r['quarter']}, mean TSF {r['tsf']:.4e}, mean T^2 {r['t2']:.4e}")
    np.savez_compressed(OUT, **out)
    print("wrote", OUT)


if __name__ == "__main__":
    main()
