"""Profiling driver: one benchmark workload, a fixed (or tuned) launch, K timed steps.

    python -m paper_2009_04604_gb300.profile_case --case duct --dtype f32 --launch 32,4,8,1

It builds the workload on the device, steps it W times untimed, then K steps
per replay (best of R replays, CUDA events on the library's stream), and prints
one JSON line with the step time and the node, record and link counts. Under
ncu, `-k regex:k_step -s W+1` skips the warm-up launches. Cases:

- duct:           the sphere duct, D3Q19 256 x 128 x 128, ELIBB-F;
- box:            the same box, all fluid and periodic (the lattice tiles alone);
- porous:         the porous medium with a moving sphere (--n per axis, 384 full size);
- porous_static:  the same without the moving sphere;
- batch_large:    the 96 batched ducts (1.26e8 nodes);
- batch_mid:      24 batched ducts of the same size range (about 3e7 nodes);
- batch_small:    96 ducts of 16-48 nodes per axis.
"""
from __future__ import annotations

import argparse
import json
import time


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--case", default="duct",
                    choices=["duct", "box", "porous", "porous_static", "batch_large", "batch_mid", "batch_small"])
    ap.add_argument("--dtype", default="f32")
    ap.add_argument("--bc", default="elibb_f")
    ap.add_argument("--launch", default=None, help="bx,by,variant,tiles (default: autotune)")
    ap.add_argument("--tune", type=int, default=10, help="steps per candidate when autotuning")
    ap.add_argument("--steps", type=int, default=64)
    ap.add_argument("--warmup", type=int, default=8)
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--n", type=int, default=384, help="porous cases: nodes per axis")
    a = ap.parse_args(argv)

    import torch
    from . import build, lbm
    from . import workloads as W
    build.build()

    def make(wl, stream=None, moving=False):
        s = lbm.Simulation(wl["lattice"], wl["dims"], wl["tau"], a.dtype, stream=stream)
        s.set_options(a.bc, wl["rho0"], wl["force"], wl["xshift"])
        s.build_geometry(wl["base"], wl["base_u"], wl["shapes"])
        if moving:
            s.set_moving_body(wl["body"], wl["traj"], 0)
        s.init(wl["rho0"])
        return s

    t0 = time.time()
    sims = None
    if a.case in ("duct", "box"):
        wl = W.sphere_duct()
        if a.case == "box":
            wl["base"] = None
            wl["base_u"] = None
            wl["shapes"] = []
        obj = s = make(wl)
        stream = s.stream
    elif a.case in ("porous", "porous_static"):
        wl = W.porous_with_moving_sphere() if a.n == 384 else W.porous_with_moving_sphere(n=a.n)
        obj = s = make(wl, moving=a.case == "porous")
        stream = s.stream
    else:
        if a.case == "batch_large":
            wls = W.batched_ducts()
        elif a.case == "batch_mid":
            wls = W.batched_ducts(n=24, target=3e7)
        else:
            wls = W.batched_ducts(lo=16, hi=48, target=None, rmin=2.0, rmax=6.0)
        stream = torch.cuda.Stream()
        sims = [make(w, stream) for w in wls]
        obj = lbm.Batch(sims)
    setup_s = time.time() - t0
    if a.launch:
        bx, by, var, tl = (int(t) for t in a.launch.split(","))
        obj.set_launch(bx, by, var, tl)
        launch = dict(bx=bx, by=by, variant=var, tiles=tl)
    else:
        launch = obj.autotune(a.tune)
    obj.step(a.warmup)
    torch.cuda.synchronize()
    best = float("inf")
    for _ in range(a.reps):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        obj.step(a.steps)
        e1.record(stream)
        e1.synchronize()
        best = min(best, e0.elapsed_time(e1) / a.steps)
    counts = [x.counts() for x in sims] if sims else [s.counts()]
    nf, nb, nl = (sum(c[k] for c in counts) for k in range(3))
    print(json.dumps(dict(case=a.case, dtype=a.dtype, n=a.n, launch=launch, us_per_step=round(best * 1e3, 2),
                          glups=round(nf / (best * 1e-3) / 1e9, 2), nfluid=nf, nb=nb, nl=nl,
                          setup_s=round(setup_s, 1))), flush=True)


if __name__ == "__main__":
    main()
