"""Shared helpers of the GPU parity tests: run one workload on the oracle and on
the CUDA library, with the direction orders matched by velocity vector."""
import numpy as np

import oracle
from paper_2009_04604_gb300 import lbm

ORACLE_SHAPES = {"sphere": oracle.SHAPE_SPHERE, "sphere_out": oracle.SHAPE_SPHERE_OUT,
                 "ellipsoid": oracle.SHAPE_ELLIPSOID, "strip": oracle.SHAPE_STRIP}
ORACLE_BC = {lbm.BC_ELIBB_F: oracle.BC_ELIBB_F, lbm.BC_ELIBB_FQ: oracle.BC_ELIBB_FQ,
             lbm.BC_BFL: oracle.BC_BFL, lbm.BC_HWBB: oracle.BC_HWBB,
             lbm.BC_ELIBB_U: oracle.BC_ELIBB_U, lbm.BC_ELIBB_UQ: oracle.BC_ELIBB_UQ}
ORACLE_COLL = {lbm.COLL_BGK: oracle.COLL_BGK, lbm.COLL_TRT: oracle.COLL_TRT}


def perm(lat):
    """P[j] = library direction of oracle direction j."""
    co, _, _ = oracle.lattice(lat)
    cl, _ = lbm.lattice_info(lat)
    return np.array([int(np.where((cl == co[j]).all(1))[0][0]) for j in range(len(co))])


def to_lib(a, P):
    """Per-link array [N, Q, ...] in oracle order -> library order."""
    b = np.empty_like(a)
    b[:, P] = a
    return b


def to_oracle(b, P):
    return b[:, P]


def oracle_shapes(shapes):
    out = []
    for s in shapes:
        s = dict(s)
        s["type"] = ORACLE_SHAPES[s["type"]]
        out.append(s)
    return out


def oracle_params(wl, bc=lbm.BC_ELIBB_F):
    return oracle.params(wl["lattice"], wl["dims"], wl["tau"], bc=ORACLE_BC[bc],
                         rho0=wl.get("rho0", 1.0), force=wl.get("force", (0, 0, 0)),
                         xshift=wl.get("xshift", 0),
                         collision=ORACLE_COLL[wl.get("collision", lbm.COLL_BGK)],
                         magic=wl.get("magic", 3.0 / 16.0), wall_neq=wl.get("wall_neq", 0))


def gpu_sim(wl, dtype, bc=lbm.BC_ELIBB_F):
    s = lbm.Simulation(wl["lattice"], wl["dims"], wl["tau"], dtype)
    s.set_options(bc, wl.get("rho0", 1.0), wl.get("force", (0, 0, 0)), wl.get("xshift", 0))
    if wl.get("collision", lbm.COLL_BGK) != lbm.COLL_BGK:
        s.set_collision(wl["collision"], wl.get("magic", 3.0 / 16.0))
    if wl.get("wall_neq", 0):
        s.set_wall_neq(wl["wall_neq"])
    return s


def rel_l2(a, b):
    a = np.asarray(a, float)
    b = np.asarray(b, float)
    return float(np.sqrt(((a - b) ** 2).sum() / max((b ** 2).sum(), 1e-300)))
