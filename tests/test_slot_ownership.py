"""Slot ownership of one step of the library's update, on the CPU. The step kernel
pulls: every fluid node x reads slot (i, x - c_i) of the state at t, for each
direction i. It writes its own post-collision population i into slot (i, x).
For each wall, open or thin-shell link i it writes the boundary value ahead into
slot (i, x - c_i), the slot that only x gathers at t+1. A node with a link ibar
across a thin shell does not store its own population i: the node across the
shell writes that slot ahead. The kernels run all nodes of a step in parallel,
so the rule is race-free only if each slot is written at most once, and the
next step reads only slots written in this one. Both are checked here on
geometries with solid shapes, thin shells and open nodes, whose link marks come
from the oracle's geometry."""
import numpy as np
import pytest

import oracle


def _geometry(lat):
    if lat == oracle.D2Q9:
        dims = (40, 34, 1)
        shapes = [dict(type=oracle.SHAPE_SHELL, tag=1, c=(17.3, 16.6, 0.0), r=(9.7, 0, 0)),
                  dict(type=oracle.SHAPE_SHELL, tag=2, c=(17.3, 16.6, 0.0), r=(4.2, 0, 0)),
                  dict(type=oracle.SHAPE_SPHERE, tag=3, c=(33.1, 7.4, 0.0), r=(3.3, 0, 0))]
    else:
        dims = (24, 20, 18)
        shapes = [dict(type=oracle.SHAPE_SHELL, tag=1, c=(10.4, 9.7, 8.6), r=(5.3, 0, 0)),
                  dict(type=oracle.SHAPE_SPHERE, tag=3, c=(19.6, 4.2, 12.3), r=(2.2, 0, 0))]
    nx, ny, nz = dims
    base = np.zeros(nx * ny * nz, np.uint8)
    X = np.arange(base.size)
    y = (X // nx) % ny
    x = X % nx
    base[y == 0] = oracle.SOLID        # a wall plane
    base[(x == nx - 1) & (y > 0)] = oracle.OPEN  # an open plane
    p = oracle.params(lat, dims, 0.8)
    flags, q, uw, uw1, tag, shell = oracle.geometry(p, base=base, shapes=shapes, with_shell=True)
    return dims, flags, shell


def _shift(dims, n, c):
    nx, ny, nz = dims
    x, y, z = n % nx, (n // nx) % ny, n // (nx * ny)
    return ((x + c[0]) % nx) + nx * (((y + c[1]) % ny) + ny * ((z + c[2]) % nz))


@pytest.mark.parametrize("lat", [oracle.D2Q9, oracle.D3Q19, oracle.D3Q27])
def test_each_slot_written_once_and_every_gathered_slot_written(oracle_lib, lat):
    dims, flags, shell = _geometry(lat)
    c, _, opp = oracle.lattice(lat)
    Qn = len(c)
    N = flags.size
    fluid = np.nonzero(flags == oracle.FLUID)[0]
    writes, reads = [], []
    nshell = 0
    for i in range(Qn):
        src = _shift(dims, fluid, -c[i])                    # x - c_i
        cut = (flags[src] != oracle.FLUID) | (shell[fluid, i] > 0)
        nshell += int((shell[fluid, i] > 0).sum())
        reads.append(i * N + src)                           # the gather at t+1
        own = shell[fluid, opp[i]] == 0                     # skip i when link ibar crosses a shell
        writes.append(i * N + fluid[own])                   # own post-collision store
        writes.append(i * N + src[cut & (i > 0)])           # written ahead for the cut link
    w = np.concatenate(writes)
    r = np.unique(np.concatenate(reads))
    slots, count = np.unique(w, return_counts=True)
    assert nshell > 20
    assert count.max() == 1, "a slot is written twice in one step"
    assert np.isin(r, slots).all(), "a gathered slot is not written in the step"


def test_without_the_skip_shell_slots_are_written_twice(oracle_lib):
    """The skip rule is needed: both nodes of a shell link would write one slot."""
    dims, flags, shell = _geometry(oracle.D2Q9)
    c, _, opp = oracle.lattice(oracle.D2Q9)
    N = flags.size
    fluid = np.nonzero(flags == oracle.FLUID)[0]
    writes = []
    for i in range(len(c)):
        src = _shift(dims, fluid, -c[i])
        cut = (flags[src] != oracle.FLUID) | (shell[fluid, i] > 0)
        writes.append(i * N + fluid)
        writes.append(i * N + src[cut & (i > 0)])
    _, count = np.unique(np.concatenate(writes), return_counts=True)
    assert count.max() == 2
