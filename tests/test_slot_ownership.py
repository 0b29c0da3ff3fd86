"""Slot ownership of one step of the library's update, on the CPU. The step kernel
pulls: every fluid node x reads slot (i, x - c_i) of the state at t, for each
direction i. It writes its own post-collision population i into slot (i, x).
For each wall, open or thin-shell link i it writes the boundary value ahead into
slot (i, x - c_i), the slot that only x gathers at t+1. A node with a link ibar
across a thin shell does not store its own population i: the node across the
shell writes that slot ahead. A non-fluid node stores values nobody reads into
its own slots (so that every 32-byte sector is written whole), in the planes its
written-ahead mask leaves free: the mask, taken from the static geometry, has
bit i where node n + c_i is fluid. In a moving body's region non-fluid nodes
store nothing, since the body's links change every step and the static mask
does not know them. The kernels run all nodes of a step in parallel, so the
rule is race-free only if each slot is written at most once, and the next step
reads only slots written in this one, never a non-fluid node's own store. Both
are checked here on geometries with solid shapes, thin shells, open nodes and a
moving body, whose link marks come from the oracle's geometry."""
import numpy as np
import pytest

import oracle


def _geometry(lat, with_body=True):
    if lat == oracle.D2Q9:
        dims = (40, 34, 1)
        shapes = [dict(type=oracle.SHAPE_SHELL, tag=1, c=(17.3, 16.6, 0.0), r=(9.7, 0, 0)),
                  dict(type=oracle.SHAPE_SHELL, tag=2, c=(17.3, 16.6, 0.0), r=(4.2, 0, 0)),
                  dict(type=oracle.SHAPE_SPHERE, tag=3, c=(33.1, 7.4, 0.0), r=(3.3, 0, 0))]
        body = dict(type=oracle.SHAPE_SPHERE, tag=4, c=(31.2, 25.3, 0.0), r=(2.6, 0, 0))
        region = ((27, 21, 0), (36, 30, 1))
    else:
        dims = (24, 20, 18)
        shapes = [dict(type=oracle.SHAPE_SHELL, tag=1, c=(10.4, 9.7, 8.6), r=(4.3, 0, 0)),
                  dict(type=oracle.SHAPE_SPHERE, tag=3, c=(19.6, 4.2, 12.3), r=(2.2, 0, 0))]
        body = dict(type=oracle.SHAPE_SPHERE, tag=4, c=(18.4, 14.1, 4.3), r=(2.1, 0, 0))
        region = ((15, 10, 1), (23, 19, 8))
    nx, ny, nz = dims
    base = np.zeros(nx * ny * nz, np.uint8)
    X = np.arange(base.size)
    y = (X // nx) % ny
    x = X % nx
    z = X // (nx * ny)
    base[y == 0] = oracle.SOLID        # a wall plane
    base[(x == nx - 1) & (y > 0)] = oracle.OPEN  # an open plane
    p = oracle.params(lat, dims, 0.8)
    static, *_ = oracle.geometry(p, base=base, shapes=shapes)
    flags, q, uw, uw1, tag, shell = oracle.geometry(p, base=base, shapes=shapes + ([body] if with_body else []),
                                                    with_shell=True)
    (x0, y0, z0), (x1, y1, z1) = region
    keep = (x >= x0) & (x < x1) & (y >= y0) & (y < y1) & (z >= z0) & (z < z1)
    return dims, static, flags, shell, keep


def _shift(dims, n, c):
    nx, ny, nz = dims
    x, y, z = n % nx, (n // nx) % ny, n // (nx * ny)
    return ((x + c[0]) % nx) + nx * (((y + c[1]) % ny) + ny * ((z + c[2]) % nz))


def _step(lat, dims, static, flags, shell, keep, use_keep=True):
    """Writes (slot ids i*N + node) of one step: (good writes, non-fluid stores, gathers)."""
    c, _, opp = oracle.lattice(lat)
    N = flags.size
    fluid = np.nonzero(flags == oracle.FLUID)[0]
    solid = np.nonzero(flags != oracle.FLUID)[0]
    if use_keep:
        solid = solid[~keep[solid]]
    good, garbage, reads = [], [], []
    for i in range(len(c)):
        src = _shift(dims, fluid, -c[i])                    # x - c_i
        cut = (flags[src] != oracle.FLUID) | (shell[fluid, i] > 0)
        reads.append(i * N + src)                           # the gather at t+1
        own = shell[fluid, opp[i]] == 0                     # skip i when link ibar crosses a shell
        good.append(i * N + fluid[own])                     # own post-collision store
        good.append(i * N + src[cut & (c[i] != 0).any()])   # written ahead for the cut link
        # a non-fluid node stores plane i unless its mask has bit i; the mask is
        # taken from the static geometry: bit i where node + c_i is fluid there,
        # and no bit at all for a node that is fluid there (a moving body's node)
        free = (static[_shift(dims, solid, c[i])] != oracle.FLUID) | (static[solid] == oracle.FLUID)
        garbage.append(i * N + solid[free])
    cat = np.concatenate
    return cat(good), cat(garbage), np.unique(cat(reads))


@pytest.mark.parametrize("lat", [oracle.D2Q9, oracle.D3Q19, oracle.D3Q27])
def test_each_slot_written_once_and_every_gathered_slot_written(oracle_lib, lat):
    dims, static, flags, shell, keep = _geometry(lat)
    assert int((shell > 0).sum()) > 20
    assert int((keep & (flags == oracle.SOLID)).sum()) > 4
    good, garbage, reads = _step(lat, dims, static, flags, shell, keep)
    slots, count = np.unique(np.concatenate([good, garbage]), return_counts=True)
    assert count.max() == 1, "a slot is written twice in one step"
    assert np.isin(reads, good).all(), "a gathered slot holds no value of this step (or a non-fluid node's store)"
    assert garbage.size > 0


def test_without_the_skip_shell_slots_are_written_twice(oracle_lib):
    """The skip rule is needed: both nodes of a shell link would write one slot."""
    dims, static, flags, shell, keep = _geometry(oracle.D2Q9, with_body=False)
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


def test_without_the_region_rule_body_slots_are_written_twice(oracle_lib):
    """The region rule is needed: the static mask does not know the moving body's
    links, so a body node's own store would meet a value written ahead."""
    dims, static, flags, shell, keep = _geometry(oracle.D2Q9)
    good, garbage, _ = _step(oracle.D2Q9, dims, static, flags, shell, keep, use_keep=False)
    _, count = np.unique(np.concatenate([good, garbage]), return_counts=True)
    assert count.max() == 2
