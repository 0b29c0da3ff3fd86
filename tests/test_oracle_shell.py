"""Pins of the oracle's thin-shell walls: a spherical shell (a circle on D2Q9) with
fluid on both of its sides, as the cylinders of the thin-shell Couette runs of
Sec. III.B and the ellipsoid of Sec. III.C are represented. Each side treats
the shell as a wall: a link that crosses it is cut from both ends, and each end
applies the boundary rule to the population that comes back to it. Checked
against facts that do not come from the oracle:

- q of every crossing link is the root of |x - t c_i - c| = r0 found by
  bisection, and the two ends of a link see the same wall point (q + q' = 1);
- no information crosses the shell: changing the state on one side leaves the
  other side bit for bit unchanged, under every rule;
- under half-way bounce-back the mass inside and the mass outside are each
  conserved;
- steady thin-shell circular Couette flow (inner shell rotating, outer shell at
  rest): rigid rotation inside the inner shell, the Couette profile in the gap,
  rest outside the outer shell, at second order; the torque counted on the inner
  shell's outer side matches the closed form.
"""
import numpy as np
import pytest

import oracle
from oracle import analytic as A


def _shell_geometry(lat, dims, shapes, tau=0.8, bc=oracle.BC_ELIBB_F, **kw):
    p = oracle.params(lat, dims, tau, bc=bc, **kw)
    flags, q, uw, uw1, tag, shell = oracle.geometry(p, shapes=shapes, with_shell=True)
    return p, flags, q, uw, uw1, tag, shell


def _coords(dims):
    nx, ny, nz = (list(dims) + [1, 1])[:3]
    n = np.arange(nx * ny * nz)
    return n % nx, (n // nx) % ny, n // (nx * ny), (nx, ny, nz)


def _nbr(dims, x, y, z, c):
    nx, ny, nz = dims
    return ((x + c[0]) % nx) + nx * (((y + c[1]) % ny) + ny * ((z + c[2]) % nz))


def _bisect(X, e, ctr, r, D):
    """Root in (0,1] of |X - t e - ctr| = r, by bisection on a sign change."""
    def g(t):
        d = (X - t * e - ctr)[:D]
        return float(d @ d) - r * r
    a, b = 0.0, 1.0
    ga = g(a)
    assert ga * g(b) <= 0.0
    for _ in range(80):
        m = 0.5 * (a + b)
        if (g(m) < 0.0) == (ga < 0.0):
            a = m
        else:
            b = m
    return 0.5 * (a + b)


SHELLS = {
    "d2q9": (oracle.D2Q9, (40, 36, 1),
             [dict(type=oracle.SHAPE_SHELL, tag=2, c=(19.3, 17.6, 0.0), r=(11.7, 0, 0))]),
    "d3q19": (oracle.D3Q19, (22, 20, 18),
              [dict(type=oracle.SHAPE_SHELL, tag=5, c=(10.4, 9.7, 8.6), r=(6.3, 0, 0))]),
    "d3q27": (oracle.D3Q27, (20, 18, 18),
              [dict(type=oracle.SHAPE_SHELL, tag=1, c=(9.6, 8.7, 9.2), r=(5.6, 0, 0))]),
}


@pytest.mark.parametrize("case", sorted(SHELLS))
def test_shell_links_are_crossings_seen_from_both_ends(oracle_lib, case):
    lat, dims, shapes = SHELLS[case]
    p, flags, q, uw, uw1, tag, shell = _shell_geometry(lat, dims, shapes)
    c, _, opp = oracle.lattice(lat)
    D = 2 if lat == oracle.D2Q9 else 3
    x, y, z, d3 = _coords(dims)
    ctr = np.array(shapes[0]["c"], float)
    r0 = shapes[0]["r"][0]
    assert (flags == oracle.FLUID).all()  # a thin shell makes no node solid
    inside = ((np.stack([x, y, z], 1)[:, :D] - ctr[:D]) ** 2).sum(1) < r0 * r0
    nshell = 0
    for n in range(len(flags)):
        X = np.array([x[n], y[n], z[n]], float)
        for i in range(1, len(c)):
            m = _nbr(d3, x[n], y[n], z[n], -c[i])
            crosses = inside[n] != inside[m]
            assert bool(shell[n, i]) == crosses
            if not crosses:
                assert q[n, i] == 0.0
                continue
            nshell += 1
            assert shell[n, i] == (2 if inside[n] else 1)
            assert shell[m, opp[i]] == (1 if inside[n] else 2)
            assert abs(q[n, i] - _bisect(X, c[i].astype(float), ctr, r0, D)) < 1e-12
            assert abs(q[n, i] + q[m, opp[i]] - 1.0) < 1e-12
            assert tag[n, i] == (-1 if inside[n] else shapes[0]["tag"])
    assert nshell > 50


def test_node_on_a_shell_is_rejected(oracle_lib):
    p = oracle.params(oracle.D2Q9, (24, 24, 1), 0.8)
    with pytest.raises(ValueError):
        oracle.geometry(p, shapes=[dict(type=oracle.SHAPE_SHELL, tag=0, c=(12, 12, 0), r=(5, 0, 0))],
                        with_shell=True)


ALL_BC = [oracle.BC_ELIBB_F, oracle.BC_ELIBB_FQ, oracle.BC_BFL, oracle.BC_HWBB, oracle.BC_ELIBB_U,
          oracle.BC_ELIBB_UQ]


@pytest.mark.parametrize("bc", ALL_BC)
@pytest.mark.parametrize("case", ["d2q9", "d3q19"])
def test_no_information_crosses_the_shell(oracle_lib, case, bc):
    lat, dims, shapes = SHELLS[case]
    shapes = [dict(shapes[0], om=(0.0, 0.0, 2e-3), om1=(0.0, 0.0, 2e-3))]  # a rotating shell
    p, flags, q, uw, uw1, tag, shell = _shell_geometry(lat, dims, shapes, tau=0.7, bc=bc,
                                                       force=(1e-5, -2e-5, 0.0))
    D = 2 if lat == oracle.D2Q9 else 3
    x, y, z, _ = _coords(dims)
    ctr = np.array(shapes[0]["c"], float)
    inside = ((np.stack([x, y, z], 1)[:, :D] - ctr[:D]) ** 2).sum(1) < shapes[0]["r"][0] ** 2
    _, w, _ = oracle.lattice(lat)
    rng = np.random.default_rng(3)
    f = w * (1.0 + 0.05 * rng.standard_normal((len(flags), len(w))))
    g = f.copy()
    g[~inside] *= 1.0 + 0.1 * rng.standard_normal(((~inside).sum(), len(w)))  # outside differs
    h = f.copy()
    h[inside] *= 1.0 + 0.1 * rng.standard_normal((inside.sum(), len(w)))      # inside differs
    for _ in range(6):
        f = oracle.step(p, flags, f, q, uw, uw1, shell=shell)
        g = oracle.step(p, flags, g, q, uw, uw1, shell=shell)
        h = oracle.step(p, flags, h, q, uw, uw1, shell=shell)
    assert np.array_equal(f[inside], g[inside])
    assert np.array_equal(f[~inside], h[~inside])
    assert not np.array_equal(f[~inside], g[~inside])


@pytest.mark.parametrize("case", sorted(SHELLS))
def test_bounce_back_conserves_mass_on_each_side(oracle_lib, case):
    lat, dims, shapes = SHELLS[case]
    p, flags, q, uw, uw1, tag, shell = _shell_geometry(lat, dims, shapes, tau=0.9, bc=oracle.BC_HWBB)
    D = 2 if lat == oracle.D2Q9 else 3
    x, y, z, _ = _coords(dims)
    ctr = np.array(shapes[0]["c"], float)
    inside = ((np.stack([x, y, z], 1)[:, :D] - ctr[:D]) ** 2).sum(1) < shapes[0]["r"][0] ** 2
    _, w, _ = oracle.lattice(lat)
    rng = np.random.default_rng(8)
    f = w * (1.0 + 0.05 * rng.standard_normal((len(flags), len(w))))
    m_in, m_out = f[inside].sum(), f[~inside].sum()
    for _ in range(20):
        f = oracle.step(p, flags, f, q, uw, uw1, shell=shell)
    assert abs(f[inside].sum() - m_in) / m_in < 1e-13
    assert abs(f[~inside].sum() - m_out) / m_out < 1e-13
    # the shell links are real walls: plain streaming would mix the two sides
    g = w * (1.0 + 0.05 * np.random.default_rng(8).standard_normal((len(flags), len(w))))
    for _ in range(20):
        g = oracle.step(p, flags, g, q, uw, uw1)
    assert abs(g[inside].sum() - m_in) / m_in > 1e-6


def thin_shell_couette(L, bc, collision=oracle.COLL_BGK, tau=0.8, steps_max=200, speed=0.01):
    """Inner shell r1 = L/4 rotating at om1 (wall speed `speed`), outer shell r2 = 0.45 L
    at rest, fluid everywhere in a periodic L x L box. Returns the relative errors
    inside r1, in the gap and outside r2, the torque on the inner shell from its
    outer side, and the closed-form torque."""
    R1, R2 = 0.25 * L, 0.45 * L
    cx = cy = L / 2.0 + 0.1  # no node on either shell
    om = speed / R1
    p = oracle.params(oracle.D2Q9, (L, L, 1), tau, bc=bc, collision=collision)
    shapes = [dict(type=oracle.SHAPE_SHELL, tag=1, c=(cx, cy, 0), r=(R1, 0, 0), om=(0, 0, om),
                   om1=(0, 0, om)),
              dict(type=oracle.SHAPE_SHELL, tag=2, c=(cx, cy, 0), r=(R2, 0, 0))]
    flags, q, uw, uw1, tag, shell = oracle.geometry(p, shapes=shapes, with_shell=True)
    X, Y = np.meshgrid(np.arange(L), np.arange(L))
    dx, dy = X.ravel() - cx, Y.ravel() - cy
    r = np.hypot(dx, dy)
    ut = np.where(r < R1, om * r, 0.0)
    gap = (r >= R1) & (r < R2)
    ut[gap] = A.cylindrical_couette(r[gap], R1, R2, om)
    uth = np.stack([-ut * dy / r, ut * dx / r, 0 * r], 1)
    s = oracle.Sim(p, flags, q, uw, uw1, oracle.init_eq(p, flags, None, uth), shell=shell)
    prev = s.macros()[1]
    for _ in range(steps_max):
        s.run(500)
        u = s.macros()[1]
        change = np.sqrt(((u - prev) ** 2).sum() / (u ** 2).sum())
        prev = u
        if change < 1e-10:
            break
    flink = s.run(1, want_force=True)
    # the force counts the outer fluid only (Sec. III.C): nothing on the inner side
    assert np.abs(flink[shell == 2]).max() == 0.0 and np.abs(flink[shell == 1]).max() > 0.0
    u = s.macros()[1]
    inner, outer = r < R1, r >= R2

    def err(region, ref_scale):
        return np.sqrt(((u[region] - uth[region]) ** 2).sum() / ref_scale)

    scale_in = (uth[inner] ** 2).sum()
    e_in = err(inner, scale_in)
    e_gap = err(gap, (uth[gap] ** 2).sum())
    e_out = err(outer, scale_in * outer.sum() / inner.sum())  # at rest: scaled by the inner speed
    # torque on the inner shell, its outer-side links only (tag 1), about the centre
    sel = tag == 1
    px = X.ravel()[:, None] - cx
    py = Y.ravel()[:, None] - cy
    torque = ((px * flink[:, :, 1] - py * flink[:, :, 0]) * sel).sum()
    mu = (tau - 0.5) / 3.0
    t_exact = -4.0 * np.pi * mu * om * R1 ** 2 * R2 ** 2 / (R2 ** 2 - R1 ** 2)
    return e_in, e_gap, e_out, torque, t_exact


@pytest.mark.parametrize("bc", [oracle.BC_ELIBB_F, oracle.BC_ELIBB_FQ])
def test_thin_shell_cylindrical_couette_second_order(oracle_lib, bc):
    """Diffusive scaling (wall speed 0.01 at L = 32, halved with each doubling): at a
    fixed speed the rigid rotation inside the inner shell carries a relative error
    proportional to the Mach number (its density follows the centrifugal
    pressure), which does not shrink with L."""
    res = [thin_shell_couette(L, bc, speed=0.01 * 32 / L) for L in (32, 64)]
    for k in range(2):  # inside, gap
        e32, e64 = res[0][k], res[1][k]
        assert e64 < 2e-3 and np.log2(e32 / e64) > 1.8, (k, e32, e64)
    # outside the outer shell (at rest) the fluid stays at rest to round-off
    assert max(res[0][2], res[1][2]) < 1e-12
    for e_in, e_gap, e_out, torque, t_exact in res[1:]:
        assert abs(torque / t_exact - 1.0) < 0.01, (torque, t_exact)
