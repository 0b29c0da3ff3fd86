"""Pins of the oracle's rigid-body pieces (Sec. III.C, App. D): the rotated
ellipse/ellipsoid geometry and the torque of the momentum exchange.

- Geometry: flags by brute force and q by bisection against an independent
  inside test written as a quadratic form (x - c)^T R D R^T (x - c) <= 1; a
  quarter turn equals the ellipse with its axes swapped.
- Torque: circular Couette flow at steady state (Sec. III.B), where the torque on
  the inner cylinder has the closed form 4 pi mu w1 r1^2 r2^2 / (r2^2 - r1^2) and
  the two cylinders' torques are equal and opposite; and a field of random link
  forces, where the sum is checked link by link from the wall points."""
import numpy as np
import pytest

import oracle
from oracle import analytic as A


def _bisect(inside, X, c, steps=200):
    lo, hi = 0.0, 1.0  # inside(X - lo c) is False, inside(X - hi c) is True
    for _ in range(steps):
        mid = 0.5 * (lo + hi)
        if inside(X - mid * c):
            hi = mid
        else:
            lo = mid
    return 0.5 * (lo + hi)


def _quadform(cen, ax, ang):
    """Inside test of the rotated ellipsoid as a quadratic form: body axes are the
    columns of R (the x, y axes turned by ang about z)."""
    ca, sa = np.cos(ang), np.sin(ang)
    R = np.array([[ca, -sa, 0.0], [sa, ca, 0.0], [0.0, 0.0, 1.0]])
    Amat = R @ np.diag(np.asarray(ax, float) ** -2.0) @ R.T

    def inside(X):
        d = X - cen
        return float(d @ Amat @ d) <= 1.0
    return inside


@pytest.mark.parametrize("lat,dims,cen,ax,ang", [
    (oracle.D2Q9, (40, 36, 1), (19.3, 17.6, 0.0), (10.2, 4.7, 1.0), 0.61),
    (oracle.D2Q9, (40, 36, 1), (19.3, 17.6, 0.0), (4.4, 11.3, 1.0), -2.3),
    (oracle.D3Q19, (24, 22, 16), (11.4, 10.7, 7.6), (8.3, 3.9, 4.6), 1.1),
])
def test_rotated_ellipsoid_flags_and_q(oracle_lib, lat, dims, cen, ax, ang):
    cen = np.array(cen)
    shape = dict(type=oracle.SHAPE_ELLIPSOID, c=cen, r=ax, ang=ang)
    p = oracle.params(lat, dims, 0.8)
    flags, q, _, _, _ = oracle.geometry(p, shapes=[shape])
    inside = _quadform(cen, ax if lat != oracle.D2Q9 else (ax[0], ax[1], 1e100), ang)
    c, _, _ = oracle.lattice(lat)
    nx, ny, nz = dims
    ncut = 0
    for n in range(nx * ny * nz):
        X = np.array([n % nx, (n // nx) % ny, n // (nx * ny)], float)
        assert flags[n] == (oracle.SOLID if inside(X) else oracle.FLUID), n
        if flags[n] != oracle.FLUID:
            continue
        for i in range(1, len(c)):
            Y = X - c[i]
            m = int(Y[0] % nx + nx * (Y[1] % ny + ny * (Y[2] % nz)))
            if flags[m] == oracle.FLUID:
                continue
            ncut += 1
            qb = _bisect(inside, X, c[i].astype(float))
            assert abs(q[n, i] - qb) < 1e-12, (n, i, q[n, i], qb)
    assert ncut > 30


def test_quarter_turn_swaps_the_axes(oracle_lib):
    p = oracle.params(oracle.D2Q9, (36, 36, 1), 0.8)
    cen = (17.4, 18.2, 0.0)
    a = dict(type=oracle.SHAPE_ELLIPSOID, c=cen, r=(9.6, 5.1, 1.0), ang=np.pi / 2)
    b = dict(type=oracle.SHAPE_ELLIPSOID, c=cen, r=(5.1, 9.6, 1.0), ang=0.0)
    fa, qa, *_ = oracle.geometry(p, shapes=[a])
    fb, qb, *_ = oracle.geometry(p, shapes=[b])
    assert np.array_equal(fa, fb)
    assert np.abs(qa - qb).max() < 1e-12


def test_torque_closed_form_circular_couette(oracle_lib):
    """Steady circular Couette (D2Q9, ELIBB-F): torque about the centre on the inner
    cylinder = -4 pi mu w1 r1^2 r2^2/(r2^2 - r1^2) (closed form), and the outer
    cylinder's torque is its opposite."""
    L, tau, uin = 32, 0.8, 0.01
    R1, R2 = 0.25 * L, 0.45 * L
    cx = cy = L / 2.0
    om = uin / R1
    p = oracle.params(oracle.D2Q9, (L, L, 1), tau, bc=oracle.BC_ELIBB_F)
    shapes = [dict(type=oracle.SHAPE_SPHERE, tag=1, c=(cx, cy, 0), r=(R1, 0, 0), om=(0, 0, om), om1=(0, 0, om)),
              dict(type=oracle.SHAPE_SPHERE_OUT, tag=2, c=(cx, cy, 0), r=(R2, 0, 0))]
    flags, q, uw, uw1, tag = oracle.geometry(p, shapes=shapes)
    X, Y = np.meshgrid(np.arange(L), np.arange(L))
    dx, dy = X.ravel() - cx, Y.ravel() - cy
    r = np.hypot(dx, dy)
    fl = flags == oracle.FLUID
    ut = np.zeros(r.size)
    ut[fl] = A.cylindrical_couette(r[fl], R1, R2, om)
    rs = np.where(r > 0, r, 1.0)
    uth = np.stack([-ut * dy / rs, ut * dx / rs, 0 * r], 1)
    s = oracle.Sim(p, flags, q, uw, uw1, oracle.init_eq(p, flags, None, uth))
    s.run(6000)
    flink = s.run(1, want_force=True)
    T1 = oracle.torque(p, q, tag, flink, (cx, cy, 0.0), 1)
    T2 = oracle.torque(p, q, tag, flink, (cx, cy, 0.0), 2)
    Tth = A.couette_torque(1.0, (tau - 0.5) / 3.0, om, R1, R2)
    assert abs(T1[0]) + abs(T1[1]) < 1e-12 * Tth    # in-plane forces have a z torque only
    assert abs(T1[2] + Tth) / Tth < 5e-3, (T1[2], Tth)
    assert abs(T1[2] + T2[2]) / Tth < 2e-3


def test_torque_of_random_link_forces(oracle_lib):
    """Link by link: each cut link contributes (x_F - q c_i - c) x F_link."""
    p = oracle.params(oracle.D3Q19, (14, 12, 10), 0.8)
    cen = np.array([6.6, 5.3, 4.8])
    shape = dict(type=oracle.SHAPE_ELLIPSOID, tag=4, c=cen, r=(3.9, 2.7, 3.1), ang=0.4)
    flags, q, uw, uw1, tag = oracle.geometry(p, shapes=[shape])
    rng = np.random.default_rng(3)
    flink = rng.standard_normal((flags.size, 19, 3))
    c, _, _ = oracle.lattice(oracle.D3Q19)
    ref = np.zeros(3)
    for n, i in np.argwhere(q > 0):
        X = np.array([n % 14, (n // 14) % 12, n // 168], float)
        ref += np.cross(X - q[n, i] * c[i] - cen, flink[n, i])
    got = oracle.torque(p, q, tag, flink, cen, 4)
    assert np.abs(got - ref).max() < 1e-11 * np.abs(ref).max()
    assert np.abs(oracle.torque(p, q, tag, flink, cen, 3)).max() == 0.0  # no link has tag 3


def _fresh_case(lat=oracle.D2Q9):
    """A periodic box with a small solid disc at t that is gone at t+1 (its nodes
    turn fluid), and a random non-equilibrium state at t."""
    dims = (20, 18, 1) if lat == oracle.D2Q9 else (14, 12, 10)
    p = oracle.params(lat, dims, 0.8, force=(1e-5, -2e-5, 0.0))
    cen = (9.3, 8.6, 0.0) if lat == oracle.D2Q9 else (6.3, 5.6, 4.4)
    old, *_ = oracle.geometry(p, shapes=[dict(type=oracle.SHAPE_SPHERE, c=cen, r=(2.4, 0, 0))])
    new = np.zeros_like(old)
    Q = {oracle.D2Q9: 9, oracle.D3Q19: 19, oracle.D3Q27: 27}[lat]
    N = old.size
    rng = np.random.default_rng(8)
    u = 0.02 * rng.standard_normal((N, 3))
    if lat == oracle.D2Q9:
        u[:, 2] = 0
    fprev = oracle.init_eq(p, old, 1.0 + 0.01 * rng.standard_normal(N), u) * (1 + 0.01 * rng.standard_normal((N, Q)))
    fprev[old != 0] = 0.0
    return p, old, new, fprev


@pytest.mark.parametrize("lat", [oracle.D2Q9, oracle.D3Q19])
def test_lir_takes_the_streamed_values(oracle_lib, lat):
    """Directions whose upstream node was fluid at t carry what streaming delivers:
    the same values or_step writes when the node is fluid (Eq. LBE)."""
    p, old, new, fprev = _fresh_case(lat)
    fresh = np.nonzero((old != 0) & (new == 0))[0]
    assert fresh.size > 3
    streamed = oracle.step(p, new, fprev)        # the fresh nodes as fluid nodes
    f = np.zeros_like(fprev)
    oracle.refill_lir(p, old, new, None, fprev, f, K=3)
    c, _, _ = oracle.lattice(lat)
    nx, ny, nz = p.nx, p.ny, p.nz
    checked = 0
    for n in fresh:
        X = np.array([n % nx, (n // nx) % ny, n // (nx * ny)])
        for i in range(len(c)):
            Y = X - c[i]
            m = int(Y[0] % nx + nx * (Y[1] % ny + ny * (Y[2] % nz)))
            if old[m] == 0:
                assert f[n, i] == streamed[n, i], (n, i)
                checked += 1
    assert checked > 10


def test_lir_keeps_a_uniform_flow_moving_with_the_body(oracle_lib):
    """Uniform equilibrium flow at U and a wall moving at U: equilibrium is a fixed
    point of the collision, and bouncing back f*_ibar plus 2 w_i rho c_i.U / c_s^2
    gives f^eq_i(rho0, U), so the refill restores the equilibrium exactly."""
    p = oracle.params(oracle.D3Q19, (12, 10, 9), 0.7)
    old, *_ = oracle.geometry(p, shapes=[dict(type=oracle.SHAPE_SPHERE, c=(5.7, 4.4, 4.2), r=(2.2, 0, 0))])
    new = np.zeros_like(old)
    U = np.array([0.03, -0.01, 0.02])
    uu = np.tile(U, (old.size, 1))
    fprev = oracle.init_eq(p, old, None, uu)
    f = oracle.step(p, old, fprev)
    oracle.refill_lir(p, old, new, uu, fprev, f, K=4)
    ref = oracle.init_eq(p, new, None, uu)
    fresh = (old != 0) & (new == 0)
    assert fresh.sum() > 10
    assert np.abs(f[fresh] - ref[fresh]).max() < 1e-15


def test_lir_iteration_start_and_fixed_point(oracle_lib):
    """K = 0 leaves the start f^eq(rho0, u_body) in the unknown directions; the
    iterations converge to the fixed point f_i = f*_ibar + 2 w_i rho c_i.u_b / c_s^2,
    with f* the BGK collision at the node's density and the body velocity."""
    p, old, new, fprev = _fresh_case()
    p.force[0] = p.force[1] = 0.0
    fresh = np.nonzero((old != 0) & (new == 0))[0]
    ub = np.tile([0.01, -0.02, 0.0], (old.size, 1))
    f0 = np.zeros_like(fprev)
    oracle.refill_lir(p, old, new, ub, fprev, f0, K=0)
    c, w, opp = oracle.lattice(oracle.D2Q9)
    feq = oracle.init_eq(p, new, None, ub)
    fk = np.zeros_like(fprev)
    oracle.refill_lir(p, old, new, ub, fprev, fk, K=5000)
    nx, ny = p.nx, p.ny
    one = oracle.params(oracle.D2Q9, (1, 1, 1), p.tau)
    for n in fresh:
        X = np.array([n % nx, n // nx, 0])
        unknown = [i for i in range(9) if old[int((X[0] - c[i][0]) % nx + nx * ((X[1] - c[i][1]) % ny))] != 0]
        assert unknown
        for i in unknown:
            assert f0[n, i] == feq[n, i]
        fn = fk[n]
        rho = fn.sum()
        eq = oracle.init_eq(one, np.zeros(1, np.uint8), np.array([rho]), ub[n][None, :])[0]
        post = fn - (fn - eq) / p.tau
        for i in unknown:
            target = post[opp[i]] + 2 * w[i] * rho * (c[i] @ ub[n]) * 3.0
            assert abs(fn[i] - target) < 1e-13, (n, i, fn[i], target)


def test_free_cylinder_spins_at_half_the_shear_rate(oracle_lib):
    """A free circular cylinder at the centre of a shear channel turns at the
    fluid's own rotation rate, half its vorticity: omega = -gamma/2 for
    u_x = gamma y. This pins free_rotation as a whole, in its sign and its size:
    the torque of the link forces about the centre, the wall velocity
    omega x (x_W - c) of the rotating wall and the Euler update of omega. A
    circle covers the same nodes at every angle, so no refill takes part. The
    spin-up time I / (4 pi mu R^2) is about 11 steps; at 200 steps the rate is
    within 1% of -gamma/2 (the walls, 14 radii apart here, shift it by a few
    parts in a thousand)."""
    from paper_2009_04604_gb300 import workloads as W
    R = 3.0
    ch = W.shear_channel_ellipse(nx=48, ny=34, U=0.02, tau=0.8, ra=R, rb=R)
    body = dict(ch["body"], type=oracle.SHAPE_SPHERE, r=(R, 0.0, 0.0))
    p = oracle.params(oracle.D2Q9, ch["dims"], ch["tau"])
    flags, *_ = oracle.geometry(p, ch["base"], ch["base_u"], [body])
    f0 = oracle.init_eq(p, flags, None, ch["u0"])
    inertia = np.pi * R ** 4 / 2.0       # solid disc of density 1
    _, _, h = oracle.free_rotation(p, ch["base"], ch["base_u"], body, inertia, f0, 200)
    ratio = h[-1, 1] / (-0.5 * ch["gamma"])
    assert abs(ratio - 1.0) < 0.01, ratio
    # the angle is the running sum of the rates
    assert np.allclose(np.cumsum(h[:, 1]), h[:, 0], rtol=0, atol=1e-15)


def test_jeffery_reference_follows_the_closed_form():
    """The oracle's Jeffery runs stored in tests/golden/jeffery_ellipse_128x98.npz
    (written by make_jeffery_reference.py from oracle.free_rotation) against what
    the paper fixes: the angle follows Jeffery's closed form for the aspect ratio
    r_a / r_b = 2 (Sec. III.C; the quarter turn within 8 % and the angle within
    0.1 rad), and the torque squared fluctuation (App. D) orders as the paper
    reports: without a refill scheme the local rule ELIBB-F fluctuates well above
    BFL, with the local iteration refill it drops and comes close to BFL."""
    import math
    import os
    ref = np.load(os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "jeffery_ellipse_128x98.npz"))
    nx, ny, U, tau, ra, rb = ref["channel"]
    gam, aspect = U / (ny - 2), ra / rb
    every = int(ref["every"])
    t_quarter = (math.pi / 2) * (aspect * aspect + 1) / (gam * aspect)
    for key in ("elibb_f_lir0", "elibb_f_lir12", "bfl_lir0", "bfl_lir12"):
        theta = -ref[key + "_angle"]
        t = every * np.arange(1, theta.size + 1, dtype=float)
        assert np.abs(theta - A.jeffery_angle(t, gam, aspect)).max() < 0.1, key
        assert abs(int(ref[key + "_quarter"]) - t_quarter) < 0.08 * t_quarter, key
    tsf = {k: float(ref[k + "_tsf"]) for k in ("elibb_f_lir0", "elibb_f_lir12", "bfl_lir0", "bfl_lir12")}
    assert tsf["elibb_f_lir0"] > 2.0 * tsf["bfl_lir0"]
    assert tsf["elibb_f_lir12"] < 0.7 * tsf["elibb_f_lir0"]
    assert tsf["elibb_f_lir12"] < 1.5 * tsf["bfl_lir12"]
