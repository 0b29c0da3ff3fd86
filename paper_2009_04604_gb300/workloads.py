"""Seeded synthetic workloads: geometries and random fields, nothing of the method.

Each builder returns a plain dict that both the CUDA library and the FP64 oracle
consume. The dict holds the lattice, the dims, tau, the body force, the x-shear,
the base node kinds (walls, inlet, outlet), the base wall velocities and a list
of analytic shapes. Shapes are dicts with string types
('sphere', 'sphere_out', 'ellipsoid', 'strip'). The inputs follow the
workloads the paper tests on (Sec. III) and the benchmark configurations:
an inclined channel, circular Couette, a shear channel with an elliptic
cylinder, a sphere in a duct, a periodic porous
medium with a moving sphere, and batches of ducts.
"""
from __future__ import annotations

import math

import numpy as np

D2Q9, D3Q19 = 0, 1
FLUID, SOLID, OPEN = 0, 1, 2


def inclined_channel(g=1e-6, tau=0.8, steps=5000):
    """D2Q9 channel of width 40 between two walls at 30 degrees (29.98) to the x axis.

    A strip cannot be periodic in a 64x64 box at 30 degrees. The walls are
    therefore taken parallel to the lattice vector (26, 15), at 29.98 degrees,
    on a sheared-periodic 52 x 84 lattice where (x + 52, y + 30) is the node
    (x, y). One y-period spans 72.8 lattice units across the channel: 40 of fluid
    and 32.8 of solid. The body force g acts along the channel.
    """
    d = np.array([26.0, 15.0])
    d = d / np.linalg.norm(d)
    nrm = np.array([-d[1], d[0], 0.0])
    ny = 84
    period = ny * nrm[1]
    strip = dict(type="strip", tag=1, nrm=nrm, off=0.41 * period, width=40.0, period=period)
    return dict(lattice=D2Q9, dims=(52, ny, 1), tau=tau, xshift=30, force=(g * d[0], g * d[1], 0.0),
                base=None, base_u=None, shapes=[strip], steps=steps, rho0=1.0,
                channel_dir=(d[0], d[1], 0.0), channel_nrm=nrm, channel_off=0.41 * period,
                channel_width=40.0, channel_period=period, g=g)


def circular_couette(L, tau=0.8, u_inner=0.01, centre=None):
    """D2Q9 annulus between R1 = 0.25 L (rotating, tangential speed u_inner) and
    R2 = 0.45 L (at rest), centred in an L x L box (Sec. III.B)."""
    R1, R2 = 0.25 * L, 0.45 * L
    cx = cy = L / 2.0 if centre is None else centre
    om = u_inner / R1
    shapes = [dict(type="sphere", tag=1, c=(cx, cy, 0.0), r=(R1, 0, 0), om=(0, 0, om), om1=(0, 0, om)),
              dict(type="sphere_out", tag=2, c=(cx, cy, 0.0), r=(R2, 0, 0))]
    return dict(lattice=D2Q9, dims=(L, L, 1), tau=tau, xshift=0, force=(0.0, 0.0, 0.0),
                base=None, base_u=None, shapes=shapes, rho0=1.0, R1=R1, R2=R2, centre=(cx, cy),
                omega1=om)


def shear_channel_ellipse(nx=128, ny=98, U=0.04, tau=0.8, ra=8.0, rb=4.0, ang0=0.0):
    """D2Q9 shear channel for Jeffery's orbit (Sec. III.C): walls at rows 0 and
    ny-1 moving at -U/2 and +U/2 (half-way walls, so the channel height is
    H = ny - 2), the linear shear flow u_x = -U/2 + U (y - 1/2) / H as the initial
    state, and an elliptic cylinder at the centre with semi-axes rb along its body
    x axis and ra along its body y axis (vertical at ang0 = 0). Its moment of
    inertia is the solid ellipse's at density 1, pi ra rb (ra^2 + rb^2) / 4."""
    H = ny - 2
    y = np.arange(nx * ny) // nx
    base = np.zeros(nx * ny, np.uint8)
    base[(y == 0) | (y == ny - 1)] = SOLID
    base_u = np.zeros((nx * ny, 3))
    base_u[y == 0, 0] = -0.5 * U
    base_u[y == ny - 1, 0] = 0.5 * U
    u0 = np.zeros((nx * ny, 3))
    u0[:, 0] = -0.5 * U + U * (y - 0.5) / H
    centre = (nx / 2.0 - 0.3, (ny - 1) / 2.0, 0.0)
    body = dict(type="ellipsoid", tag=1, c=centre, r=(rb, ra, 1.0), ang=ang0)
    return dict(lattice=D2Q9, dims=(nx, ny, 1), tau=tau, xshift=0, force=(0.0, 0.0, 0.0), rho0=1.0,
                base=base, base_u=base_u, shapes=[], u0=u0, body=body,
                inertia=math.pi * ra * rb * (ra * ra + rb * rb) / 4.0, gamma=U / H, U=U, aspect=ra / rb)


def shear_channel_spheroid(nx=96, ny=74, nz=40, U=0.04, tau=0.8, ra=8.0, rb=4.0, ang0=0.0):
    """D3Q19 shear channel for the 3-D Jeffery's orbit (Sec. III.C): walls at
    y = 0 and y = ny-1 moving at -U/2 and +U/2 (H = ny - 2), periodic in x and z,
    the linear shear flow as the initial state, and a prolate spheroid at the
    centre with semi-axis ra along its body y axis (vertical at ang0 = 0) and rb
    along its body x and z axes. With its axis in the flow-gradient plane the
    spheroid turns about z only. Its moment of inertia about z is the solid
    spheroid's at density 1, m (ra^2 + rb^2) / 5 with m = 4/3 pi ra rb^2."""
    H = ny - 2
    N = nx * ny * nz
    y = (np.arange(N) // nx) % ny
    base = np.zeros(N, np.uint8)
    base[(y == 0) | (y == ny - 1)] = SOLID
    base_u = np.zeros((N, 3))
    base_u[y == 0, 0] = -0.5 * U
    base_u[y == ny - 1, 0] = 0.5 * U
    u0 = np.zeros((N, 3))
    u0[:, 0] = -0.5 * U + U * (y - 0.5) / H
    centre = (nx / 2.0 - 0.3, (ny - 1) / 2.0, nz / 2.0 + 0.2)
    body = dict(type="ellipsoid", tag=1, c=centre, r=(rb, ra, rb), ang=ang0)
    mass = 4.0 / 3.0 * math.pi * ra * rb * rb
    return dict(lattice=D3Q19, dims=(nx, ny, nz), tau=tau, xshift=0, force=(0.0, 0.0, 0.0), rho0=1.0,
                base=base, base_u=base_u, shapes=[], u0=u0, body=body,
                inertia=mass * (ra * ra + rb * rb) / 5.0, gamma=U / H, U=U, aspect=ra / rb)


def duct_base(dims, u_in):
    """Base node kinds of a duct along x: side walls at y, z = 0 and n-1; inlet plane
    x = 0 (a wall moving with u_in, half-way from the first fluid layer); open
    outlet plane x = nx - 1."""
    nx, ny, nz = dims
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    base = np.zeros((nz, ny, nx), np.uint8)
    base_u = np.zeros((nz, ny, nx, 3))
    side = (y == 0) | (y == ny - 1) | (z == 0) | (z == nz - 1)
    base[x == 0] = SOLID
    base_u[(x == 0) & ~side, 0] = u_in
    base[(x == nx - 1) & ~side] = OPEN
    base[side] = SOLID
    return base.reshape(-1), base_u.reshape(-1, 3)


def sphere_duct(dims=(256, 128, 128), radius=16.0, centre=(64.0, 64.0, 64.0), u_in=0.02, tau=0.7):
    """D3Q19 duct with velocity inlet, pressure outlet and a fixed sphere (config of
    the sphere-in-duct benchmark; Re = u D / nu = 9.6 at the defaults)."""
    base, base_u = duct_base(dims, u_in)
    sphere = dict(type="sphere", tag=1, c=centre, r=(radius, 0, 0))
    return dict(lattice=D3Q19, dims=tuple(dims), tau=tau, xshift=0, force=(0.0, 0.0, 0.0),
                base=base, base_u=base_u, shapes=[sphere], rho0=1.0, u_in=u_in)


def sphere_duct_small(u_in=0.02, tau=0.7):
    """64 x 32 x 32 downscale of the sphere duct: R = 4 at (16, 16, 16)."""
    return sphere_duct((64, 32, 32), 4.0, (16.0, 16.0, 16.0), u_in, tau)


def porous_spheres(n=384, porosity=0.6, rmin=6.0, rmax=12.0, seed=7, moving_radius=10.0,
                   amplitude=20.0, clearance=4.0, max_attempts=200000):
    """Periodic box of non-overlapping spheres placed largest first by random
    sequential addition (radii uniform in [rmin, rmax]) towards the target
    porosity. The box around the moving sphere's path (its extent along x plus
    moving_radius + clearance on every side) is kept free. Spheres that cross the
    periodic boundary are listed once per periodic image. Random sequential
    addition jams near a solid fraction of 0.4, so the attempt budget may stop
    short of the target. Returns (static shape list, achieved porosity, path
    centre)."""
    rng = np.random.default_rng(seed)
    L = float(n)
    target_solid = (1.0 - porosity) * L ** 3
    c0 = np.array([L / 2, L / 2, L / 2])
    half = np.array([amplitude + moving_radius + clearance, moving_radius + clearance,
                     moving_radius + clearance])
    mean_vol = 4.0 / 3.0 * math.pi * (rmax ** 4 - rmin ** 4) / (4 * (rmax - rmin))
    nwant = int(target_solid / mean_vol * 1.2) + 16
    radii = np.sort(rng.uniform(rmin, rmax, nwant))[::-1]
    cell = 2 * rmax
    nc = int(L // cell)
    grid = {}
    placed = []
    vol = 0.0
    attempts = 0
    for r in radii:
        if vol >= target_solid or attempts >= max_attempts:
            break
        for _ in range(200):
            attempts += 1
            p = rng.uniform(0, L, 3)
            # keep the box around the moving sphere's path free
            gap = np.maximum(np.abs(p - c0) - half, 0.0)
            if gap @ gap < r * r:
                continue
            ci = tuple(int(v // cell) % nc for v in p)
            ok = True
            for ox in (-1, 0, 1):
                for oy in (-1, 0, 1):
                    for oz in (-1, 0, 1):
                        for (q, rq) in grid.get(((ci[0] + ox) % nc, (ci[1] + oy) % nc, (ci[2] + oz) % nc), ()):
                            dd = p - q
                            dd -= L * np.round(dd / L)
                            if dd @ dd < (r + rq) ** 2:
                                ok = False
                                break
                        if not ok:
                            break
                    if not ok:
                        break
                if not ok:
                    break
            if ok:
                grid.setdefault(ci, []).append((p, r))
                placed.append((p, r))
                vol += 4.0 / 3.0 * math.pi * r ** 3
                break
    shapes = []
    for p, r in placed:
        for ox in (-1, 0, 1):
            for oy in (-1, 0, 1):
                for oz in (-1, 0, 1):
                    c = p + L * np.array([ox, oy, oz])
                    if np.all(c + r >= -1.0) and np.all(c - r <= L):
                        shapes.append(dict(type="sphere", tag=0, c=tuple(c), r=(r, 0, 0)))
    return shapes, 1.0 - vol / L ** 3, tuple(c0)


def moving_sphere(t, c0, radius=10.0, amplitude=20.0, period=5000.0, tag=1):
    """Sphere on the prescribed path c(t) = c0 + A sin(2 pi t / T) e_x, with its pose
    and velocity at t and t + 1 (velocity = time derivative of the path)."""
    w = 2.0 * math.pi / period
    def pos(s):
        return (c0[0] + amplitude * math.sin(w * s), c0[1], c0[2])
    def vel(s):
        return (amplitude * w * math.cos(w * s), 0.0, 0.0)
    return dict(type="sphere", tag=tag, c=pos(t), r=(radius, 0, 0), v=vel(t), v1=vel(t + 1))


def random_fields(N, seed=0, amp_rho=0.02, amp_u=0.02, amp_neq=0.01, Q=19, two_d=False):
    """Seeded random density, velocity and per-population noise for parity tests."""
    rng = np.random.default_rng(seed)
    rho = 1.0 + amp_rho * rng.standard_normal(N)
    u = amp_u * rng.standard_normal((N, 3))
    if two_d:
        u[:, 2] = 0.0
    xi = amp_neq * rng.standard_normal((N, Q))
    return rho, u, xi


def random_geometry(dims, seed=0, solid_frac=0.15, open_frac=0.02, Q=19, moving=True):
    """Random node kinds and per-link q in (0,1], wall velocities and tags (stress input
    for the boundary rules: narrow gaps, corners, every q branch)."""
    rng = np.random.default_rng(seed)
    N = int(np.prod(dims))
    r = rng.random(N)
    flags = np.where(r < solid_frac, SOLID, np.where(r < solid_frac + open_frac, OPEN, FLUID)).astype(np.uint8)
    q = rng.uniform(0.0, 1.0, (N, Q))
    q = np.where(q < 1e-3, 1e-3, q)
    # hit the special values too
    special = rng.random((N, Q))
    q = np.where(special < 0.05, 0.5, q)
    q = np.where((special >= 0.05) & (special < 0.08), 1.0, q)
    q = np.where((special >= 0.08) & (special < 0.10), 0.005, q)
    uw = 0.02 * rng.standard_normal((N, Q, 3)) if moving else None
    uw1 = uw + 0.001 * rng.standard_normal((N, Q, 3)) if moving else None
    tag = rng.integers(0, 8, (N, Q)).astype(np.int32)
    return flags, q, uw, uw1, tag


def batched_ducts(n=96, lo=48, hi=192, target=1.2e8, tol=0.05, seed=11, rmin=6.0, rmax=20.0,
                  u_lo=0.005, u_hi=0.03, tau=0.7, max_draws=10000):
    """n independent D3Q19 ducts of uneven sizes (the batched configuration).

    Each axis is drawn uniformly from {lo..hi}. Independent draws average
    96 * 120^3 = 1.66e8 nodes, so a total near the 1.2e8 target is very unlikely.
    While the total exceeds target*(1 + tol), one randomly chosen duct is
    redrawn, and the draw is kept when it brings the total down. This keeps every
    axis in {lo..hi} and ends within target*(1 +- tol). A target of None keeps
    the first draw. Each duct holds a sphere or an axis-aligned
    ellipsoid with semi-axes in [rmin, rmax], clamped to fit, at a random interior
    position at least 4 nodes from the walls, and gets an inlet speed in
    [u_lo, u_hi]. Returns a list of workload dicts."""
    rng = np.random.default_rng(seed)
    dims = rng.integers(lo, hi + 1, size=(n, 3))
    vol = np.prod(dims, axis=1)
    for _ in range(max_draws):
        if target is None or vol.sum() <= target * (1 + tol):
            break
        j = int(rng.integers(n))
        d = rng.integers(lo, hi + 1, size=3)
        if np.prod(d) < vol[j]:
            dims[j] = d
            vol[j] = np.prod(d)
    out = []
    for j in range(n):
        d = tuple(int(v) for v in dims[j])
        u_in = float(rng.uniform(u_lo, u_hi))
        room = (min(d) - 2) / 2.0 - 4.0
        if rng.random() < 0.5:
            r = float(np.clip(rng.uniform(rmin, rmax), 1.0, max(1.0, room)))
            axes = (r, r, r)
            kind = "sphere"
        else:
            axes = tuple(float(np.clip(rng.uniform(rmin, rmax), 1.0, max(1.0, (d[a] - 2) / 2.0 - 4.0)))
                         for a in range(3))
            kind = "ellipsoid"
        c = tuple(float(rng.uniform(1 + axes[a] + 4, d[a] - 2 - axes[a] - 4)) if d[a] - 2 - axes[a] - 4 > 1 + axes[a] + 4
                  else (d[a] - 1) / 2.0 for a in range(3))
        base, base_u = duct_base(d, u_in)
        shape = dict(type="sphere", tag=1, c=c, r=(axes[0], 0, 0)) if kind == "sphere" else \
            dict(type="ellipsoid", tag=1, c=c, r=axes)
        out.append(dict(lattice=D3Q19, dims=d, tau=tau, xshift=0, force=(0.0, 0.0, 0.0), base=base,
                        base_u=base_u, shapes=[shape], rho0=1.0, u_in=u_in))
    return out


def porous_with_moving_sphere(n=384, seed=7, rmin=6.0, rmax=12.0, moving_radius=10.0, amplitude=20.0,
                              period=5000, tau=0.65, g=1e-6, porosity=0.6, max_attempts=200000):
    """The porous-medium configuration: D3Q19, periodic n^3 box of static spheres,
    one sphere of radius moving_radius moving on c(t) = c0 + A sin(2 pi t / T) e_x,
    and a body force g along x. The trajectory table holds one period of poses
    (centre, velocity = path derivative, zero angular velocity)."""
    shapes, por, c0 = porous_spheres(n, porosity, rmin, rmax, seed, moving_radius, amplitude,
                                     max_attempts=max_attempts)
    w = 2.0 * math.pi / period
    t = np.arange(period)
    traj = np.zeros((period, 9))
    traj[:, 0] = c0[0] + amplitude * np.sin(w * t)
    traj[:, 1] = c0[1]
    traj[:, 2] = c0[2]
    traj[:, 3] = amplitude * w * np.cos(w * t)
    body = dict(type="sphere", tag=1, r=(moving_radius, 0, 0))
    return dict(lattice=D3Q19, dims=(n, n, n), tau=tau, xshift=0, force=(g, 0.0, 0.0), base=None,
                base_u=None, shapes=shapes, rho0=1.0, body=body, traj=traj, porosity=por)
