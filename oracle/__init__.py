"""FP64 CPU oracle for the ELIBB lattice Boltzmann hot path (TEST INFRASTRUCTURE).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package. It shares no code with the CUDA library
(``paper_2009_04604_gb300``) and neither imports the other.

The arithmetic lives in ``lbm_oracle.c`` (plain C, ``-ffp-contract=off``); this
module compiles it with gcc and wraps it with ctypes. Array conventions follow
``lbm_oracle.h``: node ``n = x + nx*(y + ny*z)``, populations ``f[n, i]``,
per-link data ``q[n, i]`` for the link from node ``n`` towards ``n - c_i``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liblbm_oracle.so")
_lock = threading.Lock()
_lib = None

D2Q9, D3Q19, D3Q27 = 0, 1, 2
FLUID, SOLID, OPEN = 0, 1, 2
BC_ELIBB_F, BC_ELIBB_FQ, BC_BFL, BC_HWBB, BC_ELIBB_U, BC_ELIBB_UQ = 0, 1, 2, 3, 4, 5
SHAPE_SPHERE, SHAPE_SPHERE_OUT, SHAPE_ELLIPSOID, SHAPE_STRIP, SHAPE_SHELL = 0, 1, 2, 3, 4
COLL_BGK, COLL_TRT = 0, 1
NEQ_BOUNCE_BACK, NEQ_REGULARIZED = 0, 1


def build(force: bool = False) -> str:
    """Compile the oracle into ``oracle/_build/liblbm_oracle.so`` (gcc, OpenMP)."""
    src = os.path.join(_HERE, "lbm_oracle.c")
    hdr = os.path.join(_HERE, "lbm_oracle.h")
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= max(os.path.getmtime(src), os.path.getmtime(hdr))):
        return _LIB_PATH
    os.makedirs(_BUILD, exist_ok=True)
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fopenmp",
           "-fPIC", "-shared", src, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class Params(ctypes.Structure):
    _fields_ = [("lattice", ctypes.c_int), ("nx", ctypes.c_int), ("ny", ctypes.c_int),
                ("nz", ctypes.c_int), ("xshift", ctypes.c_int), ("bc", ctypes.c_int),
                ("tau", ctypes.c_double), ("rho0", ctypes.c_double),
                ("force", ctypes.c_double * 3), ("qcut", ctypes.c_double),
                ("wall_neq_same", ctypes.c_int), ("me_rho0", ctypes.c_int),
                ("s1_exact", ctypes.c_int), ("collision", ctypes.c_int), ("wall_neq", ctypes.c_int),
                ("magic", ctypes.c_double)]


class Shape(ctypes.Structure):
    _fields_ = [("type", ctypes.c_int), ("tag", ctypes.c_int),
                ("c", ctypes.c_double * 3), ("r", ctypes.c_double * 3),
                ("nrm", ctypes.c_double * 3), ("off", ctypes.c_double),
                ("width", ctypes.c_double), ("period", ctypes.c_double),
                ("v", ctypes.c_double * 3), ("om", ctypes.c_double * 3),
                ("v1", ctypes.c_double * 3), ("om1", ctypes.c_double * 3),
                ("ang", ctypes.c_double)]


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            P = ctypes.POINTER
            d, i32, u8 = P(ctypes.c_double), P(ctypes.c_int32), P(ctypes.c_uint8)
            lib.or_lattice.argtypes = [ctypes.c_int, P(ctypes.c_int), d, P(ctypes.c_int)]
            lib.or_init_eq.argtypes = [P(Params), u8, d, d, d]
            lib.or_step.argtypes = [P(Params), u8, d, u8, d, d, d, d, d]
            lib.or_macros.argtypes = [P(Params), u8, d, d, d]
            lib.or_mass.argtypes = [P(Params), u8, d]
            lib.or_mass.restype = ctypes.c_double
            lib.or_refill.argtypes = [P(Params), u8, u8, d, d]
            lib.or_geometry.argtypes = [P(Params), u8, d, P(Shape), ctypes.c_int, u8, d, d, d, i32, u8]
            lib.or_geometry.restype = ctypes.c_long
            lib.or_bc_weights.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_double, d, d]
            lib.or_torque.argtypes = [P(Params), d, i32, d, ctypes.c_int, d, d]
            lib.or_refill_lir.argtypes = [P(Params), u8, u8, d, d, ctypes.c_int, d]
            _lib = lib
    return _lib


def _ptr(a, ctype):
    if a is None:
        return None
    return a.ctypes.data_as(ctypes.POINTER(ctype))


def _dp(a):
    return _ptr(a, ctypes.c_double)


def lattice(lat: int):
    """Oracle lattice tables ``(c[Q,3] int, w[Q], opp[Q])``."""
    lib = _load()
    c = np.zeros((27, 3), np.int32)
    w = np.zeros(27)
    opp = np.zeros(27, np.int32)
    Qn = lib.or_lattice(lat, _ptr(c, ctypes.c_int), _dp(w), _ptr(opp, ctypes.c_int))
    return c[:Qn].copy(), w[:Qn].copy(), opp[:Qn].copy()


def params(lattice_id, dims, tau, bc=BC_ELIBB_F, rho0=1.0, force=(0.0, 0.0, 0.0), xshift=0,
           qcut=0.01, wall_neq_same=0, me_rho0=0, s1_exact=0, collision=0, magic=0.1875,
           wall_neq=0) -> Params:
    nx, ny, nz = (list(dims) + [1, 1])[:3]
    p = Params()
    p.lattice, p.nx, p.ny, p.nz, p.xshift, p.bc = lattice_id, nx, ny, nz, xshift, bc
    p.tau, p.rho0, p.qcut = tau, rho0, qcut
    for a in range(3):
        p.force[a] = float(force[a])
    p.wall_neq_same, p.me_rho0, p.s1_exact = wall_neq_same, me_rho0, s1_exact
    p.collision, p.magic, p.wall_neq = collision, magic, wall_neq
    return p


def _Q(p):
    return {D2Q9: 9, D3Q19: 19, D3Q27: 27}[p.lattice]


def _N(p):
    return p.nx * p.ny * p.nz


def _c8(a):
    return np.ascontiguousarray(a, dtype=np.uint8)


def _cd(a):
    return None if a is None else np.ascontiguousarray(a, dtype=np.float64)


def init_eq(p, flags, rho=None, u=None):
    f = np.zeros((_N(p), _Q(p)))
    rho = _cd(None if rho is None else np.reshape(rho, -1))
    u = _cd(None if u is None else np.reshape(u, (-1, 3)))
    _load().or_init_eq(ctypes.byref(p), _ptr(_c8(flags), ctypes.c_uint8), _dp(rho), _dp(u), _dp(f))
    return f


def step(p, flags, f, q=None, uw=None, uw1=None, want_force=False, shell=None):
    """One update; returns ``fout`` or ``(fout, flink[N,Q,3])``. ``shell[N,Q]``
    marks the links that cross a thin shell (1: node outside, 2: inside)."""
    f = _cd(f)
    fout = np.empty_like(f)
    flink = np.zeros((_N(p), _Q(p), 3)) if want_force else None
    sh = None if shell is None else _c8(shell)
    rc = _load().or_step(ctypes.byref(p), _ptr(_c8(flags), ctypes.c_uint8), _dp(_cd(q)),
                         _ptr(sh, ctypes.c_uint8), _dp(_cd(uw)), _dp(_cd(uw1)), _dp(f), _dp(fout),
                         _dp(flink))
    if rc != 0:
        raise ValueError("or_step rejected its arguments")
    return (fout, flink) if want_force else fout


def macros(p, flags, f):
    rho = np.zeros(_N(p))
    u = np.zeros((_N(p), 3))
    _load().or_macros(ctypes.byref(p), _ptr(_c8(flags), ctypes.c_uint8), _dp(_cd(f)), _dp(rho), _dp(u))
    return rho, u


def mass(p, flags, f) -> float:
    return _load().or_mass(ctypes.byref(p), _ptr(_c8(flags), ctypes.c_uint8), _dp(_cd(f)))


def refill(p, flags_old, flags_new, un, f):
    """In place: nodes that turned fluid get f^eq(rho0, un[n])."""
    assert f.dtype == np.float64 and f.flags.c_contiguous
    _load().or_refill(ctypes.byref(p), _ptr(_c8(flags_old), ctypes.c_uint8),
                      _ptr(_c8(flags_new), ctypes.c_uint8), _dp(_cd(un)), _dp(f))
    return f


def refill_lir(p, flags_old, flags_new, un, fprev, f, K=5):
    """In place: local iteration refill of the nodes that turned fluid (see
    or_refill_lir): streamed values from upstream nodes fluid at t (post-collision
    values of fprev), the rest from K local collide-and-bounce-back iterations."""
    assert f.dtype == np.float64 and f.flags.c_contiguous
    _load().or_refill_lir(ctypes.byref(p), _ptr(_c8(flags_old), ctypes.c_uint8),
                          _ptr(_c8(flags_new), ctypes.c_uint8), _dp(_cd(un)), _dp(_cd(fprev)), int(K), _dp(f))
    return f


def make_shapes(specs):
    """Build a ctypes array of Shape from dicts (keys as in ``Shape``)."""
    arr = (Shape * max(1, len(specs)))()
    for k, s in enumerate(specs):
        for key, val in s.items():
            if isinstance(val, (list, tuple, np.ndarray)):
                dst = getattr(arr[k], key)
                for a, x in enumerate(val):
                    dst[a] = float(x)
            else:
                setattr(arr[k], key, val)
    return arr


def geometry(p, base=None, base_u=None, shapes=(), with_shell=False):
    """Flags and per-link q, u_w(t), u_w(t+1), tag from analytic shapes; with
    ``with_shell`` also the thin-shell marks ``shell[N,Q]`` that ``step`` takes.
    Raises ValueError when a fluid node lies exactly on a thin shell."""
    N, Qn = _N(p), _Q(p)
    flags = np.zeros(N, np.uint8)
    q = np.zeros((N, Qn))
    uw = np.zeros((N, Qn, 3))
    uw1 = np.zeros((N, Qn, 3))
    tag = np.zeros((N, Qn), np.int32)
    shell = np.zeros((N, Qn), np.uint8)
    arr = make_shapes(list(shapes))
    base = None if base is None else _c8(np.reshape(base, -1))
    base_u = _cd(None if base_u is None else np.reshape(base_u, (-1, 3)))
    rc = _load().or_geometry(ctypes.byref(p), _ptr(base, ctypes.c_uint8), _dp(base_u), arr,
                             len(shapes), _ptr(flags, ctypes.c_uint8), _dp(q), _dp(uw), _dp(uw1),
                             _ptr(tag, ctypes.c_int32), _ptr(shell, ctypes.c_uint8))
    if rc == -2:
        raise ValueError("a fluid node lies exactly on a thin shell")
    if rc < 0:
        raise ValueError("or_geometry rejected its arguments")
    if with_shell:
        return flags, q, uw, uw1, tag, shell
    return flags, q, uw, uw1, tag


def set_threads(n=0):
    """OpenMP threads of the oracle's loops (n <= 0 keeps the setting); returns
    the number in use."""
    lib = _load()
    lib.or_set_threads.restype = ctypes.c_int
    return int(lib.or_set_threads(int(n)))


def torque(p, q, tag, flink, centre, want_tag=-1):
    """Torque about ``centre`` of the link forces ``flink`` (from ``step``) of the
    links with tag ``want_tag`` (-1: all): sum (x_W - c) x F, x_W = x_F - q c_i."""
    T = np.zeros(3)
    c = np.ascontiguousarray(centre, dtype=np.float64)
    _load().or_torque(ctypes.byref(p), _dp(_cd(q)), _ptr(np.ascontiguousarray(tag, dtype=np.int32), ctypes.c_int32),
                      _dp(_cd(flink)), int(want_tag), _dp(c), _dp(T))
    return T


def free_rotation(p, base, base_u, body, inertia, f0, steps, lir=0):
    """A rigid body turning freely about the z axis through its centre (the
    Jeffery's-orbit test of Sec. III.C), coupled to the fluid one step at a time:
    step the fluid with the body's links at the current angle (wall velocity
    omega x (x_W - c)), take the torque of that step's link forces (torque), turn
    the body by the semi-implicit Euler update omega += T / I, angle += omega, rebuild
    its links at the new angle, and refill the nodes it uncovered at the body
    velocity (refill, or refill_lir with ``lir`` iterations, App. D). ``body`` is
    a shape dict (SHAPE_ELLIPSOID or SHAPE_SPHERE) with keys c, r, tag and ang.
    Returns (flags, f, history) with history[k] = (angle, omega, torque) after step k+1."""
    c = np.asarray(body["c"], dtype=np.float64)
    ang, om = float(body.get("ang", 0.0)), 0.0

    def links(a, w):
        return geometry(p, base, base_u, [dict(body, ang=a, om=(0.0, 0.0, w), om1=(0.0, 0.0, w))])

    flags, q, uw, uw1, tag = links(ang, om)
    f = _cd(f0).copy()
    X = np.arange(flags.size)
    nx, ny = p.nx, p.ny
    rx = X % nx - c[0]
    ry = (X // nx) % ny - c[1]
    hist = np.zeros((steps, 3))
    for k in range(steps):
        fprev = f
        f, flink = step(p, flags, f, q, uw, uw1, want_force=True)
        T = torque(p, q, tag, flink, c, int(body["tag"]))[2]
        om += T / inertia
        ang += om
        fn, qn, uwn, uw1n, tagn = links(ang, om)
        un = np.zeros((flags.size, 3))
        un[:, 0], un[:, 1] = -om * ry, om * rx      # omega e_z x (x - c)
        if lir:
            refill_lir(p, flags, fn, un, fprev, f, K=lir)
        else:
            refill(p, flags, fn, un, f)
        flags, q, uw, uw1, tag = fn, qn, uwn, uw1n, tagn
        hist[k] = (ang, om, T)
    return flags, f, hist


def bc_weights(bc, q, qcut=0.01):
    """``[(s_j, a_j)]`` the boundary rule interpolates through at this q."""
    s = np.zeros(3)
    a = np.zeros(3)
    npnt = _load().or_bc_weights(bc, q, qcut, _dp(s), _dp(a))
    return list(zip(s[:npnt].tolist(), a[:npnt].tolist()))


class Sim:
    """Small driver holding an oracle state (flags, links, populations)."""

    def __init__(self, p, flags, q=None, uw=None, uw1=None, f=None, shell=None):
        self.p = p
        self.flags = _c8(np.reshape(flags, -1))
        self.q, self.uw, self.uw1 = q, uw, uw1
        self.shell = shell
        self.f = init_eq(p, self.flags) if f is None else _cd(f)
        self.t = 0

    def run(self, n, want_force=False):
        flink = None
        for _ in range(n):
            if want_force:
                self.f, flink = step(self.p, self.flags, self.f, self.q, self.uw, self.uw1, True,
                                     self.shell)
            else:
                self.f = step(self.p, self.flags, self.f, self.q, self.uw, self.uw1, shell=self.shell)
            self.t += 1
        return flink

    def macros(self):
        return macros(self.p, self.flags, self.f)

    def mass(self):
        return mass(self.p, self.flags, self.f)
