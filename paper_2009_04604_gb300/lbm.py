"""ctypes binding of liblbm.so (include/lbm.h): argument marshalling only.

Every step of the lattice Boltzmann path runs in the library's CUDA kernels.
The binding converts numpy/torch arguments to plain pointers and turns status
codes into exceptions. PyTorch supplies device buffers and the CUDA stream. If
liblbm.so has not been built, importing the library raises; nothing here
computes a result on the CPU.
"""
from __future__ import annotations

import ctypes
import os
import re

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
# LBM_LIBRARY selects another build of the library, e.g. the bounds-checked one
# (build.build(debug=True) writes _build_debug/liblbm.so)
LIB_PATH = os.environ.get("LBM_LIBRARY") or os.path.join(_HERE, "_build", "liblbm.so")
DEBUG_LIB_PATH = os.path.join(_HERE, "_build_debug", "liblbm.so")
HEADER = os.path.join(os.path.dirname(_HERE), "include", "lbm.h")

D2Q9, D3Q19, D3Q27 = 0, 1, 2
F64, F32, F16, BF16 = 0, 1, 2, 3
BC_ELIBB_F, BC_ELIBB_FQ, BC_BFL, BC_HWBB, BC_ELIBB_U, BC_ELIBB_UQ = 0, 1, 2, 3, 4, 5
COLL_BGK, COLL_TRT = 0, 1
NEQ_BOUNCE_BACK, NEQ_REGULARIZED = 0, 1
FLUID, SOLID, OPEN = 0, 1, 2
REFILL_EQUILIBRIUM, REFILL_LIR = 0, 1
SHAPE_TYPES = {"sphere": 0, "sphere_out": 1, "ellipsoid": 2, "strip": 3, "shell": 4}
DTYPES = {"f64": F64, "f32": F32, "f16": F16, "bf16": BF16}
BCS = {"elibb_f": BC_ELIBB_F, "elibb_fq": BC_ELIBB_FQ, "bfl": BC_BFL, "hwbb": BC_HWBB,
       "elibb_u": BC_ELIBB_U, "elibb_uq": BC_ELIBB_UQ}
COLLISIONS = {"bgk": COLL_BGK, "trt": COLL_TRT}
STATUS = {0: "LBM_OK", -1: "LBM_ERR_ARG", -2: "LBM_ERR_CUDA", -3: "LBM_ERR_OOM",
          -4: "LBM_ERR_NONFINITE", -5: "LBM_ERR_TIMEOUT", -6: "LBM_ERR_STATE", -7: "LBM_ERR_BOUNDS"}


class LBMError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{STATUS.get(code, code)}: {msg}")
        self.code = code


class Shape(ctypes.Structure):
    _fields_ = [("type", ctypes.c_int), ("tag", ctypes.c_int),
                ("c", ctypes.c_double * 3), ("r", ctypes.c_double * 3),
                ("nrm", ctypes.c_double * 3), ("off", ctypes.c_double),
                ("width", ctypes.c_double), ("period", ctypes.c_double),
                ("v", ctypes.c_double * 3), ("om", ctypes.c_double * 3),
                ("v1", ctypes.c_double * 3), ("om1", ctypes.c_double * 3),
                ("ang", ctypes.c_double)]


_lib = None
P = ctypes.POINTER
_d, _u8, _i32, _i64, _int = (P(ctypes.c_double), P(ctypes.c_uint8), P(ctypes.c_int32),
                             P(ctypes.c_int64), P(ctypes.c_int))
_SIGS = {
    "lbm_lattice_info": [ctypes.c_int, _int, _int, _d],
    "lbm_create": [ctypes.c_int, _int, ctypes.c_double, ctypes.c_int, ctypes.c_void_p, P(ctypes.c_void_p)],
    "lbm_destroy": [ctypes.c_void_p],
    "lbm_set_options": [ctypes.c_void_p, ctypes.c_int, ctypes.c_double, _d, ctypes.c_int],
    "lbm_set_collision": [ctypes.c_void_p, ctypes.c_int, ctypes.c_double],
    "lbm_set_wall_neq": [ctypes.c_void_p, ctypes.c_int],
    "lbm_set_geometry": [ctypes.c_void_p, _u8, _d, _d, _d, _i32],
    "lbm_build_geometry": [ctypes.c_void_p, _u8, _d, P(Shape), ctypes.c_int],
    "lbm_init": [ctypes.c_void_p, ctypes.c_double, _d],
    "lbm_set_populations": [ctypes.c_void_p, _d],
    "lbm_get_populations": [ctypes.c_void_p, _d],
    "lbm_step": [ctypes.c_void_p, ctypes.c_int],
    "lbm_macros": [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p],
    "lbm_wall_force": [ctypes.c_void_p, ctypes.c_int, _d],
    "lbm_mass": [ctypes.c_void_p, _d],
    "lbm_get_geometry": [ctypes.c_void_p, _u8, _d, _d, _d, _i32],
    "lbm_get_counts": [ctypes.c_void_p, _i64, _i64, _i64],
    "lbm_synchronize": [ctypes.c_void_p],
    "lbm_set_launch": [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int],
    "lbm_get_launch": [ctypes.c_void_p, _int, _int, _int, _int],
    "lbm_autotune": [ctypes.c_void_p, ctypes.c_int, _int, _int, _int, _int, _d],
    "lbm_mass_noalloc": [ctypes.c_void_p, ctypes.c_void_p],
    "lbm_save": [ctypes.c_void_p, ctypes.c_void_p, P(ctypes.c_size_t)],
    "lbm_load": [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t],
    "lbm_set_wait_limit": [ctypes.c_void_p, ctypes.c_longlong],
    "lbm_set_debug_limit": [ctypes.c_void_p, ctypes.c_longlong],
    "lbm_is_debug_build": [],
    "lbm_set_moving_body": [ctypes.c_void_p, P(Shape), _d, ctypes.c_int, ctypes.c_int],
    "lbm_set_free_body": [ctypes.c_void_p, P(Shape), ctypes.c_double, ctypes.c_int],
    "lbm_get_body_history": [ctypes.c_void_p, _d, _i64],
    "lbm_wall_torque": [ctypes.c_void_p, ctypes.c_int, _d, _d],
    "lbm_set_refill": [ctypes.c_void_p, ctypes.c_int, ctypes.c_int],
    "lbm_batch_create": [P(ctypes.c_void_p), ctypes.c_int, P(ctypes.c_void_p)],
    "lbm_batch_destroy": [ctypes.c_void_p],
    "lbm_batch_step": [ctypes.c_void_p, ctypes.c_int],
    "lbm_batch_set_launch": [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int],
    "lbm_batch_autotune": [ctypes.c_void_p, ctypes.c_int, _int, _int, _int, _int, _d],
}


def header_functions():
    """Names of the functions include/lbm.h declares."""
    text = open(HEADER).read()
    return sorted(set(re.findall(r"^\s*(?:int|const char \*)\s*(lbm_\w+)\s*\(", text, re.M)))


def load():
    """Load liblbm.so; raises if it has not been built (no fallback)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} is missing: build it with paper_2009_04604_gb300.build.build()")
        lib = ctypes.CDLL(LIB_PATH)
        for name, args in _SIGS.items():
            fn = getattr(lib, name)
            fn.argtypes = args
            fn.restype = ctypes.c_int
        lib.lbm_last_error.argtypes = [ctypes.c_void_p]
        lib.lbm_last_error.restype = ctypes.c_char_p
        lib.lbm_batch_last_error.argtypes = [ctypes.c_void_p]
        lib.lbm_batch_last_error.restype = ctypes.c_char_p
        _lib = lib
    return _lib


def is_debug_build():
    """Whether the loaded library checks population indices (LBM_DEBUG)."""
    return bool(load().lbm_is_debug_build())


def _check(rc, h=None):
    if rc != 0:
        raise LBMError(rc, load().lbm_last_error(h).decode())


def _np_ptr(a, ctype):
    return None if a is None else a.ctypes.data_as(P(ctype))


def lattice_info(lattice):
    """``(c[Q,3], w[Q])`` in the library's direction order."""
    lib = load()
    Q = ctypes.c_int()
    c = np.zeros((27, 3), np.int32)
    w = np.zeros(27)
    _check(lib.lbm_lattice_info(lattice, ctypes.byref(Q), _np_ptr(c, ctypes.c_int), _np_ptr(w, ctypes.c_double)))
    return c[:Q.value].copy(), w[:Q.value].copy()


def make_shapes(specs):
    arr = (Shape * max(1, len(specs)))()
    for k, s in enumerate(specs):
        for key, val in s.items():
            if key == "type":
                arr[k].type = SHAPE_TYPES[val] if isinstance(val, str) else int(val)
            elif isinstance(val, (list, tuple, np.ndarray)):
                dst = getattr(arr[k], key)
                for a, x in enumerate(val):
                    dst[a] = float(x)
            else:
                setattr(arr[k], key, val)
    return arr


def _f64(a, shape=None):
    if a is None:
        return None
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a if shape is None else a.reshape(shape)


class Simulation:
    """One lattice Boltzmann simulation on the current CUDA device.

    ``stream``: a ``torch.cuda.Stream`` (default: a new one). Every call of the
    library runs on it, and results handed back as torch tensors are ordered after it.
    """

    def __init__(self, lattice, dims, tau, dtype=F32, stream=None):
        import torch
        self._torch = torch
        self.lib = load()
        self.lattice = lattice
        self.Q = {D2Q9: 9, D3Q19: 19, D3Q27: 27}[lattice]
        dims = list(dims) + [1] * (3 - len(dims))
        self.dims = tuple(int(d) for d in dims)
        self.N = self.dims[0] * self.dims[1] * self.dims[2]
        self.dtype = DTYPES[dtype] if isinstance(dtype, str) else dtype
        self.stream = stream if stream is not None else torch.cuda.Stream()
        h = ctypes.c_void_p()
        d = (ctypes.c_int * 3)(*self.dims)
        _check(self.lib.lbm_create(lattice, d, float(tau), self.dtype,
                                   ctypes.c_void_p(self.stream.cuda_stream), ctypes.byref(h)))
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            self.lib.lbm_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _ok(self, rc):
        _check(rc, self.h)

    def set_options(self, bc=BC_ELIBB_F, rho0=1.0, force=(0.0, 0.0, 0.0), xshift=0):
        bc = BCS[bc] if isinstance(bc, str) else bc
        F = (ctypes.c_double * 3)(*[float(x) for x in force])
        self._ok(self.lib.lbm_set_options(self.h, bc, float(rho0), F, int(xshift)))

    def set_wall_neq(self, mode=NEQ_BOUNCE_BACK):
        """Wall non-equilibrium estimate: bounce-back (Eq. neqbb-s) or regularized (Eq. fi_neq)."""
        self._ok(self.lib.lbm_set_wall_neq(self.h, int(mode)))

    def set_collision(self, model=COLL_BGK, magic=3.0 / 16.0):
        """BGK or TRT (magic parameter Lambda, Eq. magic-parameter)."""
        model = COLLISIONS[model] if isinstance(model, str) else model
        self._ok(self.lib.lbm_set_collision(self.h, int(model), float(magic)))

    def set_geometry(self, flags, q=None, uw=None, uw1=None, tag=None):
        """Host arrays in the library's direction order: flags[N], q[N,Q], uw[N,Q,3], tag[N,Q]."""
        flags = np.ascontiguousarray(np.reshape(flags, -1), dtype=np.uint8)
        q = _f64(q, (-1,))
        uw = _f64(uw, (-1,))
        uw1 = _f64(uw1, (-1,))
        tag = None if tag is None else np.ascontiguousarray(np.reshape(tag, -1), dtype=np.int32)
        self._ok(self.lib.lbm_set_geometry(self.h, _np_ptr(flags, ctypes.c_uint8), _np_ptr(q, ctypes.c_double),
                                           _np_ptr(uw, ctypes.c_double), _np_ptr(uw1, ctypes.c_double),
                                           _np_ptr(tag, ctypes.c_int32)))

    def build_geometry(self, base=None, base_u=None, shapes=()):
        """Link geometry computed on the device from analytic shapes: dict specs with the
        fields of lbm_shape, type one of "sphere", "sphere_out", "ellipsoid", "strip" or
        "shell" (a thin shell with fluid on both sides)."""
        base = None if base is None else np.ascontiguousarray(np.reshape(base, -1), dtype=np.uint8)
        base_u = _f64(base_u, (-1,))
        arr = make_shapes(list(shapes))
        self._ok(self.lib.lbm_build_geometry(self.h, _np_ptr(base, ctypes.c_uint8),
                                             _np_ptr(base_u, ctypes.c_double), arr, len(shapes)))

    def set_moving_body(self, body, traj, t0=0):
        """Rigid body (dict spec: sphere or ellipsoid) on the trajectory traj[k] = (c[3], v[3], om[3])."""
        traj = _f64(traj, (-1, 9))
        arr = make_shapes([body])
        self._ok(self.lib.lbm_set_moving_body(self.h, arr, _np_ptr(traj, ctypes.c_double), traj.shape[0], int(t0)))

    def set_free_body(self, body, inertia, history=0):
        """Rigid body (dict spec: sphere or ellipsoid, with c, r, ang, om) turning freely
        about z through its centre under the fluid torque (lbm_set_free_body)."""
        arr = make_shapes([body])
        self._ok(self.lib.lbm_set_free_body(self.h, arr, float(inertia), int(history)))

    def set_refill(self, mode="equilibrium", iterations=10):
        """Refill of fresh nodes: "equilibrium" or "lir" (local iteration refill)."""
        m = {"equilibrium": REFILL_EQUILIBRIUM, "lir": REFILL_LIR}[mode] if isinstance(mode, str) else int(mode)
        self._ok(self.lib.lbm_set_refill(self.h, m, int(iterations)))

    def body_history(self):
        """[steps, 3] array: angle, angular velocity after each step and the step's torque."""
        n = ctypes.c_int64(0)
        self._ok(self.lib.lbm_get_body_history(self.h, None, ctypes.byref(n)))
        out = np.zeros((max(n.value, 1), 3))
        self._ok(self.lib.lbm_get_body_history(self.h, _np_ptr(out, ctypes.c_double), ctypes.byref(n)))
        return out[:n.value]

    def wall_torque(self, centre, tag=-1):
        c = np.ascontiguousarray(centre, dtype=np.float64)
        T = np.zeros(3)
        self._ok(self.lib.lbm_wall_torque(self.h, int(tag), _np_ptr(c, ctypes.c_double), _np_ptr(T, ctypes.c_double)))
        return T

    def init(self, rho=1.0, u=(0.0, 0.0, 0.0)):
        U = (ctypes.c_double * 3)(*[float(x) for x in u])
        self._ok(self.lib.lbm_init(self.h, float(rho), U))

    def set_populations(self, f):
        f = _f64(f, (-1,))
        assert f.size == self.N * self.Q
        self._ok(self.lib.lbm_set_populations(self.h, _np_ptr(f, ctypes.c_double)))

    def get_populations(self):
        f = np.zeros((self.N, self.Q))
        self._ok(self.lib.lbm_get_populations(self.h, _np_ptr(f, ctypes.c_double)))
        return f

    def step(self, n=1):
        self._ok(self.lib.lbm_step(self.h, int(n)))

    def synchronize(self):
        self._ok(self.lib.lbm_synchronize(self.h))

    def macros(self, rho=None, u=None):
        """Density [N] and velocity [N,3] as FP64 torch tensors on the device."""
        torch = self._torch
        dev = torch.device("cuda", torch.cuda.current_device())
        with torch.cuda.stream(self.stream):
            if rho is None:
                rho = torch.empty(self.N, dtype=torch.float64, device=dev)
            if u is None:
                u = torch.empty((self.N, 3), dtype=torch.float64, device=dev)
        self._ok(self.lib.lbm_macros(self.h, ctypes.c_void_p(rho.data_ptr()), ctypes.c_void_p(u.data_ptr())))
        torch.cuda.current_stream().wait_stream(self.stream)
        return rho, u

    def wall_force(self, tag=-1):
        F = np.zeros(3)
        self._ok(self.lib.lbm_wall_force(self.h, int(tag), _np_ptr(F, ctypes.c_double)))
        return F

    def mass(self):
        m = ctypes.c_double()
        self._ok(self.lib.lbm_mass(self.h, ctypes.byref(m)))
        return m.value

    def get_geometry(self):
        N, Q = self.N, self.Q
        flags = np.zeros(N, np.uint8)
        q = np.zeros((N, Q))
        uw = np.zeros((N, Q, 3))
        uw1 = np.zeros((N, Q, 3))
        tag = np.zeros((N, Q), np.int32)
        self._ok(self.lib.lbm_get_geometry(self.h, _np_ptr(flags, ctypes.c_uint8), _np_ptr(q, ctypes.c_double),
                                           _np_ptr(uw, ctypes.c_double), _np_ptr(uw1, ctypes.c_double),
                                           _np_ptr(tag, ctypes.c_int32)))
        return flags, q, uw, uw1, tag

    def counts(self):
        a, b, c = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
        self._ok(self.lib.lbm_get_counts(self.h, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)))
        return a.value, b.value, c.value

    def save(self):
        """The current state as bytes (lbm_save): header plus the raw stored populations."""
        n = ctypes.c_size_t(0)
        self._ok(self.lib.lbm_save(self.h, None, ctypes.byref(n)))
        buf = ctypes.create_string_buffer(n.value)
        self._ok(self.lib.lbm_save(self.h, ctypes.cast(buf, ctypes.c_void_p), ctypes.byref(n)))
        return buf.raw[:n.value]

    def load(self, blob):
        """Restore a state written by save() into this handle (same geometry and options)."""
        buf = ctypes.create_string_buffer(bytes(blob), len(blob))
        self._ok(self.lib.lbm_load(self.h, ctypes.cast(buf, ctypes.c_void_p), len(blob)))

    def set_wait_limit(self, polls):
        """Testing aid: poll limit of the TMA-staged step's first waits (negative: default)."""
        self._ok(self.lib.lbm_set_wait_limit(self.h, int(polls)))

    def set_debug_limit(self, elements):
        """Bounds-checked builds: population indices at or above `elements` count as
        out of range (negative: the buffer's size); see lbm_set_debug_limit."""
        self._ok(self.lib.lbm_set_debug_limit(self.h, int(elements)))

    def set_launch(self, bx, by, variant=0, tiles=4):
        self._ok(self.lib.lbm_set_launch(self.h, int(bx), int(by), int(variant), int(tiles)))

    def get_launch(self):
        a, b, c, d = ctypes.c_int(), ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        self._ok(self.lib.lbm_get_launch(self.h, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c),
                                         ctypes.byref(d)))
        return a.value, b.value, c.value, d.value

    def autotune(self, steps=20):
        """Pick the fastest step-kernel launch configuration (advances the simulation)."""
        a, b, c, d = ctypes.c_int(), ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        ms = ctypes.c_double()
        self._ok(self.lib.lbm_autotune(self.h, int(steps), ctypes.byref(a), ctypes.byref(b), ctypes.byref(c),
                                       ctypes.byref(d), ctypes.byref(ms)))
        return dict(bx=a.value, by=b.value, variant=c.value, tiles=d.value, ms_per_step=ms.value)

    def mass_noalloc(self, out):
        """Total mass into the caller's FP64 device tensor ``out[0]``, without any device
        allocation (static scratch; see lbm_mass_noalloc in include/lbm.h)."""
        self._ok(self.lib.lbm_mass_noalloc(self.h, ctypes.c_void_p(out.data_ptr())))
        self._torch.cuda.current_stream().wait_stream(self.stream)
        return out


class Batch:
    """Many simulations (same lattice, dtype and stream) advanced by one launch per step."""

    def __init__(self, sims):
        self.lib = load()
        self.sims = list(sims)
        arr = (ctypes.c_void_p * len(self.sims))(*[s.h.value for s in self.sims])
        b = ctypes.c_void_p()
        rc = self.lib.lbm_batch_create(arr, len(self.sims), ctypes.byref(b))
        if rc != 0:
            raise LBMError(rc, "lbm_batch_create rejected the simulations (lattice, dtype, stream or state)")
        self.b = b

    def _ok(self, rc):
        if rc != 0:
            raise LBMError(rc, self.lib.lbm_batch_last_error(self.b).decode())

    def step(self, n=1):
        self._ok(self.lib.lbm_batch_step(self.b, int(n)))

    def set_launch(self, bx, by, variant=0, tiles=1):
        self._ok(self.lib.lbm_batch_set_launch(self.b, int(bx), int(by), int(variant), int(tiles)))

    def autotune(self, steps=10):
        a, b_, c, d = ctypes.c_int(), ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        ms = ctypes.c_double()
        self._ok(self.lib.lbm_batch_autotune(self.b, int(steps), ctypes.byref(a), ctypes.byref(b_), ctypes.byref(c),
                                             ctypes.byref(d), ctypes.byref(ms)))
        return dict(bx=a.value, by=b_.value, variant=c.value, tiles=d.value, ms_per_step=ms.value)

    def close(self):
        if getattr(self, "b", None):
            self.lib.lbm_batch_destroy(self.b)
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
