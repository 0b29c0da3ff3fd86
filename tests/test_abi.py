"""CPU checks of the C ABI: the library loads, exports what include/lbm.h declares,
its lattice tables are the textbook sets, and host-side argument checks return
error codes. No GPU compute is called here."""
import ctypes
import os
import re
from fractions import Fraction

import numpy as np
import pytest

from paper_2009_04604_gb300 import build, lbm

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


@pytest.fixture(scope="module")
def lib():
    build.build()
    return lbm.load()


def test_exports_every_declared_function(lib):
    names = lbm.header_functions()
    assert len(names) >= 17
    for name in names:
        assert hasattr(lib, name), name
    # and the binding declares a signature for each
    assert set(names) - {"lbm_last_error", "lbm_batch_last_error"} <= set(lbm._SIGS)


def _golden(name):
    rows = {}
    for line in open(os.path.join(GOLDEN, name)):
        if line.startswith("#") or not line.strip():
            continue
        cx, cy, cz, w = line.split()
        rows[(int(cx), int(cy), int(cz))] = Fraction(w)
    return rows


@pytest.mark.parametrize("lat,name", [(lbm.D2Q9, "d2q9.txt"), (lbm.D3Q19, "d3q19.txt"),
                                      (lbm.D3Q27, "d3q27.txt")])
def test_lattice_tables(lib, lat, name):
    c, w = lbm.lattice_info(lat)
    gold = _golden(name)
    assert len(w) == len(gold)
    Q = len(w)
    for i in range(Q):
        assert w[i] == pytest.approx(float(gold[tuple(int(v) for v in c[i])]), abs=1e-16)
        assert (c[Q - 1 - i] == -c[i]).all()  # opposite direction is Q-1-i
    assert len({tuple(v) for v in c}) == Q


def test_host_argument_errors(lib):
    h = ctypes.c_void_p()
    dims = (ctypes.c_int * 3)(8, 8, 1)
    assert lib.lbm_create(lbm.D2Q9, dims, 0.5, lbm.F32, None, ctypes.byref(h)) == -1  # tau <= 1/2
    assert b"tau" in lib.lbm_last_error(None)
    assert lib.lbm_create(7, dims, 0.8, lbm.F32, None, ctypes.byref(h)) == -1
    assert lib.lbm_create(lbm.D2Q9, (ctypes.c_int * 3)(8, 8, 2), 0.8, lbm.F32, None, ctypes.byref(h)) == -1
    assert lib.lbm_create(lbm.D3Q19, (ctypes.c_int * 3)(8, 0, 2), 0.8, lbm.F32, None, ctypes.byref(h)) == -1
    assert lib.lbm_create(lbm.D3Q19, dims, 0.8, 9, None, ctypes.byref(h)) == -1
    assert lib.lbm_create(lbm.D3Q19, dims, 0.8, lbm.F32, None, None) == -1
    assert lib.lbm_step(None, 1) == -1
    assert lib.lbm_lattice_info(5, None, None, None) == -1
    # the default build does not check population indices (LBM_DEBUG)
    assert lib.lbm_is_debug_build() == 0
    assert lib.lbm_set_debug_limit(None, 5) == -1


def test_oracle_and_library_share_no_code():
    """The oracle and the CUDA package import neither each other nor shared helpers."""
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    pkg = os.path.join(root, "paper_2009_04604_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".hpp", ".h")):
                text = open(os.path.join(dirpath, f)).read()
                assert not re.search(r"^\s*(import oracle|from oracle)", text, re.M), f
                assert "lbm_oracle" not in text, f
    for f in os.listdir(os.path.join(root, "oracle")):
        if f.endswith((".py", ".c", ".h")):
            text = open(os.path.join(root, "oracle", f)).read()
            assert not re.search(r"^\s*(import|from) paper_2009_04604_gb300", text, re.M), f
            assert "include/lbm.h" not in text and "liblbm.so" not in text, f


def test_binding_constants_match_the_header():
    """Every enumerator of include/lbm.h has the same value in the Python binding."""
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    text = open(os.path.join(root, "include", "lbm.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    header = {}
    for body in re.findall(r"enum\s+\w+\s*\{(.*?)\}", text, flags=re.S):
        for name, val in re.findall(r"(LBM_\w+)\s*=\s*(-?\d+)", body):
            header[name] = int(val)
    assert len(header) >= 30
    status = {v: k for k, v in lbm.STATUS.items()}
    shapes = {"LBM_SHAPE_" + k.upper(): v for k, v in lbm.SHAPE_TYPES.items()}
    for name, val in header.items():
        if name in status:
            assert status[name] == val, name
        elif name.startswith("LBM_SHAPE_"):
            assert shapes[name] == val, name
        else:
            assert getattr(lbm, name[len("LBM_"):]) == val, name
