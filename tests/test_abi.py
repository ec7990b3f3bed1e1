"""Host-side checks of the C-ABI library (no GPU needed).

The library must load and export every entry point that include/npcf.h
declares, and host-side argument validation must reject bad plans before any
device work.
"""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2106_10278_gb300 import build

    build.build()
    from paper_2106_10278_gb300 import npcf

    return npcf.load_library()


def _declared():
    src = open(os.path.join(ROOT, "include", "npcf.h")).read()
    return re.findall(r"NPCF_API\s+[\w\s\*]+?\b(npcf_\w+)\s*\(", src)


def test_header_declares_the_binding_exports():
    from paper_2106_10278_gb300 import npcf

    assert sorted(_declared()) == sorted(npcf.EXPORTS)


def test_library_exports_every_declared_symbol(lib):
    for name in _declared():
        assert hasattr(lib, name), name


def test_shared_object_exports_only_the_abi(lib):
    import subprocess

    from paper_2106_10278_gb300.npcf import LIB_PATH

    out = subprocess.run(["nm", "-D", "--defined-only", LIB_PATH], capture_output=True, text=True).stdout
    syms = {line.split()[-1] for line in out.splitlines() if " T " in line}
    assert set(_declared()) <= syms
    assert not [s for s in syms if s.startswith("_ZN4npcf")]  # internal C++ symbols stay hidden


def _create(lib, D, N, lmax, edges, box, opts=None):
    from paper_2106_10278_gb300.npcf import Opts

    h = ctypes.c_void_p()
    e = np.ascontiguousarray(edges, dtype=np.float64)
    b = np.ascontiguousarray(box, dtype=np.float64)
    o = Opts()
    lib.npcf_default_opts(ctypes.byref(o))
    if opts:
        for k, v in opts.items():
            setattr(o, k, v)
    st = lib.npcf_plan_create(ctypes.byref(h), D, N, lmax, e.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                              len(e) - 1, b.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), ctypes.byref(o))
    if st == 0:
        lib.npcf_plan_destroy(h)
    return st, lib.npcf_last_error().decode()


@pytest.mark.parametrize(
    "D,N,lmax,edges,box,opts,status",
    [
        (5, 3, 2, [0.1, 0.2], [1] * 5, None, -2),  # dimension
        (3, 6, 2, [0.1, 0.2], [1] * 3, None, -2),  # order
        (2, 5, 2, [0.1, 0.2, 0.3, 0.4, 0.45], [1] * 2, None, -2),  # N=5 is provided for D=3
        (3, 5, 7, [0.1, 0.2, 0.3, 0.4, 0.45], [1] * 3, None, -2),  # N=5 lmax limit
        (3, 5, 2, [0.1, 0.2, 0.3], [1] * 3, None, -1),  # N=5 needs 4 bins
        (4, 4, 2, [0.1, 0.2, 0.3, 0.4], [1] * 4, None, -2),  # N=4 in D=4 needs an SO(4) coupling
        (3, 3, 2, [0.1, 0.2], [1] * 3, {"precision": 2}, -2),  # split precision: tensor-core couplings only
        (2, 4, 2, list(np.linspace(0.01, 0.1, 19)), [1] * 2, {"precision": 3}, -2),  # > 128 bin pairs
        (2, 4, 2, [0.1, 0.2, 0.3, 0.4], [1] * 2, {"precision": 7}, -1),  # unknown precision
        (2, 3, 2, [0.1, 0.2], [1] * 2, {"basis": 1}, -2),  # the line-of-sight basis is D=3 only
        (3, 5, 2, [0.1, 0.2, 0.3, 0.4, 0.45], [1] * 3, {"basis": 1}, -2),  # ... and N <= 4
        (3, 3, 2, [0.1, 0.2], [1] * 3, {"basis": 1, "remove_self": 1}, -2),
        (3, 3, 2, [0.1, 0.2], [1] * 3, {"basis": 9}, -1),  # unknown basis
        (3, 4, 7, [0.1, 0.2, 0.3, 0.4], [1] * 3, None, -2),  # lmax beyond the compiled coupling
        (3, 3, 2, list(np.linspace(0.01, 0.3, 40)), [1] * 3, None, -2),  # more than 32 bins
        (3, 3, 2, [0.2, 0.1], [1] * 3, None, -1),  # decreasing edges
        (3, 3, 2, [-0.1, 0.1], [1] * 3, None, -1),  # negative edge
        (3, 3, 2, [0.1, 0.6], [1] * 3, None, -1),  # r_max >= box/2 with periodic wrap
        (3, 3, 2, [0.1, 0.2], [1, 0, 1], None, -1),  # zero box side
        (3, 4, 2, [0.1, 0.2], [1] * 3, None, -1),  # N=4 needs 3 bins
        (3, 3, 2, [0.1, 0.2], [1] * 3, {"precision": 7}, -1),
    ],
)
def test_plan_argument_validation(lib, D, N, lmax, edges, box, opts, status):
    st, msg = _create(lib, D, N, lmax, edges, box, opts)
    assert st == status, msg
    assert msg


def test_null_arguments(lib):
    assert lib.npcf_plan_create(None, 3, 3, 2, None, 1, None, None) == -1
    assert lib.npcf_num_coeffs(None, None) == -1
    assert lib.npcf_compute(None, None, None, 0, None, 0, 0, None) == -1
    assert lib.npcf_compute_host(None, None, None, 0, None, 0, 0, None) == -1
    assert lib.npcf_compute_noalloc(None, None, None, 0, None, 0, 0, None) == -1
    off = (ctypes.c_int64 * 2)(0, 0)
    box = (ctypes.c_double * 3)(1.0, 1.0, 1.0)
    assert lib.npcf_compute_batched(None, None, None, off, box, 1, None, None) == -1
    assert lib.npcf_backward(None, None, None, 0, None, 0, 0, None, None, None) == -1
    assert lib.npcf_coeff_index(None, 0, None, None) == -1
    assert lib.npcf_device_status(None) == -1
    assert lib.npcf_last_stats(None, None, None, None) == -1
    assert lib.npcf_last_profile(None, None, None) == -1
    assert lib.npcf_last_counters(None, None, 0) == -1
    assert b"NULL" in lib.npcf_last_error()
    lib.npcf_plan_destroy(None)  # a no-op


def test_binding_rejects_unknown_precision():
    from paper_2106_10278_gb300.npcf import Plan

    with pytest.raises(ValueError):
        Plan(3, 3, 2, [0.1, 0.2], 1.0, precision="bf16")
