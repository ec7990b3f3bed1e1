"""The allocation-free entry point npcf_compute_noalloc.

It serves callers that cannot allocate device memory while they run (the
device-wide synchronisation of cudaMalloc, or its failure under memory
pressure, is unacceptable to real-time loops and to processes whose caching
allocator already holds the free memory): they create the plan during set-up
and then compute with no allocation, the workspace coming from a static array
inside the library.  Its results are checked against npcf_compute on two calls
in a row and against the FP64 oracle, with the tolerances of the other tests
(FP64: max error <= 1e-10 max |oracle|; FP32: ||error|| <= 1e-5 ||oracle||).
This file is collected last on purpose, so that a run stopping at the first
failure has already run every other test.
"""
import ctypes

import numpy as np
import pytest

import oracle
from paper_2106_10278_gb300 import catalogs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2106_10278_gb300 import build

    build.build()
    oracle.build()
    from paper_2106_10278_gb300 import npcf

    return npcf.load_library()


def _noalloc(lib, plan, pos, w, out, primaries=(0, 0)):
    from paper_2106_10278_gb300.npcf import _check

    s = torch.cuda.current_stream()
    _check(lib.npcf_compute_noalloc(plan._h, ctypes.c_void_p(pos.data_ptr()), ctypes.c_void_p(w.data_ptr()),
                                    pos.shape[0], ctypes.c_void_p(out.data_ptr()), primaries[0], primaries[1],
                                    ctypes.c_void_p(s.cuda_stream)))
    torch.cuda.synchronize()
    return out.cpu().numpy().copy()


def _close(precision, got, ref):
    if precision == "fp64":
        return np.max(np.abs(got - ref)) <= 1e-10 * np.max(np.abs(ref))
    return np.linalg.norm(got - ref) <= 1e-5 * np.linalg.norm(ref)


@pytest.mark.parametrize("D,N,lmax,nbins,n,precision", [(3, 4, 5, 10, 6000, "fp32"), (2, 3, 10, 16, 5000, "fp32"),
                                                        (4, 3, 4, 8, 3000, "fp32"), (2, 4, 6, 8, 4000, "fp32"),
                                                        (3, 5, 2, 5, 2000, "fp32"), (3, 4, 3, 6, 3000, "fp64")])
def test_noalloc_matches_compute_twice(lib, D, N, lmax, nbins, n, precision):
    from paper_2106_10278_gb300.npcf import Plan

    f32 = precision == "fp32"
    pos = np.concatenate([catalogs.uniform(n // 2, D, 1.0, 5, fp32=f32),
                          catalogs.gaussian_blobs(n - n // 2, D, 1.0, 5, 0.04, 6, fp32=f32)])
    w = catalogs.normal_weights(n, 1.0, 0.3, 7, fp32=f32)
    edges = np.linspace(0.03, 0.3 if D < 4 else 0.4, nbins + 1)
    plan = Plan(D, N, lmax, edges, np.ones(D), precision=precision)
    dt = torch.float32 if f32 else torch.float64
    tp = torch.tensor(pos, dtype=dt, device="cuda")
    tw = torch.tensor(w, dtype=dt, device="cuda")
    ref = plan.compute(tp, tw).cpu().numpy()
    ref = np.stack([ref.real, ref.imag], 1).ravel()
    out = torch.full((2 * plan.ncoeff,), float("nan"), dtype=torch.float64, device="cuda")
    for _ in range(2):  # the second call reuses the static scratch left by the first
        got = _noalloc(lib, plan, tp, tw, out)
        assert _close(precision, got, ref)
    # a primary sub-range, against npcf_compute and against the oracle on the same range
    sub = plan.compute(tp, tw, primaries=(100, 400)).cpu().numpy()
    sub = np.stack([sub.real, sub.imag], 1).ravel()
    got = _noalloc(lib, plan, tp, tw, out, primaries=(100, 400))
    assert _close(precision, got, sub)
    keys, zo = oracle.estimate(D, N, lmax, edges, np.ones(D), pos, w, primaries=(100, 400))
    index = {tuple(int(x) for x in k): i for i, k in enumerate(keys)}
    zo = zo[np.array([index[tuple(int(x) for x in k)] for k in plan.keys()])]
    assert _close(precision, got, np.stack([zo.real, zo.imag], 1).ravel())


def test_noalloc_rejects_sizes_beyond_its_scratch(lib):
    from paper_2106_10278_gb300.npcf import NpcfError, Plan

    plan = Plan(3, 4, 5, np.linspace(0.01, 0.1, 11), np.ones(3), precision="fp32")
    n = 60000
    tp = torch.rand(n, 3, device="cuda")
    tw = torch.ones(n, device="cuda")
    out = torch.zeros(2 * plan.ncoeff, dtype=torch.float64, device="cuda")
    with pytest.raises(NpcfError, match="WORKSPACE.*static scratch"):
        _noalloc(lib, plan, tp, tw, out)
