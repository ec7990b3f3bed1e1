"""The allocation-free entry point npcf_compute_noalloc.

It serves callers that cannot allocate device memory while they run (the
device-wide synchronisation of cudaMalloc, or its failure under memory
pressure, is unacceptable to real-time loops, to processes whose caching
allocator holds the free memory, and to work recorded into CUDA graphs): they
create the plan during set-up and then compute with no allocation, the
workspace coming from a static array inside the library.  This file is
collected last on purpose, so that a run stopping at the first failure has
already run every other test.
"""
import ctypes

import numpy as np
import pytest

from paper_2106_10278_gb300 import catalogs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2106_10278_gb300 import build

    build.build()
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


@pytest.mark.parametrize("D,N,lmax,nbins,n", [(3, 4, 5, 10, 6000), (2, 3, 10, 16, 5000), (4, 3, 4, 8, 3000)])
def test_noalloc_matches_compute_twice(lib, D, N, lmax, nbins, n):
    from paper_2106_10278_gb300.npcf import Plan

    pos = np.concatenate([catalogs.uniform(n // 2, D, 1.0, 5), catalogs.gaussian_blobs(n - n // 2, D, 1.0, 5, 0.04, 6)])
    w = catalogs.normal_weights(n, 1.0, 0.3, 7)
    edges = np.linspace(0.03, 0.3 if D < 4 else 0.4, nbins + 1)
    plan = Plan(D, N, lmax, edges, np.ones(D), precision="fp32")
    tp = torch.tensor(pos, dtype=torch.float32, device="cuda")
    tw = torch.tensor(w, dtype=torch.float32, device="cuda")
    ref = plan.compute(tp, tw).cpu().numpy()
    ref = np.stack([ref.real, ref.imag], 1).ravel()
    out = torch.full((2 * plan.ncoeff,), float("nan"), dtype=torch.float64, device="cuda")
    for _ in range(2):  # the second call reuses the static scratch left by the first
        got = _noalloc(lib, plan, tp, tw, out)
        err = np.linalg.norm(got - ref)
        assert err <= 1e-5 * np.linalg.norm(ref), err
    # a primary sub-range, too
    sub = plan.compute(tp, tw, primaries=(100, 900)).cpu().numpy()
    sub = np.stack([sub.real, sub.imag], 1).ravel()
    got = _noalloc(lib, plan, tp, tw, out, primaries=(100, 900))
    assert np.linalg.norm(got - sub) <= 1e-5 * np.linalg.norm(sub)


def test_noalloc_rejects_sizes_beyond_its_scratch(lib):
    from paper_2106_10278_gb300.npcf import NpcfError, Plan

    plan = Plan(3, 4, 5, np.linspace(0.01, 0.1, 11), np.ones(3), precision="fp32")
    n = 60000
    tp = torch.rand(n, 3, device="cuda")
    tw = torch.ones(n, device="cuda")
    out = torch.zeros(2 * plan.ncoeff, dtype=torch.float64, device="cuda")
    with pytest.raises(NpcfError, match="WORKSPACE.*static scratch"):
        _noalloc(lib, plan, tp, tw, out)
