"""npcf_autotune: launch shapes chosen by timing candidates on a sample of the input.

The chosen shapes must be valid (within the searched ranges), must not change the results beyond
FP32 rounding of the per-span sums (the FP64 plan: beyond 1e-10 of the oracle), and must be
cached by (device, D, N, lmax, bins, precision, size class) in the NPCF_TUNE_CACHE file, from
which a second plan loads them without timing.
"""
import os

import numpy as np
import pytest

import oracle
from paper_2106_10278_gb300 import catalogs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2106_10278_gb300 import build

    build.build()
    oracle.build()


def _plan(D, N, lmax, edges, precision, **kw):
    from paper_2106_10278_gb300.npcf import Plan

    return Plan(D, N, lmax, edges, np.ones(D), precision=precision, **kw)


def _aligned(plan, keys, ref):
    index = {tuple(int(x) for x in k): i for i, k in enumerate(keys)}
    return ref[np.array([index[tuple(int(x) for x in k)] for k in plan.keys()])]


@pytest.mark.parametrize("D,N,lmax,nbins,precision", [(3, 4, 5, 10, "fp32"), (2, 4, 6, 8, "mixed_bf16x3"),
                                                      (3, 5, 2, 5, "fp32"), (3, 3, 4, 8, "fp64")])
def test_autotune_keeps_results(D, N, lmax, nbins, precision, tmp_path, monkeypatch):
    monkeypatch.setenv("NPCF_TUNE_CACHE", str(tmp_path / "tune.txt"))
    f32 = precision != "fp64"
    n = 30000 if N < 5 else 6000
    pos = np.concatenate([catalogs.uniform(n // 2, D, 1.0, 3, fp32=f32),
                          catalogs.gaussian_blobs(n - n // 2, D, 1.0, 20, 0.03, 4, fp32=f32)])
    w = catalogs.normal_weights(n, 1.0, 0.3, 5, fp32=f32)
    edges = np.linspace(0.01, 0.12 if N < 5 else 0.2, nbins + 1)
    dt = torch.float64 if precision == "fp64" else torch.float32
    tp = torch.tensor(pos, dtype=dt, device="cuda")
    tw = torch.tensor(w, dtype=dt, device="cuda")
    plan = _plan(D, N, lmax, edges, precision)
    before = plan.compute(tp, tw, primaries=(0, 500)).cpu().numpy()
    cfg = plan.autotune(tp, tw)
    assert cfg["tuned"] == 1 and 1 <= cfg["pair_warps"] <= 16 and cfg["pair_batch"] % 32 == 0
    after = plan.compute(tp, tw, primaries=(0, 500)).cpu().numpy()
    keys, ref = oracle.estimate(D, N, lmax, edges, np.ones(D), pos, w, primaries=(0, 500))
    ref = _aligned(plan, keys, ref)
    if precision == "fp64":
        assert np.max(np.abs(after - ref)) <= 1e-10 * np.max(np.abs(ref))
    else:
        assert np.linalg.norm(after - ref) <= 1e-5 * np.linalg.norm(ref)
        assert np.linalg.norm(after - before) <= 1e-5 * np.linalg.norm(before)
    # a second plan of the same configuration loads the cached shapes
    lines = open(tmp_path / "tune.txt").read().splitlines()
    assert len(lines) == 1
    plan2 = _plan(D, N, lmax, edges, precision)
    cfg2 = plan2.autotune(tp, tw)
    assert cfg2 == cfg
    assert len(open(tmp_path / "tune.txt").read().splitlines()) == 1


def test_autotune_rejects_bad_arguments():
    from paper_2106_10278_gb300.npcf import NpcfError

    plan = _plan(3, 3, 2, np.linspace(0.1, 0.3, 3), "fp32")
    with pytest.raises(NpcfError, match="ERR_ARG"):
        plan.autotune(torch.zeros((0, 3), device="cuda"), torch.zeros(0, device="cuda"))
    assert plan.tuned_config()["tuned"] == 0
