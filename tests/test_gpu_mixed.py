"""The split-precision tensor-core coupling (NPCF_MIXED_BF16X3, NPCF_MIXED_TF32X3), through the C ABI.

The mixed plans keep the FP32 pair stage and run the D=2 4PCF coupling (eq. NPCF-estimator-discrete
with l1 + l2 + l3 = 0) as a contraction over primaries on the tensor cores, each operand split
into hi + lo.  Tolerance: ||gpu - oracle||_2 <= 1e-5 ||oracle||_2, the mixed-precision bound of this
implementation's target, for both splits.  The contraction itself is checked on plain matrices
first (npcf_selftest_tc), against an FP64 product of the same FP32 inputs.
"""
import numpy as np
import pytest

import oracle
from paper_2106_10278_gb300 import catalogs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-5
MIXED = ["mixed_bf16x3", "mixed_tf32x3"]


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2106_10278_gb300 import build

    build.build()
    oracle.build()


def _plan(D, N, lmax, edges, box, precision, **kw):
    from paper_2106_10278_gb300.npcf import Plan

    return Plan(D, N, lmax, edges, box, precision=precision, **kw)


def _aligned(plan, keys, ref):
    index = {tuple(int(x) for x in k): i for i, k in enumerate(keys)}
    return ref[np.array([index[tuple(int(x) for x in k)] for k in plan.keys()])]


def _rel(got, ref):
    scale = np.linalg.norm(ref)
    assert scale > 0
    return np.linalg.norm(got - ref) / scale


# ------------------------------------------------------------- the contraction alone
@pytest.mark.parametrize("tf32", [False, True])
@pytest.mark.parametrize("n,k", [(16, 64), (32, 128), (128, 256), (256, 512)])
def test_selftest_contraction(tf32, n, k):
    """a b^T of seeded N(0, 1) matrices against the FP64 product: the split keeps ~16 (BF16) or
    ~21 (TF32) bits per product, far better than one BF16 pass; any slip in the operand layout,
    the descriptors or the accumulator read-back gives O(1) errors."""
    from paper_2106_10278_gb300.npcf import selftest_tc

    g = torch.Generator().manual_seed(7 * n + k + int(tf32))
    a = torch.randn(128, k, generator=g)
    b = torch.randn(n, k, generator=g)
    d = selftest_tc(a.cuda(), b.cuda(), tf32=tf32).cpu().double()
    ref = a.double() @ b.double().T
    err = float(torch.linalg.norm(d - ref) / torch.linalg.norm(ref))
    one_pass = (a.bfloat16().double() @ b.bfloat16().double().T)
    err1 = float(torch.linalg.norm(one_pass - ref) / torch.linalg.norm(ref))
    assert err <= (1e-5 if tf32 else 3e-5), err
    assert err <= 0.05 * err1, (err, err1)
    # structure: a one-hot row of a picks out the matching column of b
    a1 = torch.zeros(128, k)
    a1[torch.arange(128), torch.arange(128) % k] = 1.0
    d1 = selftest_tc(a1.cuda(), b.cuda(), tf32=tf32).cpu()
    torch.testing.assert_close(d1, b[:, torch.arange(128) % k].T.contiguous(), rtol=1e-5, atol=1e-6)


def test_selftest_rejects_bad_shapes():
    from paper_2106_10278_gb300.npcf import NpcfError, selftest_tc

    a = torch.randn(128, 64, device="cuda")
    with pytest.raises(NpcfError, match="ERR_ARG"):
        selftest_tc(a, torch.randn(24, 64, device="cuda"))  # n not a multiple of 16
    with pytest.raises(NpcfError, match="ERR_ARG"):
        selftest_tc(torch.randn(128, 48, device="cuda"), torch.randn(16, 48, device="cuda"))  # k


# ----------------------------------------------------------------- the D=2 4PCF
@pytest.mark.parametrize("precision", MIXED)
@pytest.mark.parametrize("lmax,nbins,n,prims", [(6, 8, 2500, (0, 700)), (3, 3, 1500, None), (10, 16, 3000, (0, 400)),
                                                (5, 17, 2000, (100, 333))])
def test_mixed_d2n4_small_parity(precision, lmax, nbins, n, prims):
    g = np.random.default_rng(lmax + nbins)
    pos = np.concatenate([catalogs.uniform(n // 2, 2, 1.0, 9), catalogs.gaussian_blobs(n - n // 2, 2, 1.0, 7, 0.03, 10)])
    w = catalogs.normal_weights(n, 1.0, 0.3, 11) * np.where(g.random(n) < 0.3, -1.0, 1.0)
    edges = np.linspace(0.02, 0.3, nbins + 1)
    plan = _plan(2, 4, lmax, edges, np.ones(2), precision)
    z = plan.compute(torch.tensor(pos, dtype=torch.float32, device="cuda"),
                     torch.tensor(w, dtype=torch.float32, device="cuda"), primaries=prims).cpu().numpy()
    keys, ref = oracle.estimate(2, 4, lmax, edges, np.ones(2), pos, w, primaries=prims)
    assert _rel(z, _aligned(plan, keys, ref)) <= TOL


@pytest.mark.parametrize("precision", MIXED)
def test_mixed_d2n4_full_size_sampled(precision):
    """The D=2 4PCF workload at full size (200k points, 16 bins, lmax 10) on sampled primaries."""
    wl = catalogs.workload("d2n4")
    plan = _plan(wl.D, wl.N, wl.lmax, wl.edges, wl.box, precision)
    pos = torch.tensor(wl.pos, dtype=torch.float32, device="cuda")
    w = torch.tensor(wl.w, dtype=torch.float32, device="cuda")
    z = plan.compute(pos, w, primaries=(0, 400)).cpu().numpy()
    keys, ref = oracle.estimate(wl.D, wl.N, wl.lmax, wl.edges, wl.box, wl.pos, wl.w, primaries=(0, 400))
    assert _rel(z, _aligned(plan, keys, ref)) <= TOL


def test_mixed_full_launch_matches_fp32():
    """Every primary of the full-size workload (the benchmark's launch): both splits agree with the
    FP32 CUDA-core coupling to 1e-5 of the coefficient norm, and with each other."""
    wl = catalogs.workload("d2n4")
    pos = torch.tensor(wl.pos, dtype=torch.float32, device="cuda")
    w = torch.tensor(wl.w, dtype=torch.float32, device="cuda")
    z32 = _plan(wl.D, wl.N, wl.lmax, wl.edges, wl.box, "fp32").compute(pos, w).cpu().numpy()
    for prec in MIXED:
        zm = _plan(wl.D, wl.N, wl.lmax, wl.edges, wl.box, prec).compute(pos, w).cpu().numpy()
        assert _rel(zm, z32) <= TOL, prec


@pytest.mark.parametrize("precision", MIXED)
def test_mixed_batched_and_repeat(precision):
    sizes = [900, 0, 1300, 400]
    boxes = np.array([[1.0, 1.0], [0.9, 1.1], [1.2, 0.8], [1.0, 0.9]])
    parts, ws = [], []
    for i, n in enumerate(sizes):
        parts.append(catalogs.uniform(n, 2, boxes[i], 70 + i))
        ws.append(catalogs.normal_weights(n, 1.0, 0.3, 80 + i))
    pos, w = np.concatenate(parts), np.concatenate(ws)
    offsets = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    edges = np.linspace(0.02, 0.2, 7)
    plan = _plan(2, 4, 4, edges, np.ones(2), precision)
    tp = torch.tensor(pos, dtype=torch.float32, device="cuda")
    tw = torch.tensor(w, dtype=torch.float32, device="cuda")
    got = plan.compute_batched(tp, tw, offsets, boxes).cpu().numpy()
    again = plan.compute_batched(tp, tw, offsets, boxes).cpu().numpy()
    assert np.array_equal(got, again)  # fixed order: bitwise repeatable
    for i in range(len(sizes)):
        a, b = offsets[i], offsets[i + 1]
        if a == b:
            assert np.all(got[i] == 0)
            continue
        keys, ref = oracle.estimate(2, 4, 4, edges, boxes[i], pos[a:b], w[a:b])
        assert _rel(got[i], _aligned(plan, keys, ref)) <= TOL


def test_mixed_unsupported_plans_rejected():
    from paper_2106_10278_gb300.npcf import NpcfError

    with pytest.raises(NpcfError, match="UNSUPPORTED"):
        _plan(2, 4, 4, np.linspace(0.01, 0.1, 19), np.ones(2), "mixed_bf16x3")  # 18 bins: > 128 bin pairs
