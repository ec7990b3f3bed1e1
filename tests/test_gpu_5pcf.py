"""The D=3 isotropic 5PCF (N=5) on the GPU against the FP64 oracle, through the C ABI.

Tolerances as for the other orders: FP64 max |gpu - oracle| <= 1e-10 max |oracle|;
FP32 ||gpu - oracle||_2 <= 1e-5 ||oracle||_2.
"""
import numpy as np
import pytest

import oracle
from paper_2106_10278_gb300 import catalogs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL64 = 1e-10
TOL32 = 1e-5


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2106_10278_gb300 import build

    build.build()
    oracle.build()


def _plan(lmax, edges, box, precision):
    from paper_2106_10278_gb300.npcf import Plan

    return Plan(3, 5, lmax, edges, box, precision=precision)


def _compare(lmax, edges, box, pos, w, precision, primaries=None):
    plan = _plan(lmax, edges, box, precision)
    dt = torch.float64 if precision == "fp64" else torch.float32
    got = plan.compute(torch.tensor(pos, dtype=dt, device="cuda"), torch.tensor(w, dtype=dt, device="cuda"),
                       primaries=primaries).cpu().numpy()
    keys, ref = oracle.estimate(3, 5, lmax, edges, box, pos, w, primaries=primaries)
    index = {tuple(int(x) for x in k): i for i, k in enumerate(keys)}
    pk = plan.keys()
    assert pk.shape == keys.shape
    ref = ref[np.array([index[tuple(int(x) for x in k)] for k in pk])]
    if precision == "fp64":
        err, scale = np.max(np.abs(got - ref)), np.max(np.abs(ref))
        assert err <= TOL64 * scale, f"max err {err:.3e} vs scale {scale:.3e}"
    else:
        err, scale = np.linalg.norm(got - ref), np.linalg.norm(ref)
        assert err <= TOL32 * scale, f"rel err {err / scale:.3e}"
    assert scale > 0
    return plan


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("lmax,nbins", [(2, 5), (3, 6)])
def test_5pcf_small_parity(lmax, nbins, precision):
    f32 = precision == "fp32"
    pos = np.concatenate([catalogs.uniform(500, 3, 1.0, 51, fp32=f32),
                          catalogs.gaussian_blobs(500, 3, 1.0, 6, 0.05, 52, fp32=f32)])
    w = catalogs.normal_weights(1000, 1.0, 0.3, 53, fp32=f32)
    edges = np.linspace(0.05, 0.35, nbins + 1)
    _compare(lmax, edges, np.ones(3), pos, w, precision, primaries=(100, 260))


def test_5pcf_paper_example_counts_and_sampled_parity():
    """The paper's 5PCF example: uniform points in the periodic unit cube, ten radial bins in
    [0.1, 0.4], lmax = 4 -> 210 radial x 585 angular components; FP32 against the oracle on a block
    of primaries of a 3000-point catalogue."""
    wl = catalogs.workload("d3n5", scale=0.3)
    plan = _compare(wl.lmax, wl.edges, wl.box, wl.pos, wl.w, "fp32", primaries=(0, 24))
    k = plan.keys()
    assert len({tuple(x) for x in k[:, :4]}) == 210
    assert len({tuple(x) for x in k[:, 4:]}) == 585


def test_5pcf_batched_matches_oracle():
    from paper_2106_10278_gb300.npcf import Plan

    cats = [catalogs.uniform(n, 3, 1.0, 60 + i) for i, n in enumerate((400, 700))]
    boxes = np.array([[1.0, 1.0, 1.0], [1.1, 0.9, 1.0]])
    cats[1] = catalogs.uniform(700, 3, boxes[1], 61)
    pos = np.concatenate(cats)
    w = np.ones(len(pos))
    offsets = np.array([0, 400, 1100], dtype=np.int64)
    edges = np.linspace(0.05, 0.35, 6)
    plan = Plan(3, 5, 2, edges, np.ones(3), precision="fp64")
    got = plan.compute_batched(torch.tensor(pos, device="cuda"), torch.tensor(w, device="cuda"), offsets,
                               boxes).cpu().numpy()
    for i in range(2):
        a, b = offsets[i], offsets[i + 1]
        keys, ref = oracle.estimate(3, 5, 2, edges, boxes[i], pos[a:b], w[a:b])
        index = {tuple(int(x) for x in k): j for j, k in enumerate(keys)}
        ref = ref[np.array([index[tuple(int(x) for x in k)] for k in plan.keys()])]
        assert np.max(np.abs(got[i] - ref)) <= TOL64 * np.max(np.abs(ref))


# ------------------------------------------------- split-precision tensor-core contraction
MIX = "mixed_bf16x3"


@pytest.mark.parametrize("lmax,nbins,n,prims", [(2, 5, 1000, (100, 260)), (3, 6, 1000, None), (4, 10, 1500, (0, 130)),
                                                (1, 4, 300, (5, 9))])
def test_5pcf_mixed_small_parity(lmax, nbins, n, prims):
    """The BF16x3 contraction (X and Z written as hi + lo BF16 planes, three MMAs per product, FP32
    accumulation in tensor memory) against the FP64 oracle at 1e-5 of the coefficient norm: several
    chunks of 64 primaries with a partly filled last one, one chunk, and a catalogue of 4 bins (one
    bin quadruple)."""
    pos = np.concatenate([catalogs.uniform(n // 2, 3, 1.0, 71, fp32=True),
                          catalogs.gaussian_blobs(n - n // 2, 3, 1.0, 6, 0.05, 72, fp32=True)])
    w = catalogs.normal_weights(n, 1.0, 0.3, 73, fp32=True)
    edges = np.linspace(0.05, 0.35, nbins + 1)
    _compare(lmax, edges, np.ones(3), pos, w, MIX, primaries=prims)


def test_5pcf_mixed_full_size_sampled():
    """The paper's 5PCF example at full size (10^4 points, 10 bins, lmax 4), primaries [0, 40)."""
    wl = catalogs.workload("d3n5")
    _compare(wl.lmax, wl.edges, wl.box, wl.pos, wl.w, MIX, primaries=(0, 40))


def test_5pcf_mixed_full_launch_matches_fp64():
    """Every primary of the full-size example (the benchmark's launch): the BF16x3 tensor-core
    contraction agrees with the FP64 GPU path (itself pinned to the oracle at 1e-10) to 1e-5 of the
    coefficient norm, and so does the FP32 CUDA-core path; repeated calls are bitwise equal."""
    wl = catalogs.workload("d3n5")
    ref = _plan(wl.lmax, wl.edges, wl.box, "fp64").compute(torch.tensor(wl.pos, device="cuda"),
                                                           torch.tensor(wl.w, device="cuda")).cpu().numpy()
    pos = torch.tensor(wl.pos, dtype=torch.float32, device="cuda")
    w = torch.tensor(wl.w, dtype=torch.float32, device="cuda")
    for prec in ("fp32", MIX):
        plan = _plan(wl.lmax, wl.edges, wl.box, prec)
        z = plan.compute(pos, w).cpu().numpy()
        assert np.linalg.norm(z - ref) <= TOL32 * np.linalg.norm(ref), prec
        assert np.array_equal(z, plan.compute(pos, w).cpu().numpy()), prec


def test_5pcf_mixed_batched_matches_oracle():
    from paper_2106_10278_gb300.npcf import Plan

    sizes = (400, 0, 700)
    boxes = np.array([[1.0, 1.0, 1.0], [1.0, 1.0, 1.0], [1.1, 0.9, 1.0]])
    pos = np.concatenate([catalogs.uniform(n, 3, boxes[i], 80 + i, fp32=True) for i, n in enumerate(sizes)])
    w = catalogs.normal_weights(len(pos), 1.0, 0.2, 85, fp32=True)
    offsets = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    edges = np.linspace(0.05, 0.35, 6)
    plan = Plan(3, 5, 2, edges, np.ones(3), precision=MIX)
    got = plan.compute_batched(torch.tensor(pos, dtype=torch.float32, device="cuda"),
                               torch.tensor(w, dtype=torch.float32, device="cuda"), offsets, boxes).cpu().numpy()
    for i in range(len(sizes)):
        a, b = offsets[i], offsets[i + 1]
        if a == b:
            assert np.all(got[i] == 0)
            continue
        keys, ref = oracle.estimate(3, 5, 2, edges, boxes[i], pos[a:b], w[a:b])
        index = {tuple(int(x) for x in k): j for j, k in enumerate(keys)}
        ref = ref[np.array([index[tuple(int(x) for x in k)] for k in plan.keys()])]
        assert np.linalg.norm(got[i] - ref) <= TOL32 * np.linalg.norm(ref)


def test_5pcf_tf32_split_rejected():
    from paper_2106_10278_gb300.npcf import NpcfError

    with pytest.raises(NpcfError, match="UNSUPPORTED"):
        _plan(2, np.linspace(0.05, 0.35, 6), np.ones(3), "mixed_tf32x3")
