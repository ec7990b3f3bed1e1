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
