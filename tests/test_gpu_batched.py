"""npcf_compute_batched: several catalogues in one pass, each against the FP64 oracle
(or, at full size, against the single-catalogue call on the same data).

Tolerances as for the single-catalogue path: FP64 max |gpu - oracle| <= 1e-10 *
max |oracle|; FP32 ||gpu - oracle||_2 <= 1e-5 ||oracle||_2.
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


def _plan(D, N, lmax, edges, precision, **kw):
    from paper_2106_10278_gb300.npcf import Plan

    return Plan(D, N, lmax, edges, np.ones(D), precision=precision, **kw)


def _order(plan, keys):
    index = {tuple(int(x) for x in k): i for i, k in enumerate(keys)}
    return np.array([index[tuple(int(x) for x in k)] for k in plan.keys()])


def _check(precision, got, ref):
    if precision == "fp64":
        err, scale = np.max(np.abs(got - ref)), np.max(np.abs(ref))
        assert err <= TOL64 * scale, f"max err {err:.3e} vs scale {scale:.3e}"
    else:
        err, scale = np.linalg.norm(got - ref), np.linalg.norm(ref)
        assert err <= TOL32 * scale, f"rel err {err / scale:.3e}"
    assert scale > 0


def _small_batch(D, seed, fp32=True):
    """Five catalogues of different sizes (one empty) in boxes of different, non-cubic shapes
    (FP32-representable values, or a full FP64 mantissa when fp32 is False)."""
    sizes = [700, 0, 1500, 300, 1100]
    shapes = [[1.0, 1.0, 1.0, 1.0], [0.9, 1.1, 1.0, 1.0], [1.2, 1.0, 0.8, 1.1], [1.0, 0.9, 1.0, 0.9],
              [0.8, 0.8, 0.9, 1.0]]
    boxes = np.array([s[:D] for s in shapes])
    parts, ws = [], []
    for i, n in enumerate(sizes):
        half = n // 2
        p = np.concatenate([catalogs.uniform(half, D, boxes[i], seed + 10 * i, fp32=fp32),
                            catalogs.gaussian_blobs(n - half, D, boxes[i], 4, 0.03, seed + 10 * i + 1, fp32=fp32)])
        parts.append(p)
        ws.append(catalogs.normal_weights(n, 1.0, 0.3, seed + 10 * i + 2, fp32=fp32))
    offsets = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    return np.concatenate(parts), np.concatenate(ws), offsets, boxes


CASES = [
    # D, N, lmax, nbins, r_max
    (3, 3, 5, 8, 0.25),
    (3, 4, 3, 6, 0.25),
    (2, 3, 8, 10, 0.2),
    (2, 4, 4, 6, 0.2),
    (4, 3, 3, 6, 0.3),
]


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("D,N,lmax,nbins,rmax", CASES)
def test_batched_small_parity(D, N, lmax, nbins, rmax, precision):
    pos, w, offsets, boxes = _small_batch(D, 40 + D + N, fp32=precision == "fp32")
    edges = np.linspace(0.02, rmax, nbins + 1)
    plan = _plan(D, N, lmax, edges, precision)
    dt = torch.float64 if precision == "fp64" else torch.float32
    got = plan.compute_batched(torch.tensor(pos, dtype=dt, device="cuda"), torch.tensor(w, dtype=dt, device="cuda"),
                               offsets, boxes).cpu().numpy()
    assert got.shape == (len(offsets) - 1, plan.ncoeff)
    for i in range(len(offsets) - 1):
        a, b = offsets[i], offsets[i + 1]
        if a == b:
            assert np.all(got[i] == 0)
            continue
        keys, ref = oracle.estimate(D, N, lmax, edges, boxes[i], pos[a:b], w[a:b])
        _check(precision, got[i], ref[_order(plan, keys)])


def test_batched_equals_single_calls_and_repeats():
    pos, w, offsets, boxes = _small_batch(3, 7)
    edges = np.linspace(0.02, 0.25, 7)
    plan = _plan(3, 3, 4, edges, "fp64")
    tp = torch.tensor(pos, dtype=torch.float64, device="cuda")
    tw = torch.tensor(w, dtype=torch.float64, device="cuda")
    z1 = plan.compute_batched(tp, tw, offsets, boxes).clone()
    z2 = plan.compute_batched(tp, tw, offsets, boxes)  # cached layout
    assert torch.equal(z1, z2)
    for i in range(len(offsets) - 1):
        a, b = int(offsets[i]), int(offsets[i + 1])
        if a == b:
            continue
        from paper_2106_10278_gb300.npcf import Plan

        single = Plan(3, 3, 4, edges, boxes[i], precision="fp64")
        zs = single.compute(tp[a:b].contiguous(), tw[a:b].contiguous())
        err = (z1[i] - zs).abs().max().item()
        assert err <= 1e-12 * zs.abs().max().item()
    # a single catalogue through the batched entry point, then the single entry point again
    zb = plan.compute_batched(tp[:700].contiguous(), tw[:700].contiguous(), [0, 700], boxes[:1])
    zs = plan.compute(tp[:700].contiguous(), tw[:700].contiguous())
    assert (zb[0] - zs).abs().max().item() <= 1e-12 * zs.abs().max().item()


def test_batched_rejections():
    from paper_2106_10278_gb300.npcf import NpcfError

    pos, w, offsets, boxes = _small_batch(3, 9)
    edges = np.linspace(0.02, 0.25, 5)
    plan = _plan(3, 3, 2, edges, "fp64", sync_check=True)
    tp = torch.tensor(pos, dtype=torch.float64, device="cuda")
    tw = torch.tensor(w, dtype=torch.float64, device="cuda")
    bad = offsets.copy()
    bad[2], bad[3] = bad[3], bad[2]
    with pytest.raises(NpcfError) as e:
        plan.compute_batched(tp, tw, bad, boxes)
    assert e.value.status == -1
    small = boxes.copy()
    small[3] = [0.5, 0.5, 0.5]  # r_max 0.25 needs a side of at least 2.25 r_max
    with pytest.raises(NpcfError) as e:
        plan.compute_batched(tp, tw, offsets, small)
    assert e.value.status == -2
    # a particle outside its own catalogue's box (inside another's) is flagged
    moved = pos.copy()
    moved[offsets[4]] = [0.85, 0.1, 0.1]  # catalogue 4's box is 0.8 x 0.8 x 0.9
    with pytest.raises(NpcfError) as e:
        plan.compute_batched(torch.tensor(moved, dtype=torch.float64, device="cuda"), tw, offsets, boxes)
    assert e.value.status == -6


def test_batch64_full_size():
    """The 64-catalogue workload (about 1.2e7 particles in boxes of side 500-1000, 8 bins over [10, 120]):
    the 3PCF at lmax 10 and the 4PCF at lmax 4 in FP32 through one batched call, against the
    single-catalogue call on the smallest, the largest and one more catalogue; the single call is pinned
    to the oracle on a block of primaries of the smallest catalogue."""
    from paper_2106_10278_gb300.npcf import Plan

    bw = catalogs.batch64()
    sizes = np.diff(bw.offsets)
    picks = [int(np.argmin(sizes)), int(np.argmax(sizes)), 17]
    tp = torch.tensor(bw.pos, dtype=torch.float32, device="cuda")
    tw = torch.tensor(bw.w, dtype=torch.float32, device="cuda")
    for N, lmax in ((3, 10), (4, 4)):
        plan = Plan(3, N, lmax, bw.edges, np.full(3, 1000.0), precision="fp32")
        zb = plan.compute_batched(tp, tw, bw.offsets, bw.boxes).cpu().numpy()
        assert plan.stats()["pairs"] > 4e10
        for i in picks:
            a, b = int(bw.offsets[i]), int(bw.offsets[i + 1])
            single = Plan(3, N, lmax, bw.edges, bw.boxes[i], precision="fp32")
            zs = single.compute(tp[a:b].contiguous(), tw[a:b].contiguous()).cpu().numpy()
            _check("fp32", zb[i], zs)
            if i == picks[0]:
                prims = (1000, 1040)
                zp = single.compute(tp[a:b].contiguous(), tw[a:b].contiguous(), primaries=prims).cpu().numpy()
                p, ww, box = bw.catalogue(i)
                keys, ref = oracle.estimate(3, N, lmax, bw.edges, box, p, ww, primaries=prims)
                _check("fp32", zp, ref[_order(single, keys)])
