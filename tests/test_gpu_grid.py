"""The FFT form of the gridded-field estimator (Sec. "Application to Gridded Data", reading R16) on
the GPU, through the C ABI, against the FP64 oracle's direct sum over node offsets
(oracle.estimate_grid).  The oracle's gridded estimator is pinned in test_oracle_grid.py (NGP deposit
= discrete estimator at cell centres; numpy's FFT form of a^b_l).

Fields are lognormal densities (mean 1, power-law spectrum).  Tolerances: FP64 max error <= 1e-10
max |oracle| (the transforms round at ~1e-16 times log2 of the node count); FP32 ||error||_2 <=
2e-5 ||oracle||_2 (FP32 transforms round each convolution at ~1e-7 log2(nodes) of its own norm;
three factors and the node sum add a few of those)."""
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


def _plan(D, N, lmax, edges, box, precision, **kw):
    from paper_2106_10278_gb300.npcf import Plan

    return Plan(D, N, lmax, np.asarray(edges), np.asarray(box, dtype=np.float64), precision=precision,
                periodic=True, **kw)


def _grid(plan, X):
    dt = torch.float64 if plan.precision == "fp64" else torch.float32
    return plan.compute_grid(torch.tensor(X, dtype=dt, device="cuda")).cpu().numpy()


def _aligned(plan, keys, ref):
    index = {tuple(int(x) for x in k): i for i, k in enumerate(keys)}
    return ref[np.array([index[tuple(int(x) for x in k)] for k in plan.keys()])]


def _check(precision, got, ref):
    scale = np.max(np.abs(ref))
    assert scale > 0
    if precision == "fp64":
        err = np.max(np.abs(got - ref))
        assert err <= 1e-10 * scale, f"max err {err:.3e} vs scale {scale:.3e}"
    else:
        err, nrm = np.linalg.norm(got - ref), np.linalg.norm(ref)
        assert err <= 2e-5 * nrm, f"rel err {err / nrm:.3e}"


GRID_CASES = [
    # D, N, lmax, dims, box, edges
    (2, 3, 6, (32, 32), (1.0, 1.0), [0.07, 0.13, 0.2, 0.27, 0.33]),
    (2, 4, 4, (40, 24), (1.25, 0.75), [0.06, 0.12, 0.18, 0.24, 0.3]),
    (3, 3, 5, (16, 16, 16), (1.0, 1.0, 1.0), [0.07, 0.13, 0.2, 0.27, 0.33]),
    (3, 4, 3, (18, 14, 20), (0.9, 0.7, 1.0), [0.06, 0.12, 0.18, 0.24, 0.3]),
    (3, 5, 2, (16, 16, 16), (1.0, 1.0, 1.0), [0.09, 0.15, 0.22, 0.29, 0.36]),
    (4, 3, 3, (8, 8, 8, 8), (1.0, 1.0, 1.0, 1.0), [0.13, 0.2, 0.3, 0.37]),
]


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("D,N,lmax,dims,box,edges", GRID_CASES)
def test_grid_matches_oracle(D, N, lmax, dims, box, edges, precision):
    X = catalogs.lognormal_field(dims, 500 + 10 * D + N, fp32=precision == "fp32")
    plan = _plan(D, N, lmax, edges, box, precision)
    got = _grid(plan, X)
    keys, ref = oracle.estimate_grid(N, lmax, np.asarray(edges), np.asarray(box), X)
    _check(precision, got, _aligned(plan, keys, ref))


def test_grid_cached_kernels_follow_the_shape():
    """The kernels' transforms are cached for the last grid shape: a second call on the same shape
    gives the same bits; a call on another shape, and then on the first shape again, rebuilds them."""
    edges = [0.07, 0.13, 0.2, 0.27]
    plan = _plan(3, 3, 3, edges, (1.0, 1.0, 1.0), "fp64")
    Xa = catalogs.lognormal_field((16, 16, 16), 71, fp32=False)
    Xb = catalogs.lognormal_field((12, 20, 16), 72, fp32=False)
    a1, a2 = _grid(plan, Xa), _grid(plan, Xa)
    assert np.array_equal(a1, a2)
    b = _grid(plan, Xb)
    a3 = _grid(plan, Xa)
    assert np.array_equal(a1, a3)
    for X, got in ((Xa, a1), (Xb, b)):
        keys, ref = oracle.estimate_grid(3, 3, np.asarray(edges), np.ones(3), X)
        _check("fp64", got, _aligned(plan, keys, ref))


def test_grid_constant_field():
    """A constant field X: a^b_00 = X dV (nodes in shell b) / (v_b sqrt(4 pi)), so the l = 0
    coefficient of the 3PCF is X a^0_00 a^1_00 (the node sum of dV X over the box is X V), with the
    shell's nodes counted directly; the rest is compared with the oracle as usual."""
    edges = np.array([0.1, 0.2, 0.3])
    X = np.full((20, 20, 20), 1.5)
    plan = _plan(3, 3, 2, edges, (1.0, 1.0, 1.0), "fp64")
    got = _grid(plan, X)
    keys, ref = oracle.estimate_grid(3, 2, edges, np.ones(3), X)
    _check("fp64", got, _aligned(plan, keys, ref))
    h = 1.0 / 20
    o = np.arange(-6, 7)
    r2 = (o[:, None, None] ** 2 + o[None, :, None] ** 2 + o[None, None, :] ** 2) * h * h
    cnt = [np.count_nonzero((r2 >= edges[b] ** 2) & (r2 < edges[b + 1] ** 2) & (r2 > 0)) for b in range(2)]
    vb = [4 * np.pi / 3 * (edges[b + 1] ** 3 - edges[b] ** 3) for b in range(2)]
    a0 = [1.5 * h ** 3 * cnt[b] / vb[b] / np.sqrt(4 * np.pi) for b in range(2)]
    k = plan.keys()
    i = [j for j in range(len(k)) if k[j][0] == 0 and k[j][1] == 1 and all(x == 0 for x in k[j][3:])]
    assert len(i) == 1
    expect = 1.5 * a0[0] * a0[1]
    assert abs(got[i[0]] - expect) <= 1e-12 * abs(expect)


def test_grid_refusals():
    from paper_2106_10278_gb300.npcf import NpcfError, Plan

    edges = np.array([0.1, 0.2, 0.3])
    X = torch.ones((16, 16, 16), dtype=torch.float64, device="cuda")
    plan = Plan(3, 3, 2, edges, np.ones(3), precision="fp64", periodic=False)
    with pytest.raises(NpcfError, match="UNSUPPORTED"):
        plan.compute_grid(X)
    plan = _plan(3, 3, 2, edges, (1.0, 1.0, 1.0), "fp64")
    with pytest.raises(TypeError):
        plan.compute_grid(X.float())
    with pytest.raises(ValueError):
        plan.compute_grid(X[0])
    plan = _plan(3, 3, 2, edges, (1.0, 1.0, 1.0), "fp64", remove_self=True)
    with pytest.raises(NpcfError, match="UNSUPPORTED"):
        plan.compute_grid(X)
