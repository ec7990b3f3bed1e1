"""The remove_self and parity plan options on the GPU, against the FP64 oracle, through the C ABI.

remove_self subtracts, for N=3 keys with b1 = b2, the tuples whose two secondaries coincide (the
naive sum of eq. NPCF-estimator-intro-discrete keeps them; the oracle's remove_self option is
pinned against the naive sum that skips them).  parity returns the components of one behaviour
under r -> -r, (-1)^(l1+l2+l3), of the D=3 4PCF.  Tolerances as elsewhere: FP64 max error
<= 1e-10 max |oracle| (full-mantissa inputs); FP32 ||error||_2 <= 1e-5 ||oracle||_2.
"""
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

    return Plan(D, N, lmax, edges, box, precision=precision, **kw)


def _aligned(plan, keys, ref):
    index = {tuple(int(x) for x in k): i for i, k in enumerate(keys)}
    return ref[np.array([index[tuple(int(x) for x in k)] for k in plan.keys()])]


def _check(precision, got, ref):
    if precision == "fp64":
        err, scale = np.max(np.abs(got - ref)), np.max(np.abs(ref))
        assert err <= 1e-10 * scale, f"max err {err:.3e} vs scale {scale:.3e}"
    else:
        err, scale = np.linalg.norm(got - ref), np.linalg.norm(ref)
        assert err <= 1e-5 * scale, f"rel err {err / scale:.3e}"
    assert scale > 0


def _catalog(D, n, seed, precision):
    f32 = precision == "fp32"
    pos = np.concatenate([catalogs.uniform(n // 2, D, 1.0, seed, fp32=f32),
                          catalogs.gaussian_blobs(n - n // 2, D, 1.0, 6, 0.03, seed + 1, fp32=f32)])
    w = catalogs.normal_weights(n, 1.0, 0.4, seed + 2, fp32=f32)
    return pos, w


def _run(plan, pos, w, primaries=None):
    dt = torch.float64 if plan.precision == "fp64" else torch.float32
    return plan.compute(torch.tensor(pos, dtype=dt, device="cuda"), torch.tensor(w, dtype=dt, device="cuda"),
                        primaries=primaries).cpu().numpy()


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("D,lmax,nbins", [(2, 8, 8), (3, 5, 10), (4, 3, 6)])
def test_remove_self_matches_oracle(D, lmax, nbins, precision):
    pos, w = _catalog(D, 2500, 20 + D, precision)
    edges = np.linspace(0.01, 0.25 if D < 4 else 0.35, nbins + 1)
    plan = _plan(D, 3, lmax, edges, np.ones(D), precision, remove_self=True)
    got = _run(plan, pos, w, primaries=(0, 900))
    keys, ref = oracle.estimate(D, 3, lmax, edges, np.ones(D), pos, w, primaries=(0, 900), remove_self=True)
    _check(precision, got, _aligned(plan, keys, ref))
    # only the b1 = b2 keys change, and by the coincident terms
    base = _run(_plan(D, 3, lmax, edges, np.ones(D), precision), pos, w, primaries=(0, 900))
    k = plan.keys()
    same = k[:, 0] != k[:, 1]
    assert np.array_equal(got[same], base[same])
    assert np.all(got[~same] != base[~same])


def test_remove_self_batched_and_bins_lt():
    pos, w = _catalog(3, 2000, 31, "fp64")
    edges = np.linspace(0.02, 0.2, 6)
    offsets = np.array([0, 1200, 2000], dtype=np.int64)
    boxes = np.ones((2, 3))
    plan = _plan(3, 3, 4, edges, np.ones(3), "fp64", remove_self=True)
    got = plan.compute_batched(torch.tensor(pos, device="cuda"), torch.tensor(w, device="cuda"), offsets,
                               boxes).cpu().numpy()
    for i in range(2):
        a, b = offsets[i], offsets[i + 1]
        keys, ref = oracle.estimate(3, 3, 4, edges, boxes[i], pos[a:b], w[a:b], remove_self=True)
        _check("fp64", got[i], _aligned(plan, keys, ref))
    # with b1 < b2 keys there is nothing to remove
    lt = _plan(3, 3, 4, edges, np.ones(3), "fp64", remove_self=True, bin_lt=True)
    lt0 = _plan(3, 3, 4, edges, np.ones(3), "fp64", bin_lt=True)
    assert np.array_equal(_run(lt, pos, w), _run(lt0, pos, w))


def test_remove_self_refused_by_backward():
    from paper_2106_10278_gb300.npcf import NpcfError

    plan = _plan(3, 3, 2, np.linspace(0.1, 0.3, 3), np.ones(3), "fp64", remove_self=True)
    pos = torch.rand(50, 3, dtype=torch.float64, device="cuda")
    w = torch.ones(50, dtype=torch.float64, device="cuda")
    with pytest.raises(NpcfError, match="UNSUPPORTED"):
        plan.backward(pos, w, torch.zeros(2 * plan.ncoeff, dtype=torch.float64, device="cuda"))


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_parity_selection_d3n4(precision):
    pos, w = _catalog(3, 2500, 41, precision)
    edges = np.linspace(0.02, 0.25, 7)
    full = _plan(3, 4, 4, edges, np.ones(3), precision)
    zf = _run(full, pos, w, primaries=(0, 300))
    kf = {tuple(k): i for i, k in enumerate(full.keys())}
    keys, ref = oracle.estimate(3, 4, 4, edges, np.ones(3), pos, w, primaries=(0, 300))
    n = 0
    for par, want in (("even", 0), ("odd", 1)):
        plan = _plan(3, 4, 4, edges, np.ones(3), precision, parity=par)
        k = plan.keys()
        assert np.all((k[:, 3] + k[:, 4] + k[:, 5]) % 2 == want)
        z = _run(plan, pos, w, primaries=(0, 300))
        # the same arithmetic as the full plan, the columns selected in the final reduction
        assert np.array_equal(z, zf[[kf[tuple(x)] for x in k]])
        _check(precision, z, _aligned(plan, keys, ref))
        if want == 1:  # odd components are imaginary
            assert np.max(np.abs(z.real)) <= 1e-6 * np.max(np.abs(z.imag))
        n += plan.ncoeff
    assert n == full.ncoeff


def test_parity_refusals():
    from paper_2106_10278_gb300.npcf import NpcfError

    for D, N, nb in ((3, 3, 3), (2, 4, 4), (3, 5, 5)):
        with pytest.raises(NpcfError, match="UNSUPPORTED"):
            _plan(D, N, 2, np.linspace(0.05, 0.3, nb + 1), np.ones(D), "fp32", parity="odd")
    even = _plan(3, 3, 3, np.linspace(0.05, 0.3, 4), np.ones(3), "fp32", parity="even")
    assert even.ncoeff == _plan(3, 3, 3, np.linspace(0.05, 0.3, 4), np.ones(3), "fp32").ncoeff
