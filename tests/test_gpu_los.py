"""The basis about the x_3 line of sight (Sec. "Large-Scale Structure"; reading R18) on the GPU,
against the FP64 oracle's estimate_aniso, through the C ABI.

N=3 keys (b1, b2; l1, l2, L), N=4 keys (b1 < b2 < b3; l1, l2, l12, l3, L).  The L = 0 slice must
equal the isotropic plan's coefficients.  Tolerances as elsewhere: FP64 max error <= 1e-10 max
|oracle| on full-mantissa inputs; FP32 ||error||_2 <= 1e-5 ||oracle||_2.
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


def _plan(N, lmax, edges, precision, **kw):
    from paper_2106_10278_gb300.npcf import Plan

    return Plan(3, N, lmax, edges, np.ones(3), precision=precision, **kw)


def _run(plan, pos, w, primaries=None):
    dt = torch.float64 if plan.precision == "fp64" else torch.float32
    return plan.compute(torch.tensor(pos, dtype=dt, device="cuda"), torch.tensor(w, dtype=dt, device="cuda"),
                        primaries=primaries).cpu().numpy()


def _check(precision, got, ref):
    if precision == "fp64":
        err, scale = np.max(np.abs(got - ref)), np.max(np.abs(ref))
        assert err <= 1e-10 * scale, f"max err {err:.3e} vs scale {scale:.3e}"
    else:
        err, scale = np.linalg.norm(got - ref), np.linalg.norm(ref)
        assert err <= 1e-5 * scale, f"rel err {err / scale:.3e}"
    assert scale > 0


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("N,lmax,nbins,prims", [(3, 4, 6, (0, 800)), (3, 5, 10, (0, 400)), (4, 3, 5, (0, 200))])
def test_los_matches_oracle(N, lmax, nbins, prims, precision):
    f32 = precision == "fp32"
    n = 2500
    pos = np.concatenate([catalogs.uniform(n // 2, 3, 1.0, 61, fp32=f32),
                          catalogs.gaussian_blobs(n - n // 2, 3, 1.0, 6, 0.04, 62, fp32=f32)])
    w = catalogs.normal_weights(n, 1.0, 0.3, 63, fp32=f32)
    edges = np.linspace(0.02, 0.25, nbins + 1)
    plan = _plan(N, lmax, edges, precision, basis="los")
    got = _run(plan, pos, w, prims)
    keys, ref = oracle.estimate_aniso(N, lmax, edges, np.ones(3), pos, w, primaries=prims)
    pk = plan.keys()
    assert pk.shape == keys.shape
    index = {tuple(int(x) for x in k): i for i, k in enumerate(keys)}
    _check(precision, got, ref[np.array([index[tuple(int(x) for x in k)] for k in pk])])
    # L = 0 is the isotropic basis
    iso = _plan(N, lmax, edges, precision)
    zi = _run(iso, pos, w, prims)
    ik = {tuple(int(x) for x in k): i for i, k in enumerate(iso.keys())}
    sel, idx = [], []
    for i, k in enumerate(pk):
        if N == 3 and k[5] == 0:
            sel.append(i)
            idx.append(ik[(k[0], k[1], -1, k[3], 0, 0)])
        if N == 4 and k[7] == 0:  # L = 0 forces l3 = l12
            sel.append(i)
            idx.append(ik[(k[0], k[1], k[2], k[3], k[4], k[6])])
    assert len(sel) > 0
    _check(precision, got[sel], zi[idx])


def test_los_refusals():
    from paper_2106_10278_gb300.npcf import NpcfError, Plan

    edges = np.linspace(0.05, 0.3, 5)
    for kw in ({"remove_self": True}, {"precision": "mixed_bf16x3"}, {"parity": "even"}):
        with pytest.raises(NpcfError, match="UNSUPPORTED"):
            Plan(3, 3, 3, edges, np.ones(3), basis="los", **kw)
    with pytest.raises(NpcfError, match="UNSUPPORTED"):
        Plan(2, 3, 3, edges, np.ones(2), basis="los")
    plan = Plan(3, 3, 2, edges, np.ones(3), basis="los", precision="fp64")
    with pytest.raises(NpcfError, match="UNSUPPORTED"):
        plan.backward(torch.rand(20, 3, dtype=torch.float64, device="cuda"),
                      torch.ones(20, dtype=torch.float64, device="cuda"),
                      torch.zeros(2 * plan.ncoeff, dtype=torch.float64, device="cuda"))
