"""Points on the unit 2-sphere (Sec. "Cosmic Microwave Background", reading R17) on the GPU,
through the C ABI, against the FP64 oracle's estimate_sphere: the D = 2 basis about every
primary, bins in cos theta, 1/(4 pi) for 1/V.  The oracle's sphere estimator is pinned in
test_oracle_sphere.py (naive sum, rotations and a reflection, a frame-free 3PCF, l = 0 pair
counts, the paper's 35 x 120 components).

Tolerances: FP64 max error <= 1e-10 max |oracle| (inputs with a full FP64 mantissa and random
lengths); FP32 ||error||_2 <= 1e-5 ||oracle||_2 (inputs rounded to FP32)."""
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


def _clumpy(n, seed, fp32=True, lengths=False):
    """Half uniform directions, half in 40 clumps of angular width ~0.05 rad; optional random
    lengths in [0.5, 2) (the estimator normalises)."""
    rng = np.random.default_rng(seed)
    nu = n // 2
    v = rng.normal(size=(n, 3))
    centres = rng.normal(size=(40, 3))
    centres /= np.linalg.norm(centres, axis=1, keepdims=True)
    c = centres[rng.integers(0, 40, n - nu)]
    v[nu:] = c + 0.05 * rng.normal(size=(n - nu, 3))
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    if lengths:
        v *= rng.uniform(0.5, 2.0, size=(n, 1))
    return v.astype(np.float32).astype(np.float64) if fp32 else v


def _plan(N, lmax, ce, precision):
    from paper_2106_10278_gb300.npcf import Plan

    return Plan(2, N, lmax, np.asarray(ce), None, precision=precision, geometry="sphere")


def _run(plan, pos, w, primaries=None):
    dt = torch.float64 if plan.precision == "fp64" else torch.float32
    return plan.compute(torch.tensor(pos, dtype=dt, device="cuda"), torch.tensor(w, dtype=dt, device="cuda"),
                        primaries=primaries).cpu().numpy()


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
        assert err <= 1e-5 * nrm, f"rel err {err / nrm:.3e}"


CASES = [
    # N, lmax, cos theta edges, n, primaries
    (3, 4, np.linspace(-0.5, 0.5, 11), 3000, None),          # the paper's example binning
    (4, 4, np.linspace(0.2, 0.9, 7), 2500, (0, 600)),
    (3, 8, np.linspace(0.95, 0.999, 9), 20000, (0, 2500)),    # small angles, several cells per bin
    (4, 3, np.array([0.0, 0.3, 0.6, 0.8, 0.95, 1.0]), 2000, (0, 500)),  # up to theta = 0
]


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("N,lmax,ce,n,prims", CASES)
def test_sphere_matches_oracle(N, lmax, ce, n, prims, precision):
    f32 = precision == "fp32"
    pos = _clumpy(n, 70 + N + lmax, fp32=f32, lengths=not f32)
    w = catalogs.normal_weights(n, 1.0, 0.3, 71 + N, fp32=f32)
    plan = _plan(N, lmax, ce, precision)
    got = _run(plan, pos, w, prims)
    keys, ref = oracle.estimate_sphere(N, lmax, ce, pos, w, primaries=prims)
    _check(precision, got, _aligned(plan, keys, ref))


def test_sphere_coincident_points_and_ranges():
    """Duplicated directions (cos theta = 1) are no pair on either side; the sum over two
    primary ranges equals the whole."""
    pos = _clumpy(1500, 5, fp32=True)
    pos = np.concatenate([pos, pos[:200]])
    w = catalogs.normal_weights(len(pos), 1.0, 0.3, 6)
    ce = np.array([0.5, 0.8, 0.95, 1.0])
    plan = _plan(3, 4, ce, "fp64")
    whole = _run(plan, pos, w)
    keys, ref = oracle.estimate_sphere(3, 4, ce, pos, w)
    _check("fp64", whole, _aligned(plan, keys, ref))
    half = _run(plan, pos, w, (0, 800)) + _run(plan, pos, w, (800, len(pos)))
    _check("fp64", half, whole)


def test_sphere_refusals():
    from paper_2106_10278_gb300.npcf import NpcfError, Plan

    ce = np.linspace(0.0, 0.5, 4)
    with pytest.raises(NpcfError, match="UNSUPPORTED"):
        Plan(3, 3, 4, ce, None, geometry="sphere")
    with pytest.raises(NpcfError, match="UNSUPPORTED"):
        Plan(2, 3, 4, ce, None, geometry="sphere", remove_self=True)
    with pytest.raises(NpcfError, match="ERR_ARG"):
        Plan(2, 3, 4, np.array([-1.0, 0.0, 0.5]), None, geometry="sphere")
    with pytest.raises(NpcfError, match="ERR_ARG"):
        Plan(2, 3, 4, np.array([0.0, 0.5, 1.5]), None, geometry="sphere")
    plan = Plan(2, 3, 4, ce, None, geometry="sphere", precision="fp64")
    pos = torch.tensor(_clumpy(100, 1, fp32=False), device="cuda")
    w = torch.ones(100, dtype=torch.float64, device="cuda")
    with pytest.raises(NpcfError, match="UNSUPPORTED"):
        plan.backward(pos, w, torch.zeros(2 * plan.ncoeff, dtype=torch.float64, device="cuda"))
    with pytest.raises(NpcfError, match="UNSUPPORTED"):
        plan.compute_batched(pos, w, [0, 50, 100], np.ones((2, 2)))
    with pytest.raises(ValueError):
        plan.compute(pos[:, :2].contiguous(), w)
