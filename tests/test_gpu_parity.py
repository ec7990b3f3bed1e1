"""Parity of the CUDA path with the FP64 oracle, through the C ABI.

Tolerances (both stated by the target of this implementation):
  FP64 plans:  max |gpu - oracle| <= 1e-10 * max |oracle|
  FP32 plans:  ||gpu - oracle||_2 <= 1e-5 * ||oracle||_2
Bin decisions are exact on both paths (pairs near an edge are re-decided in
FP64 from the original coordinates), so the pair sets agree exactly.  FP64
plans are tested on positions and weights with a full FP64 mantissa (the
generators' fp32=False), FP32 plans on FP32-representable ones.
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


def _plan(D, N, lmax, edges, box, precision, **kw):
    from paper_2106_10278_gb300.npcf import Plan

    return Plan(D, N, lmax, edges, box, precision=precision, **kw)


def _run(plan, pos, w, primaries=None):
    dt = torch.float64 if plan.precision == "fp64" else torch.float32
    z = plan.compute(torch.tensor(pos, dtype=dt, device="cuda"), torch.tensor(w, dtype=dt, device="cuda"),
                     primaries=primaries)
    torch.cuda.synchronize()
    return z.cpu().numpy()


def _aligned_oracle(plan, keys, ref):
    index = {tuple(int(x) for x in k): i for i, k in enumerate(keys)}
    order = np.array([index[tuple(int(x) for x in k)] for k in plan.keys()])
    assert len(order) == len(keys)
    return ref[order]


def _check(plan, got, ref):
    if plan.precision == "fp64":
        err = np.max(np.abs(got - ref))
        scale = np.max(np.abs(ref))
        assert err <= TOL64 * scale, f"max err {err:.3e} vs scale {scale:.3e}"
    else:
        err = np.linalg.norm(got - ref)
        scale = np.linalg.norm(ref)
        assert err <= TOL32 * scale, f"rel err {err / scale:.3e}"
    assert scale > 0


def _compare(D, N, lmax, edges, box, pos, w, precision, primaries=None, periodic=True, bin_lt=False):
    plan = _plan(D, N, lmax, edges, box, precision, periodic=periodic, bin_lt=bin_lt)
    got = _run(plan, pos, w, primaries)
    keys, ref = oracle.estimate(D, N, lmax, edges, box, pos, w, primaries=primaries, periodic=periodic,
                                bin_lt=bin_lt)
    ref = _aligned_oracle(plan, keys, ref)
    _check(plan, got, ref)
    return plan, got, ref


# ----------------------------------------------------------- small, all (D, N)
CASES = [
    # D, N, lmax, nbins, n, primaries
    (2, 3, 10, 16, 3000, None),
    (3, 3, 5, 10, 2500, None),
    (4, 3, 4, 8, 2500, None),
    (2, 4, 6, 8, 2500, (0, 700)),
    (3, 4, 5, 10, 2500, (0, 150)),
    (3, 4, 2, 5, 2000, (100, 900)),
]


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("D,N,lmax,nbins,n,prims", CASES)
def test_parity_small(D, N, lmax, nbins, n, prims, precision):
    g = np.random.default_rng(D * 100 + N * 10 + lmax)
    f32 = precision == "fp32"
    pos = np.concatenate([catalogs.uniform(n // 2, D, 1.0, D + 7, fp32=f32),
                          catalogs.gaussian_blobs(n - n // 2, D, 1.0, 7, 0.03, D + 8, fp32=f32)])
    w = catalogs.normal_weights(n, 1.0, 0.3, D + 9, fp32=f32) * np.where(g.random(n) < 0.3, -1.0, 1.0)
    if not f32:  # the FP64 path must not narrow its inputs: they carry more than FP32's 24 bits
        assert not np.array_equal(pos.astype(np.float32).astype(np.float64), pos)
        assert not np.array_equal(w.astype(np.float32).astype(np.float64), w)
    edges = np.linspace(0.02, 0.3 if D < 4 else 0.4, nbins + 1)
    _compare(D, N, lmax, edges, np.ones(D), pos, w, precision, primaries=prims)


def test_fp64_d3n3_workload_full():
    """D=3 3PCF in FP64, n=2000 in a periodic cube of side 250 (full-mantissa positions), 10 bins over
    [0, 100], lmax=5; the weights get a full mantissa too."""
    wl = catalogs.workload("d3n3_fp64")
    assert not np.array_equal(wl.pos.astype(np.float32).astype(np.float64), wl.pos)
    w = catalogs.normal_weights(wl.n, 1.0, 0.3, 17, fp32=False)
    _compare(wl.D, wl.N, wl.lmax, wl.edges, wl.box, wl.pos, w, "fp64")


def test_fp64_d3n3_bruteforce_n200():
    """The GPU against the naive N-tuplet sum projected on the same basis (n=200)."""
    wl = catalogs.workload("d3n3_fp64", scale=0.1)
    w = catalogs.normal_weights(wl.n, 1.0, 0.3, 18, fp32=False)
    plan = _plan(3, 3, 5, wl.edges, wl.box, "fp64")
    got = _run(plan, wl.pos, w)
    keys, ref = oracle.estimate(3, 3, 5, wl.edges, wl.box, wl.pos, w, brute=True)
    _check(plan, got, _aligned_oracle(plan, keys, ref))


def test_bins_lt_and_open_boundaries():
    pos = catalogs.uniform(1200, 3, 1.0, 3) * 0.98 + 0.01
    pos = pos.astype(np.float32).astype(np.float64)
    w = np.ones(1200)
    edges = np.linspace(0.05, 0.25, 5)
    _compare(3, 3, 4, edges, np.ones(3), pos, w, "fp32", periodic=False)
    _compare(3, 3, 4, edges, np.ones(3), pos, w, "fp64", bin_lt=True)


def test_pairs_exactly_on_bin_edges():
    """Integer positions in a box of side 16 put many separations exactly on the
    integer bin edges: both paths must decide them as [e_b, e_{b+1}) does."""
    g = np.random.default_rng(3)
    pos = g.integers(0, 16, size=(600, 3)).astype(np.float64)
    pos = np.unique(pos, axis=0)
    w = g.normal(1.0, 0.5, len(pos))
    edges = np.array([0.0, 1.0, 2.0, 3.0, 4.0, 5.0, 6.0])
    for prec in ("fp64", "fp32"):
        _compare(3, 3, 3, edges, np.full(3, 16.0), pos, w, prec)
    _compare(3, 4, 2, edges, np.full(3, 16.0), pos, w, "fp32", primaries=(0, 120))


def test_dense_clump_overfills_queues():
    """All particles in one tight clump: every pair lands in few bins, which
    drives the per-bin queues to capacity."""
    g = np.random.default_rng(5)
    pos = (0.5 + g.normal(0, 0.01, size=(1500, 3))).astype(np.float32).astype(np.float64)
    w = np.ones(1500)
    edges = np.array([0.0, 0.005, 0.01, 0.02, 0.08])
    _compare(3, 3, 4, edges, np.ones(3), pos, w, "fp32")
    _compare(2, 3, 6, edges, np.ones(2), pos[:, :2], w, "fp32")


def test_empty_and_tiny_inputs():
    edges = np.linspace(0.1, 0.3, 4)
    plan = _plan(3, 3, 3, edges, np.ones(3), "fp32")
    z = plan.compute(torch.zeros((0, 3), device="cuda"), torch.zeros(0, device="cuda"))
    assert torch.count_nonzero(z).item() == 0
    z = plan.compute(torch.full((1, 3), 0.5, device="cuda"), torch.ones(1, device="cuda"))
    assert torch.count_nonzero(z).item() == 0
    pos = np.array([[0.5, 0.5, 0.5], [0.6, 0.5, 0.5], [0.5, 0.72, 0.5]])
    _compare(3, 3, 3, edges, np.ones(3), pos, np.array([1.0, 2.0, -0.5]), "fp64")


def test_primary_ranges_add_up():
    """zeta over [0, n) equals the sum over a partition of the primaries."""
    pos = catalogs.uniform(3000, 3, 1.0, 21)
    w = catalogs.normal_weights(3000, 1.0, 0.2, 22)
    edges = np.linspace(0.03, 0.2, 7)
    plan = _plan(3, 4, 3, edges, np.ones(3), "fp64")
    full = _run(plan, pos, w)
    parts = sum(_run(plan, pos, w, primaries=(a, b)) for a, b in [(0, 700), (700, 701), (701, 2500), (2500, 3000)])
    np.testing.assert_allclose(parts, full, rtol=0, atol=1e-12 * np.max(np.abs(full)))


def test_deterministic_bitwise():
    pos = catalogs.uniform(4000, 3, 1.0, 31)
    w = catalogs.normal_weights(4000, 1.0, 0.2, 32)
    plan = _plan(3, 4, 4, np.linspace(0.02, 0.2, 8), np.ones(3), "fp32")
    a = _run(plan, pos, w)
    b = _run(plan, pos, w)
    assert np.array_equal(a, b)


def test_invalid_input_reported():
    from paper_2106_10278_gb300.npcf import NpcfError

    plan = _plan(3, 3, 2, np.linspace(0.1, 0.3, 3), np.ones(3), "fp32")
    pos = torch.rand(100, 3, device="cuda")
    w = torch.ones(100, device="cuda")
    pos[7, 1] = float("nan")
    with pytest.raises(NpcfError, match="NONFINITE"):
        plan.compute(pos, w)
    pos[7, 1] = 1.5  # outside [0, box)
    with pytest.raises(NpcfError, match="NONFINITE"):
        plan.compute(pos, w)
    with pytest.raises(NpcfError, match="ERR_ARG"):
        plan.compute(torch.rand(10, 3, device="cuda"), torch.ones(10, device="cuda"), primaries=(5, 11))


def test_host_entry_point_matches_device_entry_point():
    pos = catalogs.uniform(2000, 3, 1.0, 41)
    w = catalogs.normal_weights(2000, 1.0, 0.2, 42)
    plan = _plan(3, 4, 3, np.linspace(0.03, 0.2, 6), np.ones(3), "fp32")
    dev = _run(plan, pos, w)
    host = plan.compute_host(pos, w)
    assert np.array_equal(dev, host)


# ------------------------------------------- full-size workloads, sampled primaries
@pytest.mark.parametrize("name,prims", [("d3n4", (0, 6)), ("d3n4", (1_000_100, 1_000_104)), ("d2n4", (0, 400)),
                                        ("d2n3", (0, 3000)), ("d4n3", (0, 2000)), ("d3n5", (0, 8))])
def test_full_size_workload_sampled_primaries(name, prims):
    """The benchmark workloads at full size (same cell grid and launch as the
    benchmark), compared on a sample of primaries the oracle can afford."""
    wl = catalogs.workload(name)
    _compare(wl.D, wl.N, wl.lmax, wl.edges, wl.box, wl.pos, wl.w, "fp32", primaries=prims)


@pytest.mark.parametrize("name", ["d3n4", "d3n5"])
def test_full_size_launch_equals_sum_of_ranges(name):
    """The benchmark's own launch (every primary of the full-size workload, its coupling grid
    and cross-CTA reduce) against two half-range calls: the coefficients are sums over
    primaries, so the two must agree to FP32 rounding of the per-group sums."""
    wl = catalogs.workload(name)
    plan = _plan(wl.D, wl.N, wl.lmax, wl.edges, wl.box, "fp32")
    pos = torch.tensor(wl.pos, dtype=torch.float32, device="cuda")
    w = torch.tensor(wl.w, dtype=torch.float32, device="cuda")
    full = plan.compute(pos, w).cpu().numpy()
    half = wl.n // 2
    parts = plan.compute(pos, w, primaries=(0, half)).cpu().numpy() + \
        plan.compute(pos, w, primaries=(half, wl.n)).cpu().numpy()
    err, scale = np.linalg.norm(full - parts), np.linalg.norm(full)
    assert scale > 0 and err <= TOL32 * scale, f"rel err {err / scale:.3e}"


# --------------------------- a field on a periodic grid, through the particle path
GRID_FIELDS = [
    # D, N, lmax, nodes per axis, edges
    (2, 3, 6, 32, [0.07, 0.13, 0.2, 0.27, 0.33]),
    (3, 4, 2, 16, [0.07, 0.13, 0.2, 0.27, 0.33]),
    (4, 3, 3, 8, [0.13, 0.2, 0.3, 0.37]),
    (3, 5, 2, 16, [0.09, 0.15, 0.22, 0.29, 0.36]),
]


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("D,N,lmax,M,edges", GRID_FIELDS)
def test_grid_field_as_lattice_particles(D, N, lmax, M, edges, precision):
    """The gridded estimator's direct sums (Sec. "Application to Gridded Data") are the discrete
    estimator of one particle per node with weight X dV.  The nodes put separations on the axes
    (directions such as (0, 0, 0, 1)) and repeat every distance many times; the spacing is a power
    of two, so positions and weights are exact in FP32, and no lattice distance lies on an edge."""
    h = 1.0 / M
    dV = h ** D
    X = np.random.default_rng(40 + D + N).normal(size=(M,) * D)
    w = (X * dV).astype(np.float32).astype(np.float64).reshape(-1)
    pos = np.stack(np.indices((M,) * D), -1).reshape(-1, D) * h
    edges = np.asarray(edges)
    plan = _plan(D, N, lmax, edges, np.ones(D), precision)
    got = _run(plan, pos, w)
    keys, ref = oracle.estimate_grid(N, lmax, edges, 1.0, (w / dV).reshape((M,) * D))
    _check(plan, got, _aligned_oracle(plan, keys, ref))


def test_host_entry_point_rejects_bad_ranges_before_copying():
    """npcf_compute_host validates n and the primary range on the host, before any copy; the plan
    stays usable afterwards."""
    from paper_2106_10278_gb300.npcf import NpcfError

    plan = _plan(3, 3, 2, np.linspace(0.1, 0.3, 3), np.ones(3), "fp32")
    pos = catalogs.uniform(10, 3, 1.0, 3)
    w = np.ones(10)
    for prims in ((5, 11), (6, 2), (-1, 3)):
        with pytest.raises(NpcfError, match="ERR_ARG"):
            plan.compute_host(pos, w, primaries=prims)
    keys, ref = oracle.estimate(3, 3, 2, np.linspace(0.1, 0.3, 3), np.ones(3), pos, w)
    _check(plan, plan.compute_host(pos, w), _aligned_oracle(plan, keys, ref))
