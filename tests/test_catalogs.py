"""The seeded input generators: every position is FP32-representable and inside [0, L) (so the
FP32 device copy and the FP64 oracle copy are the same points), draws are reproducible, and the
named workloads carry the stated parameters."""
import numpy as np

from paper_2106_10278_gb300 import catalogs


def _fp32_in_box(x, L):
    L = np.broadcast_to(np.asarray(L, dtype=np.float64), (x.shape[1],))
    assert np.all(x >= 0.0) and np.all(x < L)
    assert np.array_equal(x.astype(np.float32).astype(np.float64), x)


def test_generators_fp32_in_box_and_reproducible():
    u = catalogs.uniform(5000, 3, [1.0, 2.0, 0.5], 7)
    _fp32_in_box(u, [1.0, 2.0, 0.5])
    assert np.array_equal(u, catalogs.uniform(5000, 3, [1.0, 2.0, 0.5], 7))
    b = catalogs.gaussian_blobs(5000, 4, 1.0, 20, 0.05, 8)
    _fp32_in_box(b, 1.0)
    ln = catalogs.lognormal_poisson(2e4, 300.0, 9, grid=32)
    _fp32_in_box(ln, 300.0)
    assert abs(len(ln) - 2e4) < 5 * np.sqrt(2e4)  # Poisson total around the mean
    w = catalogs.normal_weights(1000, 1.0, 0.1, 3)
    assert np.array_equal(w.astype(np.float32).astype(np.float64), w)


def test_full_mantissa_generators_for_fp64_plans():
    """fp32=False keeps the FP64 mantissa (the inputs of FP64 plans), inside the same box and with the
    same underlying draws (the FP32 variant is their rounding)."""
    u = catalogs.uniform(5000, 3, [1.0, 2.0, 0.5], 7, fp32=False)
    assert np.all(u >= 0.0) and np.all(u < [1.0, 2.0, 0.5])
    assert not np.array_equal(u.astype(np.float32).astype(np.float64), u)
    u32 = catalogs.uniform(5000, 3, [1.0, 2.0, 0.5], 7)
    assert np.max(np.abs(u - u32)) <= 2.0 ** -23
    b = catalogs.gaussian_blobs(5000, 4, 1.0, 20, 0.05, 8, fp32=False)
    assert np.all(b >= 0.0) and np.all(b < 1.0)
    assert not np.array_equal(b.astype(np.float32).astype(np.float64), b)
    w = catalogs.normal_weights(1000, 1.0, 0.1, 3, fp32=False)
    assert not np.array_equal(w.astype(np.float32).astype(np.float64), w)
    np.testing.assert_allclose(w, catalogs.normal_weights(1000, 1.0, 0.1, 3), rtol=1e-7)
    wl = catalogs.workload("d3n3_fp64", scale=0.1)
    assert wl.precision == "fp64" and not np.array_equal(wl.pos.astype(np.float32).astype(np.float64), wl.pos)


def test_sphere_directions_fp32_and_unit():
    v = catalogs.sphere_uniform(4000, 5)
    assert np.array_equal(v.astype(np.float32).astype(np.float64), v)
    np.testing.assert_allclose(np.linalg.norm(v, axis=1), 1.0, rtol=1e-6)
    assert np.all(np.abs(v.mean(axis=0)) < 0.05)  # isotropic: no preferred direction
    assert np.array_equal(v, catalogs.sphere_uniform(4000, 5))


def test_named_workloads():
    wl = catalogs.workload("d3n5", scale=0.1)
    assert (wl.D, wl.N, wl.lmax) == (3, 5, 4)
    np.testing.assert_allclose(wl.edges, np.linspace(0.1, 0.4, 11))
    assert np.all(wl.box == 1.0) and wl.n == 1000
    _fp32_in_box(wl.pos, wl.box)
    wl = catalogs.workload("d3n4", scale=0.01)
    assert (wl.D, wl.N, wl.lmax) == (3, 4, 5)
    np.testing.assert_allclose(wl.edges, np.linspace(20.0, 160.0, 11))
    assert set(np.unique(wl.w)) == {-1.0, 1.0}  # data +1, randoms -1
    _fp32_in_box(wl.pos, wl.box)
    wl = catalogs.workload("d4n3", scale=0.05)
    assert (wl.D, wl.N, wl.lmax) == (4, 3, 4)
    np.testing.assert_allclose(wl.edges, np.linspace(0.01, 0.12, 9))


def test_batch_layout():
    bw = catalogs.batch64(ncat=3, scale=0.02)
    assert bw.ncat == 3 and bw.offsets[0] == 0 and bw.offsets[-1] == len(bw.pos)
    assert np.all(np.diff(bw.offsets) > 0)
    assert np.all((bw.boxes >= 500.0) & (bw.boxes <= 1000.0))
    for i in range(bw.ncat):
        p, w, box = bw.catalogue(i)
        _fp32_in_box(p, box)
