"""Pins of the oracle's NPCF of points on the 2-sphere (Sec. "Cosmic Microwave Background").

The D = 2 basis about every primary, with the great-circle angle as radial coordinate, bins in
cos(theta) and 1/(4 pi) in place of 1/V (reading R17).  The pins: separable = naive sum on the
same basis; invariance under rotations of the sphere (and conjugation under a reflection, which
reverses the azimuth); the 3PCF written without any local frame, from the relative azimuth of
two tangent vectors; l = 0 as weighted pair counts from dot products alone; the paper's
35 x 120 components of its 4PCF example.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2106_10278_gb300 import catalogs


def _rotation(seed):
    q, r = np.linalg.qr(np.random.default_rng(seed).normal(size=(3, 3)))
    q = q * np.sign(np.diag(r))
    if np.linalg.det(q) < 0:
        q[:, 0] = -q[:, 0]
    return q


def _cat(n, seed):
    return catalogs.sphere_uniform(n, seed), catalogs.normal_weights(n, 1.0, 0.3, seed + 1)


@pytest.mark.parametrize("N,lmax", [(3, 5), (4, 3)])
def test_sphere_separable_equals_naive_sum(N, lmax):
    pos, w = _cat(60 if N == 3 else 40, 3)
    ce = np.linspace(-0.5, 0.5, 5)
    k1, z1 = oracle.estimate_sphere(N, lmax, ce, pos, w, primaries=(0, 15))
    k2, z2 = oracle.estimate_sphere(N, lmax, ce, pos, w, primaries=(0, 15), brute=True)
    assert np.array_equal(k1, k2)
    scale = np.max(np.abs(z1))
    assert scale > 0 and np.max(np.abs(z1.imag)) > 1e-3 * scale  # odd parts exist
    np.testing.assert_allclose(z1, z2, rtol=0, atol=1e-12 * scale)


@pytest.mark.parametrize("N,lmax", [(3, 5), (4, 3)])
def test_sphere_rotation_invariance_and_reflection(N, lmax):
    """A rotation of the sphere leaves every coefficient unchanged (the local frames turn with
    it); a reflection reverses every azimuth and conjugates the coefficients; the inputs are
    directions, so their length does not matter."""
    pos, w = _cat(50, 5)
    ce = np.linspace(-0.6, 0.4, 6)
    _, z = oracle.estimate_sphere(N, lmax, ce, pos, w)
    scale = np.max(np.abs(z))
    for seed in (1, 2):
        _, zr = oracle.estimate_sphere(N, lmax, ce, pos @ _rotation(seed).T, w)
        np.testing.assert_allclose(zr, z, rtol=0, atol=1e-12 * scale)
    _, zm = oracle.estimate_sphere(N, lmax, ce, pos * np.array([1.0, -1.0, 1.0]), w)
    np.testing.assert_allclose(zm, z.conj(), rtol=0, atol=1e-12 * scale)
    _, zs = oracle.estimate_sphere(N, lmax, ce, 2.5 * pos, w)
    np.testing.assert_allclose(zs, z, rtol=0, atol=1e-12 * scale)


def _neighbours(pos, j, ce):
    u = pos / np.linalg.norm(pos, axis=1, keepdims=True)
    c = u @ u[j]
    b = np.searchsorted(ce, c, side="right") - 1
    ok = (np.arange(len(u)) != j) & (b >= 0) & (b < len(ce) - 1)
    return u, c, b, ok


def test_sphere_3pcf_frame_free_closed_form():
    """zeta_l(b1, b2) = (1/4pi) sum_j w_j sum_{k in b1, k' in b2} w_k w_k' e^{-il(phi_k - phi_k')}
    / (2 pi v1 v2), with the relative azimuth from the tangent vectors t = n_k - (n_j.n_k) n_j:
    cos = t.t'/(|t||t'|), sin = n_j.(t' x t)/(|t||t'|) (counter-clockwise seen from outside)."""
    pos, w = _cat(70, 9)
    ce = np.linspace(-0.5, 0.5, 4)
    lmax = 5
    keys, z = oracle.estimate_sphere(3, lmax, ce, pos, w)
    vb = 2 * np.pi * np.diff(ce)
    index = {(k[0], k[1], k[3]): i for i, k in enumerate(keys)}
    ref = np.zeros(len(keys), complex)
    for j in range(len(pos)):
        u, c, b, ok = _neighbours(pos, j, ce)
        t = u[ok] - c[ok, None] * u[j]
        t /= np.linalg.norm(t, axis=1, keepdims=True)
        cosd = t @ t.T
        sind = np.einsum("a,kpa->kp", u[j], np.cross(t[None, :, :], t[:, None, :]))
        delta = np.arctan2(sind, cosd)  # phi_k - phi_k'
        bb, ww = b[ok], w[ok]
        for b1 in range(3):
            for b2 in range(b1, 3):
                m = np.outer((bb == b1) * ww, (bb == b2) * ww)
                for l in range(lmax + 1):
                    ref[index[(b1, b2, l)]] += w[j] * np.sum(m * np.exp(-1j * l * delta)) / (2 * np.pi * vb[b1] * vb[b2])
    ref /= 4 * np.pi
    np.testing.assert_allclose(z, ref, rtol=0, atol=1e-12 * np.max(np.abs(ref)))


def test_sphere_l0_weighted_pair_counts():
    """l = 0 needs no azimuth: zeta_0(b1, b2) = (1/4pi) sum_j w_j W_j(b1) W_j(b2) / (2 pi v1 v2),
    W_j(b) the weight in the annulus c_b <= n_j.n_k < c_{b+1}, v_b = 2 pi (c_{b+1} - c_b)."""
    pos, w = _cat(80, 13)
    ce = np.array([-0.7, -0.2, 0.1, 0.55, 0.9])
    keys, z = oracle.estimate_sphere(3, 2, ce, pos, w)
    vb = 2 * np.pi * np.diff(ce)
    W = np.zeros((len(pos), 4))
    for j in range(len(pos)):
        _, _, b, ok = _neighbours(pos, j, ce)
        for bb in range(4):
            W[j, bb] = np.sum(w[ok & (b == bb)])
    for k, v in zip(keys, z):
        if k[3] != 0:
            continue
        ref = np.sum(w * W[:, k[0]] * W[:, k[1]]) / (4 * np.pi * 2 * np.pi * vb[k[0]] * vb[k[1]])
        assert abs(v - ref) <= 1e-12 * max(1.0, abs(ref))


def test_sphere_coinciding_directions_are_skipped():
    """Duplicated directions (and a rescaled copy, the same direction) are no pair -- they have no
    azimuth, as r = 0 has no direction in a box -- while every other pair up to cos theta = 1
    counts: the l = 0 weighted pair counts from dot products, with identical unit vectors left
    out, give zeta_0 again."""
    pos, w = _cat(60, 21)
    pos = np.concatenate([pos, pos[:10], 3.0 * pos[10:15]])
    w = catalogs.normal_weights(len(pos), 1.0, 0.3, 22)
    ce = np.array([-0.3, 0.2, 0.7, 1.0])
    keys, z = oracle.estimate_sphere(3, 2, ce, pos, w)
    assert np.all(np.isfinite(z))
    u = pos / np.linalg.norm(pos, axis=1, keepdims=True)
    vb = 2 * np.pi * np.diff(ce)
    W = np.zeros((len(pos), 3))
    for j in range(len(pos)):
        c = u @ u[j]
        b = np.searchsorted(ce, c, side="right") - 1
        same = np.all(np.isclose(u, u[j], rtol=0, atol=1e-15), axis=1)
        ok = ~same & (b >= 0) & (b < 3)
        for bb in range(3):
            W[j, bb] = np.sum(w[ok & (b == bb)])
    for k, v in zip(keys, z):
        if k[3] != 0:
            continue
        ref = np.sum(w * W[:, k[0]] * W[:, k[1]]) / (4 * np.pi * 2 * np.pi * vb[k[0]] * vb[k[1]])
        assert abs(v - ref) <= 1e-12 * max(1.0, abs(ref))


def test_sphere_4pcf_paper_example_component_counts():
    """The paper's 2-sphere example: 4PCF, ten bins over cos(theta) in [-0.5, 0.5), lmax = 4 ->
    35 angular and 120 radial components."""
    pos, w = _cat(30, 17)
    keys, z = oracle.estimate_sphere(4, 4, np.linspace(-0.5, 0.5, 11), pos, w, primaries=(0, 2))
    assert len({tuple(k[:3]) for k in keys}) == 120
    assert len({tuple(k[3:]) for k in keys}) == 35
    assert len(z) == 120 * 35


def test_sphere_rejects_undefined_azimuth_and_bad_edges():
    pos, w = _cat(10, 19)
    with pytest.raises(ValueError):
        oracle.estimate_sphere(3, 2, np.array([-1.0, 0.0, 0.5]), pos, w)  # antipodes: azimuth undefined
    with pytest.raises(ValueError):
        oracle.estimate_sphere(3, 2, np.array([0.0, 0.5, 1.2]), pos, w)
    with pytest.raises(ValueError):
        oracle.estimate_sphere(3, 2, np.array([0.5, 0.0]), pos, w)
    with pytest.raises(ValueError):
        oracle.estimate_sphere(5, 2, np.linspace(-0.5, 0.5, 6), pos, w)
    assert math.isclose(np.linalg.norm(pos[0]), 1.0, rel_tol=1e-6)
