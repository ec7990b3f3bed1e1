"""Pins of the oracle's anisotropic basis about the x_3 line of sight (Sec. "Large-Scale
Structure", reading R18): the states of combined angular momentum (0, L) in D = 3.

The pins: separable = naive sum on the same basis; the L = 0 slice is the isotropic NPCF; closed
forms of the basis written with numpy and scipy only (l2 = 0: Legendre multipoles of the
line-of-sight cosine; l1 = l2 = 1: dot, cross and zz products); invariance under rotations about
x_3 (and not about x_1 once L > 0); the parities of reflections of x_3 and of x_2.
"""
import math

import numpy as np
import pytest
from scipy.special import eval_legendre

import oracle
from paper_2106_10278_gb300 import catalogs


def _cat(n, seed):
    return catalogs.uniform(n, 3, 1.0, seed), catalogs.normal_weights(n, 1.0, 0.3, seed + 1)


def test_aniso_key_counts():
    """N=3: every (l1, l2) <= lmax with L from |l1 - l2| to l1 + l2; N=4: l12 and L likewise."""
    lmax, nb = 3, 4
    per3 = sum(2 * min(a, b) + 1 for a in range(lmax + 1) for b in range(lmax + 1))
    assert len(oracle.aniso_keys(3, lmax, nb)) == nb * (nb + 1) // 2 * per3
    assert len(oracle.aniso_keys(3, lmax, nb, bin_lt=True)) == nb * (nb - 1) // 2 * per3
    per4 = sum(2 * min(l12, c) + 1 for a in range(3) for b in range(3) for l12 in range(abs(a - b), a + b + 1)
               for c in range(3))
    assert len(oracle.aniso_keys(4, 2, nb)) == math.comb(nb, 3) * per4


@pytest.mark.parametrize("N,lmax", [(3, 3), (4, 2)])
def test_aniso_separable_equals_naive_sum(N, lmax):
    pos, w = _cat(45 if N == 3 else 30, 3)
    edges = np.linspace(0.05, 0.45, 5 if N == 4 else 4)
    k1, z1 = oracle.estimate_aniso(N, lmax, edges, 1.0, pos, w, primaries=(0, 12))
    k2, z2 = oracle.estimate_aniso(N, lmax, edges, 1.0, pos, w, primaries=(0, 12), brute=True)
    assert np.array_equal(k1, k2)
    scale = np.max(np.abs(z1))
    assert scale > 0
    np.testing.assert_allclose(z1, z2, rtol=0, atol=1e-12 * scale)


def test_aniso_l0_slice_is_the_isotropic_npcf():
    """L = 0 forces l1 = l2 (N=3) or l12 = l3 (N=4), where <.. ..|0 0> is the isotropic coupling."""
    pos, w = _cat(50, 7)
    edges = np.linspace(0.05, 0.45, 5)
    ka, za = oracle.estimate_aniso(3, 3, edges, 1.0, pos, w)
    ki, zi = oracle.estimate(3, 3, 3, edges, np.ones(3), pos, w)
    iso = {(k[0], k[1], k[3]): v for k, v in zip(ki, zi)}
    scale = np.max(np.abs(zi))
    n3 = 0
    for k, v in zip(ka, za):
        if k[5] == 0:
            assert k[3] == k[4]
            assert abs(v - iso[(k[0], k[1], k[3])]) <= 1e-12 * scale
            n3 += 1
    assert n3 == len(zi)
    ka, za = oracle.estimate_aniso(4, 2, edges, 1.0, pos, w, primaries=(0, 15))
    ki, zi = oracle.estimate(3, 4, 2, edges, np.ones(3), pos, w, primaries=(0, 15))
    iso = {(k[0], k[1], k[2], k[3], k[4], k[5]): v for k, v in zip(ki, zi)}
    scale = np.max(np.abs(zi))
    n4 = 0
    for k, v in zip(ka, za):
        if k[7] == 0:
            assert k[5] == k[6]
            assert abs(v - iso[(k[0], k[1], k[2], k[3], k[4], k[6])]) <= 1e-12 * scale
            n4 += 1
    assert n4 == len(zi)


def test_aniso_3pcf_closed_forms():
    """With Condon-Shortley Y_1m written out (the (-1)^m of another phase convention cancels as
    m1 + m2 = 0), the basis P^{0L}_{l1 l2}(a, b) of the redshift-space 3PCF is
      l1 = l2 = 1:  L=0: -sqrt(3)/(4pi) a.b;  L=1: 3i/(4pi sqrt 2) (a x b)_3;
                    L=2: 3/(4pi sqrt 6) (3 a_3 b_3 - a.b);
      l2 = 0 (L = l1), or l1 = 0 (L = l2): sqrt(2L+1)/(4pi) P_L(cos) of the line-of-sight cosine;
    zeta = (1/V) sum_j w_j sum_{k in b1, k' in b2} w_k w_k' conj(P(u_k, u_k')) / (v1 v2)."""
    pos, w = _cat(70, 21)
    edges = np.linspace(0.08, 0.45, 4)
    nb, lmax = 3, 3
    keys, z = oracle.estimate_aniso(3, lmax, edges, 1.0, pos, w)
    vb = 4 * np.pi / 3 * (edges[1:] ** 3 - edges[:-1] ** 3)
    index = {(k[0], k[1], k[3], k[4], k[5]): i for i, k in enumerate(keys)}
    ref = {}
    for j in range(len(pos)):
        d = pos - pos[j]
        d -= np.round(d)
        r = np.linalg.norm(d, axis=1)
        b = np.searchsorted(edges, r, side="right") - 1
        ok = (np.arange(len(pos)) != j) & (b >= 0) & (b < nb)
        u, bb, ww = d[ok] / r[ok, None], b[ok], w[ok]
        dot = u @ u.T
        cz = np.cross(u[:, None, :], u[None, :, :])[..., 2]
        P = {0: -math.sqrt(3) / (4 * np.pi) * dot, 1: 3j / (4 * np.pi * math.sqrt(2)) * cz,
             2: 3 / (4 * np.pi * math.sqrt(6)) * (3 * np.outer(u[:, 2], u[:, 2]) - dot)}
        for b1 in range(nb):
            for b2 in range(b1, nb):
                m = np.outer((bb == b1) * ww, (bb == b2) * ww) / (vb[b1] * vb[b2])
                for L in range(3):
                    key = (b1, b2, 1, 1, L)
                    ref[key] = ref.get(key, 0) + w[j] * np.sum(m * np.conj(P[L]))
                W1, W2 = np.sum((bb == b1) * ww) / vb[b1], np.sum((bb == b2) * ww) / vb[b2]
                for L in range(1, lmax + 1):
                    c = math.sqrt(2 * L + 1) / (4 * np.pi)
                    f1 = np.sum((bb == b1) * ww * eval_legendre(L, u[:, 2])) / vb[b1]
                    f2 = np.sum((bb == b2) * ww * eval_legendre(L, u[:, 2])) / vb[b2]
                    for key, val in (((b1, b2, L, 0, L), c * f1 * W2), ((b1, b2, 0, L, L), c * W1 * f2)):
                        ref[key] = ref.get(key, 0) + w[j] * val
    scale = np.max(np.abs(z))
    assert len(ref) == 6 * (3 + 2 * lmax)
    for key, v in ref.items():
        assert abs(z[index[key]] - v) <= 1e-12 * scale, key
    assert max(abs(v.imag) for k, v in ref.items() if k[2:] == (1, 1, 1)) > 1e-6 * scale


def _rot(axis, t):
    c, s = math.cos(t), math.sin(t)
    i, j = [(1, 2), (2, 0), (0, 1)][axis]
    R = np.eye(3)
    R[i, i], R[i, j], R[j, i], R[j, j] = c, -s, s, c
    return R


@pytest.mark.parametrize("N,lmax", [(3, 3), (4, 2)])
def test_aniso_line_of_sight_symmetries(N, lmax):
    """Open boundaries: a rotation about x_3 changes nothing; one about x_1 keeps the L = 0 part and
    changes the rest; x_3 -> -x_3 multiplies by (-1)^{l1+l2(+l3)}; x_2 -> -x_2 conjugates."""
    pos, w = _cat(40, 31)
    pos = pos - 0.5
    edges = np.linspace(0.05, 0.4, 5 if N == 4 else 4)
    keys, z = oracle.estimate_aniso(N, lmax, edges, 1.0, pos, w, periodic=False)
    scale = np.max(np.abs(z))
    Lcol = 5 if N == 3 else 7
    lsum = keys[:, 3] + keys[:, 4] + (keys[:, 6] if N == 4 else 0)
    _, zr = oracle.estimate_aniso(N, lmax, edges, 1.0, pos @ _rot(2, 0.7).T, w, periodic=False)
    np.testing.assert_allclose(zr, z, rtol=0, atol=1e-11 * scale)
    _, zx = oracle.estimate_aniso(N, lmax, edges, 1.0, pos @ _rot(0, 0.7).T, w, periodic=False)
    iso = keys[:, Lcol] == 0
    np.testing.assert_allclose(zx[iso], z[iso], rtol=0, atol=1e-11 * scale)
    assert np.max(np.abs(zx[~iso] - z[~iso])) > 1e-3 * scale
    _, zm = oracle.estimate_aniso(N, lmax, edges, 1.0, pos * np.array([1.0, 1.0, -1.0]), w, periodic=False)
    np.testing.assert_allclose(zm, np.where(lsum % 2 == 0, 1.0, -1.0) * z, rtol=0, atol=1e-11 * scale)
    _, zy = oracle.estimate_aniso(N, lmax, edges, 1.0, pos * np.array([1.0, -1.0, 1.0]), w, periodic=False)
    np.testing.assert_allclose(zy, z.conj(), rtol=0, atol=1e-11 * scale)
