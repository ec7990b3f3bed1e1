"""Pins of the oracle's gridded-data estimator (Sec. "Application to Gridded Data").

The oracle evaluates the plain definition, a direct sum over node offsets.  Two pins tie it to
things outside itself:
  * a particle catalogue deposited on the grid by nearest grid point (NGP) gives exactly the
    discrete estimator (eq. NPCF-estimator-discrete) of the same particles moved to their cell
    centres, which the discrete pins in test_oracle_pins.py tie to closed forms and the naive sum;
  * the paper's FFT form of a^b_l, written here with numpy's FFT, reproduces the direct sum, with
    the kernel read as Y*_l Theta^b (reading R16) -- the kernel as printed, Y_l Theta^b, does not.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2106_10278_gb300 import catalogs

AREA = {2: 2 * np.pi, 3: 4 * np.pi, 4: 2 * np.pi ** 2}


def _ngp(pos, w, M, L):
    D = pos.shape[1]
    h = L / M
    c = np.floor(pos / h).astype(np.int64) % M
    X = np.zeros((M,) * D)
    np.add.at(X, tuple(c.T), w / h ** D)
    return X, (c + 0.5) * h


GRID_CASES = [
    # D, N, lmax, M, n, edges
    (2, 3, 6, 32, 300, [0.07, 0.13, 0.2, 0.27, 0.33]),
    (3, 3, 4, 16, 300, [0.07, 0.13, 0.2, 0.27, 0.33]),
    (4, 3, 3, 8, 200, [0.13, 0.2, 0.3, 0.37]),
    (2, 4, 3, 24, 200, [0.07, 0.13, 0.2, 0.27, 0.33]),
    (3, 4, 2, 12, 200, [0.07, 0.13, 0.2, 0.27, 0.33]),
    (3, 5, 2, 10, 150, [0.09, 0.15, 0.22, 0.29, 0.36, 0.42]),
]


@pytest.mark.parametrize("D,N,lmax,M,n,edges", GRID_CASES)
def test_grid_ngp_deposit_equals_discrete_at_cell_centres(D, N, lmax, M, n, edges):
    """With X = sum_k w_k delta(cell of k)/dV, the node sums of the gridded estimator are the
    particle sums of the discrete one at the cell centres (two particles in one cell are at
    r = 0 on both sides and skipped on both)."""
    edges = np.asarray(edges)
    pos = catalogs.uniform(n, D, 1.0, 200 + 10 * D + N)
    w = catalogs.normal_weights(n, 1.0, 0.3, 300 + D + N)
    X, centres = _ngp(pos, w, M, 1.0)
    kg, zg = oracle.estimate_grid(N, lmax, edges, 1.0, X)
    kd, zd = oracle.estimate(D, N, lmax, edges, np.ones(D), centres, w)
    assert np.array_equal(kg, kd)
    scale = np.max(np.abs(zd))
    assert scale > 0
    np.testing.assert_allclose(zg, zd, rtol=0, atol=1e-12 * scale)


@pytest.mark.parametrize("D,M,lmax", [(2, 24, 6), (3, 12, 4), (4, 8, 3)])
def test_grid_alm_equals_paper_fft_form(D, M, lmax):
    """a^b_l = (-1)^{l_{D-1}} FFT^{-1}[FFT(X) FFT(K)] with K(o h) = dV Y*_l(unit(o)) Theta^b(|o h|)/v_b
    at node o mod M, for a Gaussian random field on the grid; the offsets and bins are built here
    with numpy."""
    h = 1.0 / M
    X = np.random.default_rng(1).normal(size=(M,) * D)
    edges = np.array([0.09, 0.17, 0.26, 0.37]) if D < 4 else np.array([0.13, 0.2, 0.3, 0.37])
    A = oracle.grid_alm(lmax, edges, 1.0, X)
    st = oracle.states(D, lmax)
    sign = np.where(st[:, D - 2] % 2 == 0, 1.0, -1.0)
    vb = AREA[D] / D * (edges[1:] ** D - edges[:-1] ** D)
    K = int(np.floor(edges[-1] / h))
    o = np.stack(np.meshgrid(*[np.arange(-K, K + 1)] * D, indexing="ij"), -1).reshape(-1, D)
    r = np.linalg.norm(o * h, axis=1)
    b = np.searchsorted(edges, r, side="right") - 1
    ok = (r > 0) & (b >= 0) & (b < len(vb))
    o, b = o[ok], b[ok]
    Y = oracle.harmonics(D, lmax, o * h)
    FX = np.fft.fftn(X)
    scale = np.max(np.abs(A))
    literal_err = 0.0
    for bb in range(len(vb)):
        sel = b == bb
        for s in range(len(st)):
            for conj in (True, False):
                ker = np.zeros((M,) * D, complex)
                vals = (np.conj(Y[sel, s]) if conj else Y[sel, s]) * h ** D / vb[bb]
                np.add.at(ker, tuple((o[sel] % M).T), vals)
                a = sign[s] * np.fft.ifftn(FX * np.fft.fftn(ker)).reshape(-1)
                if conj:
                    np.testing.assert_allclose(a, A[:, bb, s], rtol=0, atol=1e-12 * scale)
                else:
                    literal_err = max(literal_err, np.max(np.abs(a - A[:, bb, s])))
    assert literal_err > 0.1 * scale


def test_grid_l0_is_shell_average():
    """a^b_0 needs no harmonic: Y_0 = 1/sqrt(|S^{D-1}|), so a^b_0(s) is dV/(v_b sqrt|S|) times the sum
    of X over the nodes in the shell around s (numpy below)."""
    D, M = 3, 12
    h = 1.0 / M
    X = np.random.default_rng(2).normal(size=(M,) * D)
    edges = np.array([0.1, 0.2, 0.3])
    A = oracle.grid_alm(2, edges, 1.0, X)
    vb = AREA[D] / D * (edges[1:] ** D - edges[:-1] ** D)
    K = int(np.floor(edges[-1] / h))
    ref = np.zeros((M ** D, 2))
    for o in np.stack(np.meshgrid(*[np.arange(-K, K + 1)] * D, indexing="ij"), -1).reshape(-1, D):
        r = np.linalg.norm(o * h)
        bb = np.searchsorted(edges, r, side="right") - 1
        if r == 0 or bb < 0 or bb >= 2:
            continue
        ref[:, bb] += np.roll(X, shift=tuple(-o), axis=tuple(range(D))).reshape(-1)
    ref *= h ** D / (vb * math.sqrt(AREA[D]))
    np.testing.assert_allclose(A[:, :, 0].real, ref, rtol=0, atol=1e-13)
    assert np.max(np.abs(A[:, :, 0].imag)) < 1e-15


def test_grid_rejects_offsets_that_alias():
    """Every offset within r_max must reach a distinct node (2 floor(r_max/h) < M)."""
    X = np.zeros((8, 8, 8))
    with pytest.raises(ValueError):
        oracle.grid_alm(2, np.array([0.1, 0.5]), 1.0, X)
    with pytest.raises(ValueError):
        oracle.estimate_grid(3, 2, np.array([0.1, 0.5]), 1.0, X)


def test_grid_constant_field_shell_counts():
    """A constant field X: a^b_00 = X dV (nodes in shell b, offset 0 excluded) / (v_b sqrt(4 pi)),
    every node alike, so the l = 0 coefficient of the 3PCF is X a^0_00 a^1_00 (the node sum of
    dV X is X V); the shell's nodes are counted here by brute force."""
    edges = np.array([0.1, 0.2, 0.3])
    X = np.full((20, 20, 20), 1.5)
    keys, z = oracle.estimate_grid(3, 2, edges, np.ones(3), X)
    h = 1.0 / 20
    o = np.arange(-6, 7)
    r2 = (o[:, None, None] ** 2 + o[None, :, None] ** 2 + o[None, None, :] ** 2) * h * h
    cnt = [np.count_nonzero((r2 >= edges[b] ** 2) & (r2 < edges[b + 1] ** 2) & (r2 > 0)) for b in range(2)]
    vb = [4 * np.pi / 3 * (edges[b + 1] ** 3 - edges[b] ** 3) for b in range(2)]
    a0 = [1.5 * h ** 3 * cnt[b] / vb[b] / np.sqrt(4 * np.pi) for b in range(2)]
    i = [j for j in range(len(keys)) if keys[j][0] == 0 and keys[j][1] == 1 and all(x == 0 for x in keys[j][3:])]
    assert len(i) == 1
    expect = 1.5 * a0[0] * a0[1]
    assert abs(z[i[0]] - expect) <= 1e-13 * abs(expect)
