"""Pins of the FP64 oracle against facts fixed by the paper and by mathematics.

None of these checks re-types an oracle formula: each compares the oracle with
an independent library (scipy, sympy, mpmath), a closed form, an identity, a
brute-force definition or a count printed in the paper.
"""
import json
import math
import os

import numpy as np
import pytest

import oracle
from paper_2106_10278_gb300 import catalogs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _rand_dirs(D, n, seed):
    g = np.random.default_rng(seed)
    d = g.normal(size=(n, D))
    return d * g.uniform(0.3, 3.0, size=(n, 1))


# ---------------------------------------------------------------- harmonics
def test_harmonics_d3_match_scipy_up_to_phase():
    """eq. hypersph-def in D=3 is the spherical harmonic; scipy gives the
    Condon-Shortley Y.  With DLMF's Ferrers functions the paper's Y_{m l}
    equals (-1)^m Y^CS_{lm} (a phase that cancels in every L=0 component)."""
    from scipy.special import sph_harm_y

    d = _rand_dirs(3, 50, 1)
    Y = oracle.harmonics(3, 6, d)
    st = oracle.states(3, 6)
    r = np.linalg.norm(d, axis=1)
    theta = np.arccos(d[:, 2] / r)
    phi = np.arctan2(d[:, 1], d[:, 0])
    for i, (m, l, _) in enumerate(st):
        ref = (-1.0) ** m * sph_harm_y(l, m, theta, phi)
        np.testing.assert_allclose(Y[:, i], ref, rtol=0, atol=1e-12)


def test_ferrers_half_matches_mpmath():
    """The half-odd Ferrers functions behind the D=4 harmonic (eq. hypersph-def, K=3)."""
    mpmath = pytest.importorskip("mpmath")
    for L in range(0, 7):
        for k in range(0, L + 1):
            for th in (0.2, 0.9, 1.7, 2.9):
                ref = float(mpmath.legenp(L + 0.5, -(k + 0.5), mpmath.cos(th), type=2))
                got = oracle.ferrers_half(L, k, th)
                assert abs(got - ref) <= 1e-11 * max(1.0, abs(ref)), (L, k, th, got, ref)


def test_ferrers_int_matches_mpmath():
    mpmath = pytest.importorskip("mpmath")
    for n in range(0, 8):
        for mu in range(-n, n + 1):
            for x in (-0.83, -0.1, 0.37, 0.95):
                ref = float(mpmath.legenp(n, mu, x, type=2))
                assert abs(oracle.ferrers_int(n, mu, x) - ref) <= 1e-11 * max(1.0, abs(ref))


def _sphere_quadrature(D, n1=48, n2=40, n3=40):
    """Product quadrature on S^{D-1} in hyperspherical angles (reading R5)."""
    t1 = np.arange(n1) * 2 * np.pi / n1
    w1 = np.full(n1, 2 * np.pi / n1)
    if D == 2:
        return np.stack([np.cos(t1), np.sin(t1)], 1), w1
    x2, w2 = np.polynomial.legendre.leggauss(n2)  # cos(theta_2), measure sin(theta_2) d theta_2
    s2 = np.sqrt(1 - x2 ** 2)
    if D == 3:
        T1, X2 = np.meshgrid(t1, x2, indexing="ij")
        S2 = np.sqrt(1 - X2 ** 2)
        pts = np.stack([S2 * np.cos(T1), S2 * np.sin(T1), X2], -1).reshape(-1, 3)
        return pts, (w1[:, None] * w2[None, :]).ravel()
    # D=4: theta_3 in (0, pi) with measure sin^2(theta_3); Gauss-Legendre in theta_3
    u, wu = np.polynomial.legendre.leggauss(n3)
    t3 = (u + 1) * np.pi / 2
    w3 = wu * np.pi / 2 * np.sin(t3) ** 2
    T1, X2, T3 = np.meshgrid(t1, x2, t3, indexing="ij")
    S2 = np.sqrt(1 - X2 ** 2)
    S3 = np.sin(T3)
    pts = np.stack([S3 * S2 * np.cos(T1), S3 * S2 * np.sin(T1), S3 * X2, np.cos(T3)], -1).reshape(-1, 4)
    W = (w1[:, None, None] * w2[None, :, None] * w3[None, None, :]).ravel()
    return pts, W


@pytest.mark.parametrize("D,lmax", [(2, 6), (3, 5), (4, 4)])
def test_harmonics_orthonormal(D, lmax):
    """Orthonormality of the hyperspherical harmonics on S^{D-1} (the inner product after eq. single-particle-eigenfun)."""
    pts, W = _sphere_quadrature(D)
    Y = oracle.harmonics(D, lmax, pts)
    G = (Y.conj() * W[:, None]).T @ Y
    np.testing.assert_allclose(G, np.eye(Y.shape[1]), atol=1e-11)


@pytest.mark.parametrize("D,lmax", [(3, 6), (4, 5)])
def test_harmonics_addition_theorem(D, lmax):
    """sum over intermediate labels of Y(u) Y*(v) = dim_l/|S^{D-1}| C^{(D/2-1)}_l(u.v)/C_l(1);
    dim_l is the state count quoted with eq. single-particle-eigenfun."""
    from scipy.special import eval_gegenbauer

    u = _rand_dirs(D, 30, 2)
    v = _rand_dirs(D, 30, 3)
    Yu = oracle.harmonics(D, lmax, u)
    Yv = oracle.harmonics(D, lmax, v)
    st = oracle.states(D, lmax)
    tot = st[:, D - 2]
    uu = u / np.linalg.norm(u, axis=1, keepdims=True)
    vv = v / np.linalg.norm(v, axis=1, keepdims=True)
    t = np.sum(uu * vv, axis=1)
    lam = D / 2 - 1
    area = 2 * np.pi ** (D / 2) / math.gamma(D / 2)
    for l in range(lmax + 1):
        sel = tot == l
        s = np.sum(Yu[:, sel] * Yv[:, sel].conj(), axis=1)
        dim = math.comb(l + D - 3, D - 3) * (2 * l + D - 2) / (D - 2)
        ref = dim / area * eval_gegenbauer(l, lam, t) / eval_gegenbauer(l, lam, 1.0)
        np.testing.assert_allclose(s, ref, atol=1e-12)
        assert dim == np.count_nonzero(sel)


@pytest.mark.parametrize("D", [3, 4])
def test_harmonics_continuous_at_axis_directions(D):
    """Grid offsets hit the axes, where an angle of eq. hypersph-def is undefined or a factor
    is 0 x infinity: the values there are finite and are the limits of nearby directions."""
    lmax = 5
    axes = np.vstack([np.eye(D), -np.eye(D), np.eye(D)[[0]] + np.eye(D)[[D - 1]]] +
                     ([np.array([[0.0, 0.0, 2.0, 3.0], [0.0, 0.0, -1.0, -2.0]])] if D == 4 else []))
    Y = oracle.harmonics(D, lmax, axes)
    assert np.all(np.isfinite(Y))
    g = np.random.default_rng(0)
    for eps in (1e-7, 1e-9):
        for _ in range(10):
            near = oracle.harmonics(D, lmax, axes + eps * g.normal(size=axes.shape))
            assert np.max(np.abs(near - Y)) < 100 * eps


def _rotate_plane(x, a, b, t):
    y = x.copy()
    c, s = math.cos(t), math.sin(t)
    y[:, a] = c * x[:, a] - s * x[:, b]
    y[:, b] = s * x[:, a] + c * x[:, b]
    return y


@pytest.mark.parametrize("D,lmax", [(2, 6), (3, 5), (4, 4)])
def test_harmonics_casimir_eigenvalues_of_every_label(D, lmax):
    """Every label of the chain is an eigenvalue label: the Laplacian of the sub-sphere S^K
    spanned by coordinates 1..K+1, written as the sum of squared rotation generators L_ab,
    a < b <= K+1, has Y as eigenfunction with eigenvalue -l_K (l_K + K - 1) (-l_1^2 for K = 1).
    For K = D-1 this is the Casimir of eq. single-particle-eigenfun.  The second derivatives along
    exact plane rotations are central differences with one Richardson step."""
    x = np.random.default_rng(5).normal(size=(25, D))
    Y = oracle.harmonics(D, lmax, x)
    st = oracle.states(D, lmax)

    def casimir(K, h):
        acc = np.zeros_like(Y)
        for b in range(1, K + 1):
            for a in range(b):
                acc += (oracle.harmonics(D, lmax, _rotate_plane(x, a, b, h)) - 2 * Y
                        + oracle.harmonics(D, lmax, _rotate_plane(x, a, b, -h))) / h ** 2
        return acc

    h = 2e-2
    for K in range(1, D):
        lK = st[:, K - 1].astype(np.float64)
        eig = -(lK * (lK + K - 1))
        got = (4 * casimir(K, h / 2) - casimir(K, h)) / 3
        np.testing.assert_allclose(got, eig[None, :] * Y, rtol=0, atol=2e-5)


def test_harmonics_conjugation_and_parity():
    """eq. complex-conj-hypersph: Y* = (-1)^{l_1} Y_{-l_1...} (D>=3) and P[Y] = (-1)^{l_{D-1}} Y."""
    for D, lmax in [(3, 5), (4, 4)]:
        d = _rand_dirs(D, 20, 5)
        Y = oracle.harmonics(D, lmax, d)
        Ym = oracle.harmonics(D, lmax, -d)
        st = [tuple(s) for s in oracle.states(D, lmax)]
        for i, s in enumerate(st):
            j = st.index((-s[0],) + s[1:])
            np.testing.assert_allclose(Y[:, i].conj(), (-1.0) ** s[0] * Y[:, j], atol=1e-12)
            np.testing.assert_allclose(Ym[:, i], (-1.0) ** s[D - 2] * Y[:, i], atol=1e-12)


# ------------------------------------------------------------ 3j / coupling
def test_wigner3j_matches_sympy():
    from sympy.physics.wigner import wigner_3j

    for j1 in range(0, 5):
        for j2 in range(0, 5):
            for j3 in range(abs(j1 - j2), j1 + j2 + 1):
                for m1 in range(-j1, j1 + 1):
                    for m2 in range(-j2, j2 + 1):
                        m3 = -m1 - m2
                        if abs(m3) > j3:
                            continue
                        ref = float(wigner_3j(j1, j2, j3, m1, m2, m3))
                        assert abs(oracle.wigner3j(j1, j2, j3, m1, m2, m3) - ref) < 1e-13


def test_cg_orthonormality_and_zero_coupling():
    """eq. CG-orthonorm for D=3, and <l m, l -m | 0 0> = (-1)^{l-m}/sqrt(2l+1) (DLMF 34.3.1)."""
    for l1 in range(0, 4):
        for l2 in range(0, 4):
            for L in range(abs(l1 - l2), l1 + l2 + 1):
                for Lp in range(abs(l1 - l2), l1 + l2 + 1):
                    for M in range(-L, L + 1):
                        for Mp in range(-Lp, Lp + 1):
                            s = sum(oracle.cg_d3(l1, m1, l2, m2, L, M) * oracle.cg_d3(l1, m1, l2, m2, Lp, Mp)
                                    for m1 in range(-l1, l1 + 1) for m2 in range(-l2, l2 + 1))
                            assert abs(s - (1.0 if (L == Lp and M == Mp) else 0.0)) < 1e-12
    for l in range(0, 8):
        for m in range(-l, l + 1):
            assert abs(oracle.cg_d3(l, m, l, -m, 0, 0) - (-1) ** (l - m) / math.sqrt(2 * l + 1)) < 1e-14


def test_d3_n4_coupling_is_signed_3j():
    """C^{Lambda;0} of eq. Coupling-C for D=3, N=4 equals (-1)^{l1+l2+l3} (l1 l2 l3; m1 m2 m3)
    (sympy's 3j, an independent evaluation)."""
    from sympy.physics.wigner import wigner_3j

    lmax = 3
    st = [tuple(s) for s in oracle.states(3, lmax)]
    keys = oracle.keys(3, 4, lmax, 3)
    lams = []
    for k in keys[:, 3:]:
        if tuple(k) not in lams:
            lams.append(tuple(k))
    for il, (l1, l2, l3) in enumerate(lams):
        s, c = oracle.coupling_terms(3, 4, lmax, il)
        got = {(st[a][0], st[b][0], st[e][0]): cc for (a, b, e), cc in zip(s, c)}
        for m1 in range(-l1, l1 + 1):
            for m2 in range(-l2, l2 + 1):
                m3 = -m1 - m2
                if abs(m3) > l3:
                    continue
                ref = (-1) ** (l1 + l2 + l3) * float(wigner_3j(l1, l2, l3, m1, m2, m3))
                assert abs(got.get((m1, m2, m3), 0.0) - ref) < 1e-13


def _random_rotation(D, seed):
    g = np.random.default_rng(seed)
    q, r = np.linalg.qr(g.normal(size=(D, D)))
    q *= np.sign(np.diag(r))
    if np.linalg.det(q) < 0:
        q[:, 0] *= -1
    return q


def test_isotropic_basis_rotation_invariant_d3_n4():
    """P^0_Lambda (eq. N-1-particle-basis-wavefunction with L=0) is invariant under a joint rotation."""
    lmax = 3
    R = _random_rotation(3, 9)
    r1, r2, r3 = (_rand_dirs(3, 10, s) for s in (11, 12, 13))
    keys = oracle.keys(3, 4, lmax, 3)
    nl = len({tuple(k) for k in keys[:, 3:]})
    Y = [oracle.harmonics(3, lmax, r) for r in (r1, r2, r3)]
    YR = [oracle.harmonics(3, lmax, r @ R.T) for r in (r1, r2, r3)]
    for il in range(nl):
        s, c = oracle.coupling_terms(3, 4, lmax, il)
        P = sum(cc * Y[0][:, a] * Y[1][:, b] * Y[2][:, e] for (a, b, e), cc in zip(s, c))
        PR = sum(cc * YR[0][:, a] * YR[1][:, b] * YR[2][:, e] for (a, b, e), cc in zip(s, c))
        np.testing.assert_allclose(P, PR, atol=1e-12)


# ------------------------------------------------------------------ counts
@pytest.mark.parametrize("name", ["d2_4pcf_lmax4", "d3_5pcf_lmax4"])
def test_component_counts_printed_in_paper(name):
    g = json.load(open(os.path.join(GOLDEN, "paper_counts.json")))[name]
    k = oracle.keys(g["D"], g["N"], g["lmax"], g["nbins"])
    nb = g["N"] - 1
    assert len({tuple(x) for x in k[:, nb:]}) == g["angular"]
    assert len({tuple(x) for x in k[:, :nb]}) == g["radial"]


# ------------------------------------------------------------------ 5PCF (N = 5, D = 3)
def _lams5(lmax, nbins=4):
    keys = oracle.keys(3, 5, lmax, nbins)
    lams = []
    for k in keys[:, 4:]:
        if tuple(k) not in lams:
            lams.append(tuple(int(x) for x in k))
    return lams


def test_5pcf_coupling_equals_printed_3j_form():
    """C^{Lambda;0} of the chain of eq. Coupling-C for N=5, D=3 equals the printed isotropic 5PCF
    form (-1)^{l1+l2+l3+l4} (-1)^{l12-m12} sqrt(2 l12 + 1) (l1 l2 l12; m1 m2 -m12)(l12 l3 l4; m12 m3 m4)
    (the printed sqrt(2 l12 - 1) read as sqrt(2 l12 + 1), eq. CG-examples), with sympy's 3j."""
    from sympy.physics.wigner import wigner_3j

    lmax = 2
    st = [tuple(s) for s in oracle.states(3, lmax)]
    for il, (l1, l2, l12, l3, l4) in enumerate(_lams5(lmax)):
        s, c = oracle.coupling_terms(3, 5, lmax, il)
        got = {tuple(st[x][0] for x in row): cc for row, cc in zip(s, c)}
        for m1 in range(-l1, l1 + 1):
            for m2 in range(-l2, l2 + 1):
                m12 = m1 + m2
                if abs(m12) > l12:
                    continue
                for m3 in range(-l3, l3 + 1):
                    m4 = -m12 - m3
                    if abs(m4) > l4:
                        continue
                    ref = ((-1) ** (l1 + l2 + l3 + l4 + l12 - m12) * np.sqrt(2 * l12 + 1) *
                           float(wigner_3j(l1, l2, l12, m1, m2, -m12)) * float(wigner_3j(l12, l3, l4, m12, m3, m4)))
                    assert abs(got.get((m1, m2, m3, m4), 0.0) - ref) < 1e-13, (l1, l2, l12, l3, l4, m1, m2, m3)


def test_5pcf_basis_rotation_invariant():
    lmax = 2
    R = _random_rotation(3, 19)
    rs = [_rand_dirs(3, 8, s) for s in (21, 22, 23, 24)]
    Y = [oracle.harmonics(3, lmax, r) for r in rs]
    YR = [oracle.harmonics(3, lmax, r @ R.T) for r in rs]
    for il in range(len(_lams5(lmax))):
        s, c = oracle.coupling_terms(3, 5, lmax, il)
        P = sum(cc * Y[0][:, a] * Y[1][:, b] * Y[2][:, e] * Y[3][:, f] for (a, b, e, f), cc in zip(s, c))
        PR = sum(cc * YR[0][:, a] * YR[1][:, b] * YR[2][:, e] * YR[3][:, f] for (a, b, e, f), cc in zip(s, c))
        np.testing.assert_allclose(P, PR, atol=1e-12)


def test_5pcf_separable_equals_naive_sum():
    """Separable 5PCF = the naive 5-tuplet sum on the same basis (the paper's machine-precision check)."""
    pos, w = _tiny(3, 40, 1.0, 131)
    edges = np.array([0.1, 0.25, 0.33, 0.39, 0.44])
    k1, z1 = oracle.estimate(3, 5, 2, edges, np.ones(3), pos, w, primaries=(0, 6))
    k2, z2 = oracle.estimate(3, 5, 2, edges, np.ones(3), pos, w, primaries=(0, 6), brute=True)
    assert np.array_equal(k1, k2)
    scale = np.max(np.abs(z1))
    assert scale > 0
    np.testing.assert_allclose(z1, z2, rtol=0, atol=1e-12 * scale)


def test_5pcf_l4_zero_slice_is_4pcf_times_a00():
    """With l4 = 0 the last two couplings force l12 = l3 and leave the N=4 coupling, so for one
    primary zeta_5(b1,b2,b3,b4; l1,l2,l3,l3,0) = zeta_4(b1,b2,b3; l1,l2,l3) * a_00(b4)."""
    pos, w = _tiny(3, 60, 1.0, 141)
    edges = np.linspace(0.05, 0.45, 6)
    j = 7
    k5, z5 = oracle.estimate(3, 5, 2, edges, np.ones(3), pos, w, primaries=(j, j + 1))
    k4, z4 = oracle.estimate(3, 4, 2, edges, np.ones(3), pos, w, primaries=(j, j + 1))
    idx4 = {tuple(int(x) for x in k): i for i, k in enumerate(k4)}
    d = pos - pos[j]
    d -= np.round(d)
    r = np.sqrt((d * d).sum(1))
    r[j] = -1.0
    vb = 4 * np.pi / 3 * (edges[1:] ** 3 - edges[:-1] ** 3)
    a00 = np.array([w[(r >= edges[b]) & (r < edges[b + 1])].sum() for b in range(5)]) / np.sqrt(4 * np.pi) / vb
    checked = 0
    for i, k in enumerate(k5):
        b1, b2, b3, b4, l1, l2, l12, l3, l4 = (int(x) for x in k)
        if l4 != 0:
            continue
        assert l12 == l3
        ref = z4[idx4[(b1, b2, b3, l1, l2, l3)]] * a00[b4]
        assert abs(z5[i] - ref) <= 1e-12 * max(1.0, np.max(np.abs(z5)))
        checked += 1
    assert checked > 50


# --------------------------------------------------------------- estimator
def _tiny(D, n, L, seed, w_mode="normal"):
    pos = catalogs.uniform(n, D, L, seed)
    if w_mode == "pm":
        w = np.where(np.arange(n) % 2 == 0, 1.0, -1.0)
    else:
        w = catalogs.normal_weights(n, 1.0, 0.3, seed + 1)
    return pos, w


@pytest.mark.parametrize("D,N,lmax,nb", [(2, 3, 4, 3), (3, 3, 3, 3), (4, 3, 2, 3), (2, 4, 3, 4), (3, 4, 2, 4)])
def test_separable_equals_naive_sum(D, N, lmax, nb):
    """The paper checks that the separable estimator reproduces the naive N-tuplet sum
    projected on the same basis to machine precision (timing-figure caption)."""
    n = 40 if N == 3 else 22
    pos, w = _tiny(D, n, 1.0, 100 + D + N)
    edges = np.linspace(0.05, 0.45, nb + 1)
    box = np.ones(D)
    k1, z1 = oracle.estimate(D, N, lmax, edges, box, pos, w, primaries=(0, 12))
    k2, z2 = oracle.estimate(D, N, lmax, edges, box, pos, w, primaries=(0, 12), brute=True)
    assert np.array_equal(k1, k2)
    scale = np.max(np.abs(z1))
    assert scale > 0
    np.testing.assert_allclose(z1, z2, rtol=0, atol=1e-12 * scale)


@pytest.mark.parametrize("D", [2, 3, 4])
def test_remove_self_equals_naive_sum_over_distinct_secondaries(D):
    """Excluding coincident secondaries (k = k', only on N=3 keys with b1 = b2): the separable
    form minus its degenerate term equals the naive pair sum that skips k = k', and the amount
    removed is the basis at coincident directions, (-1)^l sqrt(dim_l)/|S^{D-1}| for D >= 3 and
    1/(2 pi) for D = 2, times (1/V) sum_j w_j sum_{k in b} w_k^2 / v_b^2 (numpy below)."""
    lmax, nb = {2: 5, 3: 4, 4: 3}[D], 3
    pos, w = _tiny(D, 50, 1.0, 70 + D)
    edges = np.linspace(0.08, 0.45, nb + 1)
    box = np.ones(D)
    prim = (0, 20)
    k0, z_keep = oracle.estimate(D, 3, lmax, edges, box, pos, w, primaries=prim)
    k1, z_rm = oracle.estimate(D, 3, lmax, edges, box, pos, w, primaries=prim, remove_self=True)
    k2, z_rm_naive = oracle.estimate(D, 3, lmax, edges, box, pos, w, primaries=prim, brute=True, remove_self=True)
    assert np.array_equal(k0, k1) and np.array_equal(k1, k2)
    scale = np.max(np.abs(z_keep))
    np.testing.assert_allclose(z_rm, z_rm_naive, rtol=0, atol=1e-12 * scale)

    area = {2: 2 * np.pi, 3: 4 * np.pi, 4: 2 * np.pi ** 2}[D]
    vb = area / D * (edges[1:] ** D - edges[:-1] ** D)
    if D == 2:
        coinc = [1.0 / (2 * np.pi)] * (lmax + 1)
    else:
        dim = [2 * l + 1 if D == 3 else (l + 1) ** 2 for l in range(lmax + 1)]
        coinc = [(-1) ** l * math.sqrt(dim[l]) / area for l in range(lmax + 1)]
    s2 = np.zeros(nb)
    for j in range(*prim):
        d = pos - pos[j]
        d -= np.round(d)
        r = np.linalg.norm(d, axis=1)
        b = np.searchsorted(edges, r, side="right") - 1
        ok = (np.arange(len(pos)) != j) & (b >= 0) & (b < nb)
        for bb in range(nb):
            s2[bb] += w[j] * np.sum(w[ok][b[ok] == bb] ** 2)
    ref = np.array([s2[k[0]] * coinc[k[3]] / vb[k[0]] ** 2 if k[0] == k[1] else 0.0 for k in k0])
    assert np.count_nonzero(ref) > 0
    np.testing.assert_allclose(z_keep - z_rm, ref, rtol=0, atol=1e-12 * scale)


def test_remove_self_changes_nothing_without_coincident_bins():
    """Keys with strictly ordered bins (N=4, or N=3 with b1 < b2) have no coincident secondaries."""
    pos, w = _tiny(3, 30, 1.0, 90)
    edges = np.linspace(0.05, 0.45, 5)
    _, z = oracle.estimate(3, 4, 2, edges, np.ones(3), pos, w, primaries=(0, 8))
    _, zr = oracle.estimate(3, 4, 2, edges, np.ones(3), pos, w, primaries=(0, 8), remove_self=True)
    assert np.array_equal(z, zr)
    _, z = oracle.estimate(3, 3, 3, edges, np.ones(3), pos, w, primaries=(0, 8), bin_lt=True)
    _, zr = oracle.estimate(3, 3, 3, edges, np.ones(3), pos, w, primaries=(0, 8), bin_lt=True, remove_self=True)
    assert np.array_equal(z, zr)


def test_d3_3pcf_legendre_closed_form():
    """D=3, N=3: the basis is the Legendre polynomial rescaled by (-1)^l 4pi/sqrt(2l+1)
    (text after eq. zero-ang-mom-states), so zeta_l equals
    (1/V) sum_j w_j sum_{k,k'} w_k w_k' (-1)^l sqrt(2l+1)/(4pi) P_l(cos gamma)/(v v'),
    computed here with numpy and scipy only."""
    from scipy.special import eval_legendre

    D, lmax, nb = 3, 4, 4
    pos, w = _tiny(D, 60, 1.0, 7)
    edges = np.linspace(0.1, 0.45, nb + 1)
    keys, z = oracle.estimate(D, 3, lmax, edges, np.ones(3), pos, w)
    vb = 4 * np.pi / 3 * (edges[1:] ** 3 - edges[:-1] ** 3)
    ref = {}
    for j in range(len(pos)):
        d = pos - pos[j]
        d -= np.round(d)
        r = np.linalg.norm(d, axis=1)
        b = np.searchsorted(edges, r, side="right") - 1
        ok = (np.arange(len(pos)) != j) & (b >= 0) & (b < nb) & (r > 0)
        u = d[ok] / r[ok, None]
        bb = b[ok]
        ww = w[ok]
        t = np.clip(u @ u.T, -1, 1)
        for b1 in range(nb):
            for b2 in range(b1, nb):
                m = np.outer(bb == b1, bb == b2) * np.outer(ww, ww)
                for l in range(lmax + 1):
                    val = w[j] * np.sum(m * eval_legendre(l, t)) * (-1) ** l * math.sqrt(2 * l + 1) / (4 * np.pi)
                    ref[(b1, b2, l)] = ref.get((b1, b2, l), 0.0) + val / (vb[b1] * vb[b2])
    got = {(k[0], k[1], k[3]): v for k, v in zip(keys, z)}
    scale = max(abs(v) for v in ref.values())
    for kk, v in ref.items():
        assert abs(got[kk] - v) < 1e-12 * scale
        assert abs(got[kk].imag) < 1e-12 * scale


def test_d2_3pcf_exponential_closed_form():
    """D=2, N=3: zeta_l = (1/V) sum_j w_j a_l(b1) a_{-l}(b2) with a_l = (1/v) sum w e^{-il theta}/sqrt(2pi)
    (the D=2 basis of exponentials in the CMB section), written here with numpy."""
    D, lmax, nb = 2, 5, 3
    pos, w = _tiny(D, 80, 1.0, 17)
    edges = np.linspace(0.05, 0.4, nb + 1)
    keys, z = oracle.estimate(D, 3, lmax, edges, np.ones(2), pos, w)
    vb = np.pi * (edges[1:] ** 2 - edges[:-1] ** 2)
    ref = np.zeros(len(keys), complex)
    index = {(k[0], k[1], k[3]): i for i, k in enumerate(keys)}
    for j in range(len(pos)):
        d = pos - pos[j]
        d -= np.round(d)
        r = np.linalg.norm(d, axis=1)
        b = np.searchsorted(edges, r, side="right") - 1
        ok = (np.arange(len(pos)) != j) & (b >= 0) & (b < nb)
        th = np.arctan2(d[ok, 1], d[ok, 0])
        for l in range(lmax + 1):
            a = np.array([np.sum(w[ok][b[ok] == bb] * np.exp(-1j * l * th[b[ok] == bb])) for bb in range(nb)])
            am = np.array([np.sum(w[ok][b[ok] == bb] * np.exp(1j * l * th[b[ok] == bb])) for bb in range(nb)])
            a /= math.sqrt(2 * np.pi) * vb
            am /= math.sqrt(2 * np.pi) * vb
            for b1 in range(nb):
                for b2 in range(b1, nb):
                    ref[index[(b1, b2, l)]] += w[j] * a[b1] * am[b2]
    np.testing.assert_allclose(z, ref, atol=1e-12 * np.max(np.abs(ref)))


@pytest.mark.parametrize("D", [2, 3, 4])
def test_n3_separable_equals_addition_theorem(D):
    """Two routes to the same N=3 coefficients: harmonics + coupling (eq. NPCF-estimator-discrete)
    and the addition theorem (Gegenbauer of r1.r2; for D=2 the exponential of the relative
    angle), which uses neither."""
    lmax = {2: 6, 3: 4, 4: 3}[D]
    pos, w = _tiny(D, 70 if D == 3 else 60, 1.0, 31 + D)
    edges = np.linspace(0.1, 0.45, 4)
    k1, z1 = oracle.estimate(D, 3, lmax, edges, np.ones(D), pos, w)
    k2, z2 = oracle.estimate_n3_closed(D, lmax, edges, np.ones(D), pos, w)
    assert np.array_equal(k1, k2)
    np.testing.assert_allclose(z1, z2, atol=1e-12 * np.max(np.abs(z1)))


def test_l0_reduces_to_weighted_pair_counts():
    """zeta_0 needs no harmonic: Y_0 = 1/sqrt(|S^{D-1}|), coupling 1 (D=2) or 1/sqrt(dim_0)=1."""
    for D in (2, 3, 4):
        pos, w = _tiny(D, 50, 1.0, 41 + D)
        edges = np.linspace(0.1, 0.45, 4)
        keys, z = oracle.estimate(D, 3, 2, edges, np.ones(D), pos, w)
        area = 2 * np.pi ** (D / 2) / math.gamma(D / 2)
        vb = area / D * (edges[1:] ** D - edges[:-1] ** D)
        W = np.zeros((len(pos), 3))
        for j in range(len(pos)):
            d = pos - pos[j]
            d -= np.round(d)
            r = np.linalg.norm(d, axis=1)
            b = np.searchsorted(edges, r, side="right") - 1
            for bb in range(3):
                sel = (b == bb) & (np.arange(len(pos)) != j)
                W[j, bb] = np.sum(w[sel])
        for k, v in zip(keys, z):
            if k[3] != 0:
                continue
            ref = np.sum(w * W[:, k[0]] * W[:, k[1]]) / (area * vb[k[0]] * vb[k[1]])
            assert abs(v - ref) < 1e-12 * max(1.0, abs(ref))


def test_d3_4pcf_l3_zero_slice_factorises():
    """For one primary, zeta_{l l 0}(b1,b2,b3) = zeta^{N=3}_l(b1,b2) * a_00(b3), a_00 = W(b3)/(sqrt(4pi) v_b3):
    the l3=0 coupling (-1)^{2l}(l l 0; m -m 0) is the N=3 CG."""
    pos, w = _tiny(3, 60, 1.0, 51)
    edges = np.linspace(0.05, 0.45, 5)
    j = 7
    k4, z4 = oracle.estimate(3, 4, 3, edges, np.ones(3), pos, w, primaries=(j, j + 1))
    k3, z3 = oracle.estimate(3, 3, 3, edges, np.ones(3), pos, w, primaries=(j, j + 1))
    z3d = {(k[0], k[1], k[3]): v for k, v in zip(k3, z3)}
    d = pos - pos[j]
    d -= np.round(d)
    r = np.linalg.norm(d, axis=1)
    b = np.searchsorted(edges, r, side="right") - 1
    vb = 4 * np.pi / 3 * (edges[1:] ** 3 - edges[:-1] ** 3)
    n_checked = 0
    for k, v in zip(k4, z4):
        b1, b2, b3, l1, l2, l3 = k
        if l3 != 0:
            continue
        sel = (b == b3) & (np.arange(len(pos)) != j)
        a00 = np.sum(w[sel]) / (math.sqrt(4 * np.pi) * vb[b3])
        # the oracle's zeta already carries w_j/V once; the N=3 value too
        ref = z3d[(b1, b2, l1)] * a00
        assert abs(v - ref) < 1e-12 * max(1e-30, np.max(np.abs(z4)))
        n_checked += 1
    assert n_checked > 0


def test_translation_and_rotation_invariance():
    D = 3
    pos, w = _tiny(D, 45, 1.0, 61)
    edges = np.linspace(0.05, 0.45, 4)
    _, z = oracle.estimate(D, 4, 2, edges, np.ones(D), pos, w)
    shift = np.array([0.31, 0.77, 0.05])
    _, zt = oracle.estimate(D, 4, 2, edges, np.ones(D), np.mod(pos + shift, 1.0), w)
    np.testing.assert_allclose(zt, z, atol=1e-11 * np.max(np.abs(z)))
    # open boundary: rotate the cloud; the isotropic coefficients are unchanged
    R = _random_rotation(D, 3)
    _, zo = oracle.estimate(D, 4, 2, edges, np.ones(D), pos, w, periodic=False)
    _, zr = oracle.estimate(D, 4, 2, edges, np.ones(D), pos @ R.T, w, periodic=False)
    np.testing.assert_allclose(zr, zo, atol=1e-11 * np.max(np.abs(zo)))


def test_periodic_cube_symmetries():
    """The 48 signed axis permutations map the periodic unit cube onto itself: the 24 rotations
    leave every D=3 4PCF coefficient unchanged; the 24 improper ones keep the even-parity
    coefficients and flip the odd ones (eq. basis-parity-conj).  The 5PCF keeps only even
    parity, so all 48 leave it unchanged."""
    import itertools

    pos, w = _tiny(3, 36, 1.0, 65)
    edges = np.linspace(0.05, 0.45, 4)
    keys, z = oracle.estimate(3, 4, 2, edges, np.ones(3), pos, w)
    odd = (keys[:, 3] + keys[:, 4] + keys[:, 5]) % 2 == 1
    scale = np.max(np.abs(z))
    p5, w5 = _tiny(3, 24, 1.0, 66)
    e5 = np.linspace(0.05, 0.45, 5)
    _, z5 = oracle.estimate(3, 5, 2, e5, np.ones(3), p5, w5, primaries=(0, 6))
    s5 = np.max(np.abs(z5))
    assert s5 > 0 and np.any(odd)
    count = 0
    for perm in itertools.permutations(range(3)):
        for signs in itertools.product((1.0, -1.0), repeat=3):
            M = np.zeros((3, 3))
            for i in range(3):
                M[i, perm[i]] = signs[i]
            proper = np.linalg.det(M) > 0
            _, zc = oracle.estimate(3, 4, 2, edges, np.ones(3), np.mod(pos @ M.T, 1.0), w)
            expect = z if proper else np.where(odd, -z, z)
            np.testing.assert_allclose(zc, expect, rtol=0, atol=1e-11 * scale)
            _, zc5 = oracle.estimate(3, 5, 2, e5, np.ones(3), np.mod(p5 @ M.T, 1.0), w5, primaries=(0, 6))
            np.testing.assert_allclose(zc5, z5, rtol=0, atol=1e-11 * s5)
            count += 1
    assert count == 48


@pytest.mark.parametrize("D,N", [(3, 4), (2, 4), (2, 3)])
def test_parity_reflection_and_reality(D, N):
    """Even-parity coefficients are real and unchanged by a reflection; odd ones are imaginary and
    change sign (eq. basis-parity-conj and the discussion after it)."""
    pos, w = _tiny(D, 40, 1.0, 71 + D)
    edges = np.linspace(0.05, 0.45, 4 if N == 4 else 3)
    keys, z = oracle.estimate(D, N, 3, edges, np.ones(D), pos, w, periodic=False)
    refl = pos.copy()
    refl[:, 0] = -refl[:, 0]
    _, zr = oracle.estimate(D, N, 3, edges, np.ones(D), refl, w, periodic=False)
    scale = np.max(np.abs(z))
    if D == 3:
        odd = (keys[:, 3] + keys[:, 4] + keys[:, 5]) % 2 == 1
        assert np.max(np.abs(z[~odd].imag)) < 1e-12 * scale
        assert np.max(np.abs(z[odd].real)) < 1e-12 * scale
        np.testing.assert_allclose(zr[~odd], z[~odd], atol=1e-11 * scale)
        np.testing.assert_allclose(zr[odd], -z[odd], atol=1e-11 * scale)
    else:
        # D=2: a reflection conjugates e^{i l theta}: real parts even, imaginary parts odd
        np.testing.assert_allclose(zr, z.conj(), atol=1e-11 * scale)
        assert np.max(np.abs(z.imag)) > 1e-6 * scale  # odd parts exist for N > D


@pytest.mark.parametrize("D", [2, 3, 4])
def test_gradient_matches_finite_differences_and_identities(D):
    """The N=3 gradient oracle: central differences away from bin edges, translation invariance
    (sum_i dL/dy_i = 0) and degree-3 homogeneity in the weights (sum_i w_i dL/dw_i = 3 L)."""
    lmax = {2: 4, 3: 3, 4: 2}[D]
    g = np.random.default_rng(5)
    pos, w = _tiny(D, 40, 1.0, 81)
    edges = np.linspace(0.1, 0.5, 4)
    keys, z = oracle.estimate_n3_closed(D, lmax, edges, np.ones(D), pos, w)
    gc = g.normal(size=len(keys)) + 1j * g.normal(size=len(keys))
    _, z0, gp, gw = oracle.estimate_n3_closed(D, lmax, edges, np.ones(D), pos, w, grad_coeffs=gc)
    L0 = float(np.sum(gc.real * z0.real + gc.imag * z0.imag))
    if D == 2:
        assert np.max(np.abs(z0.imag)) > 1e-6 * np.max(np.abs(z0))  # the imaginary parts are exercised
    np.testing.assert_allclose(gp.sum(axis=0), 0.0, atol=1e-10 * np.max(np.abs(gp)))
    assert abs(np.sum(w * gw) - 3 * L0) < 1e-10 * max(1.0, abs(L0))

    def loss(p, ww):
        _, zz = oracle.estimate_n3_closed(D, lmax, edges, np.ones(D), p, ww)
        return float(np.sum(gc.real * zz.real + gc.imag * zz.imag))

    h = 1e-6
    # pick coordinates whose pairs are all far from the edges
    d = pos[:, None, :] - pos[None, :, :]
    d -= np.round(d)
    r = np.linalg.norm(d, axis=2)
    gap = np.min(np.abs(r[..., None] - edges[None, None, :]), axis=2)
    np.fill_diagonal(gap, 1.0)
    safe = [i for i in range(len(pos)) if np.min(gap[i]) > 1e-4]
    assert len(safe) >= 3
    for i in safe[:4]:
        for a in range(D):
            pp = pos.copy(); pp[i, a] += h
            pm = pos.copy(); pm[i, a] -= h
            fd = (loss(pp, w) - loss(pm, w)) / (2 * h)
            assert abs(fd - gp[i, a]) < 1e-6 * max(1.0, np.max(np.abs(gp)))
        wp = w.copy(); wp[i] += h
        wm = w.copy(); wm[i] -= h
        fd = (loss(pos, wp) - loss(pos, wm)) / (2 * h)
        assert abs(fd - gw[i]) < 1e-6 * max(1.0, np.max(np.abs(gw)))


def test_d2_4pcf_exponential_closed_form():
    """D=2, N=4: zeta_{l1 l2 l3}(b1,b2,b3) = (1/V) sum_j w_j a_l1(b1) a_l2(b2) a_l3(b3), l1+l2+l3=0,
    with a_l = (1/v) sum w e^{-il theta}/sqrt(2pi) (the CMB-section basis of exponentials)."""
    D, lmax, nb = 2, 3, 4
    pos, w = _tiny(D, 60, 1.0, 19)
    edges = np.linspace(0.05, 0.45, nb + 1)
    keys, z = oracle.estimate(D, 4, lmax, edges, np.ones(2), pos, w)
    vb = np.pi * (edges[1:] ** 2 - edges[:-1] ** 2)
    ref = np.zeros(len(keys), complex)
    for j in range(len(pos)):
        d = pos - pos[j]
        d -= np.round(d)
        r = np.linalg.norm(d, axis=1)
        b = np.searchsorted(edges, r, side="right") - 1
        ok = (np.arange(len(pos)) != j) & (b >= 0) & (b < nb)
        th = np.arctan2(d[ok, 1], d[ok, 0])
        bo = b[ok]
        wo = w[ok]
        a = {}
        for l in range(-lmax, lmax + 1):
            a[l] = np.array([np.sum(wo[bo == bb] * np.exp(-1j * l * th[bo == bb])) for bb in range(nb)])
            a[l] /= math.sqrt(2 * np.pi) * vb
        for i, k in enumerate(keys):
            ref[i] += w[j] * a[k[3]][k[0]] * a[k[4]][k[1]] * a[k[5]][k[2]]
    assert np.all(keys[:, 3] + keys[:, 4] + keys[:, 5] == 0)
    np.testing.assert_allclose(z, ref, atol=1e-12 * np.max(np.abs(ref)))
