"""The work counts bench.py reports, against the counts stated for the paper's isotropic bases:
(Lambda, m1, m2) coupling terms per bin triple of the D=3 4PCF (3555 at lmax 5, 1439 at lmax 4),
the D=2 4PCF label count (176 at lmax 10 with l1 >= 0), the pair-count helper, and the tiling
behind the 5PCF tensor-core MMA count."""
import math
import os
import sys

import numpy as np

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import bench  # noqa: E402


def test_coupling_terms_per_primary():
    assert bench.coupling_terms_per_primary(3, 4, 5, 10) == math.comb(10, 3) * 3555
    assert bench.coupling_terms_per_primary(3, 4, 4, 8) == math.comb(8, 3) * 1439
    assert bench.coupling_terms_per_primary(2, 4, 10, 16) == math.comb(16, 3) * 176
    assert bench.coupling_terms_per_primary(3, 5, 4, 10) == math.comb(10, 4) * 61749
    # N=3: one term per (l, m) per bin pair with b1 <= b2
    assert bench.coupling_terms_per_primary(3, 3, 5, 10) == 36 * 55


def test_flop_counts_are_stated_values():
    assert bench.pair_flops_per_pair(3, 5) == 133
    assert bench.pair_flops_per_pair(3, 10) == 423
    assert bench.adjoint_flops_per_pair(4, 4) == 2130


def test_count_pairs_numpy_brute_force():
    g = np.random.default_rng(0)
    pos = g.random((300, 3))
    edges = np.array([0.05, 0.1, 0.2])
    d = pos[:, None, :] - pos[None, :, :]
    d -= np.round(d)
    r = np.sqrt((d * d).sum(-1))
    np.fill_diagonal(r, -1.0)
    want = int(np.count_nonzero((r >= 0.05) & (r < 0.2)))
    assert bench.count_pairs_numpy(pos, edges, np.ones(3), (0, 300)) == want


def test_d3n5_tensor_tiles_cover_every_key_once():
    """The tiling behind the 5PCF tensor-core MMA count: the entries of the kept tiles that are
    keys (b2 < b3 within one parity) are exactly the paper's 5PCF components -- 210 bin quadruples
    x 585 label sets at 10 bins and lmax 4 -- each in one tile; 58 tiles with K per primary
    summing to 416 there."""
    for lmax, nbins in ((4, 10), (2, 6), (1, 4)):
        keys = set()
        for l12, rows, cols in bench.d3n5_tc_tiles(lmax, nbins):
            for b2, b1, (l1, l2) in rows:
                for b3, b4, (l3, l4) in cols:
                    if b2 < b3:
                        k = (b1, b2, b3, b4, l1, l2, l12, l3, l4)
                        assert k not in keys
                        keys.add(k)
        # every even-parity label set (l1, l2, l12, l3, l4) with the two triangle conditions, for
        # every b1 < b2 < b3 < b4
        lam = [(l1, l2, l12, l3, l4) for l1 in range(lmax + 1) for l2 in range(lmax + 1)
               for l12 in range(abs(l1 - l2), l1 + l2 + 1) for l3 in range(lmax + 1) for l4 in range(lmax + 1)
               if abs(l12 - l3) <= l4 <= l12 + l3 and (l1 + l2 + l3 + l4) % 2 == 0]
        assert len(keys) == math.comb(nbins, 4) * len(lam)
        if (lmax, nbins) == (4, 10):
            assert len(lam) == 585 and math.comb(nbins, 4) == 210
            assert len(bench.d3n5_tc_tiles(lmax, nbins)) == 58
            assert bench.d3n5_tc_k1_sum(lmax, nbins) == 416
