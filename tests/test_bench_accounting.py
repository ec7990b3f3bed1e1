"""The work counts bench.py reports, against the counts stated for the paper's isotropic bases:
(Lambda, m1, m2) coupling terms per bin triple of the D=3 4PCF (3555 at lmax 5, 1439 at lmax 4),
the D=2 4PCF label count (176 at lmax 10 with l1 >= 0), and the pair-count helper."""
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
