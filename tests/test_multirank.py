"""Host logic of the multi-process paths with 2 gloo ranks on the CPU; each rank's share is
computed by the FP64 oracle, so the results must equal the single-process oracle."""
import os
import socket

import numpy as np
import pytest

import oracle
from paper_2106_10278_gb300 import catalogs, shard

torch = pytest.importorskip("torch")


def test_primary_ranges_cover_once():
    for n in (0, 1, 7, 100, 2000144):
        for world in (1, 2, 3, 8):
            r = shard.primary_ranges(n, world)
            assert r[0][0] == 0 and r[-1][1] == n
            assert all(a[1] == b[0] for a, b in zip(r, r[1:]))
            sizes = [b - a for a, b in r]
            assert max(sizes) - min(sizes) <= 1


def test_lpt_assign_balances_and_covers():
    costs = np.array([9.0, 7.0, 6.0, 5.0, 5.0, 4.0, 3.0, 1.0])
    a = shard.lpt_assign(costs, 3)
    assert sorted(i for lst in a for i in lst) == list(range(len(costs)))
    loads = [costs[lst].sum() for lst in a]
    assert max(loads) <= 14.0  # optimum 40/3 -> 14 here; LPT is within 4/3 of it
    assert shard.lpt_assign(costs, 3) == a  # deterministic


def test_estimated_pairs_uniform_count():
    pos = catalogs.uniform(3000, 3, 1.0, 5)
    edges = np.array([0.05, 0.15])
    est = shard.estimated_pairs([3000], [[1.0, 1.0, 1.0]], edges, 3)[0]
    d = pos[:, None, :] - pos[None, :, :]
    d -= np.round(d)
    r = np.sqrt((d * d).sum(-1))
    got = np.count_nonzero((r >= 0.05) & (r < 0.15))
    assert abs(got - est) < 0.05 * est


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _as_tensor(z):
    out = np.empty(2 * len(z))
    out[0::2], out[1::2] = z.real, z.imag
    return torch.tensor(out, dtype=torch.float64)


def _worker(rank, world, port, q):
    import torch.distributed as dist

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        oracle.build()
        wl = catalogs.workload("d3n3_fp64", scale=0.15)
        full = shard.sharded_compute(
            lambda pb, pe: _as_tensor(oracle.estimate(3, 3, 5, wl.edges, wl.box, wl.pos, wl.w,
                                                      primaries=(pb, pe))[1]), wl.n)
        # a batch of three catalogues spread by LPT
        cats = [catalogs.uniform(n, 3, 1.0, 70 + i) for i, n in enumerate((150, 400, 250))]
        edges = np.linspace(0.05, 0.3, 5)
        costs = shard.estimated_pairs([len(c) for c in cats], np.ones((3, 3)), edges, 3)
        res = shard.sharded_batch(
            lambda i: _as_tensor(oracle.estimate(3, 4, 2, edges, np.ones(3), cats[i], np.ones(len(cats[i])))[1]),
            costs)
        q.put((rank, full.numpy(), [r.numpy() for r in res]))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_match_single_process():
    import torch.multiprocessing as mp

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = [q.get(timeout=300) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    wl = catalogs.workload("d3n3_fp64", scale=0.15)
    ref = _as_tensor(oracle.estimate(3, 3, 5, wl.edges, wl.box, wl.pos, wl.w)[1]).numpy()
    cats = [catalogs.uniform(n, 3, 1.0, 70 + i) for i, n in enumerate((150, 400, 250))]
    edges = np.linspace(0.05, 0.3, 5)
    refs = [_as_tensor(oracle.estimate(3, 4, 2, edges, np.ones(3), c, np.ones(len(c)))[1]).numpy() for c in cats]
    for rank, full, res in got:
        np.testing.assert_allclose(full, ref, rtol=0, atol=1e-12 * np.abs(ref).max())
        for a, b in zip(res, refs):
            assert np.array_equal(a, b)  # each catalogue computed whole on one rank
