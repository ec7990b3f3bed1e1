#!/usr/bin/env python
"""Benchmark of the separable isotropic NPCF estimator on GB300.

One step = one full evaluation (cell list, pair kernel, coupling kernel, FP64
reduction) of the D=3 isotropic 4PCF on the data-minus-randoms workload:
~1M Poisson draws from a lognormal field (256^3 grid, P(k) ~ k^-1.5) plus 1M
uniform randoms with weight -1, periodic box of side 1000, 10 radial bins
over [20, 160], lmax = 5 (13,320 complex coefficients).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--workload d3n4|d3n3_fp64|d2n3|d2n4|d4n3|d3n5|s2n4|d4n3-grad|batch64] [--scale S]

Other workloads: d4n3-grad times one gradient step of the D=4 3PCF (forward,
chi^2 upstream gradient, backward: npcf_backward); batch64 times the 64
catalogues of the batched workload through npcf_compute_batched (the 3PCF at
lmax 10 and the 4PCF at lmax 4, one call each).  --scale < 1 shrinks a
workload for profiling; --no-cpu-baseline / --no-e2e skip those legs.

Under torchrun (N > 1) every rank runs its own catalogue (seed + rank):
independent problems, no data-path collective ("scaling": "weak").
Prints one JSON line on rank 0.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "pairs/s and NPCF coeffs/s, 3D iso 4PCF n=1M, mixed vs FP32 at stated rel err"
BATCH_METRIC = "pairs/s, batched D=3 3PCF (lmax 10) + 4PCF (lmax 4) of 64 catalogues"
GRAD_METRIC = "pairs/s, D=4 3PCF gradient step (forward + chi^2 + backward)"
GRAD_WORKLOAD = ("d4n3-grad: D=4 3PCF, n=100k (50k uniform + 50k in 200 Gaussian blobs, sigma 0.01) in the "
                 "periodic unit 4-cube, 8 bins over [0.01,0.12], lmax 4; chi^2 loss against the seed-104 catalogue")


def batch_workload(ncat, n):
    return (f"batch64: {ncat} catalogues, n={n}, boxes 500-1000, 8 bins over [10,120]; 3PCF lmax 10 and 4PCF "
            "lmax 4 (two batched calls, pairs counted once)")
WORKLOAD = ("d3n4: D=3 isotropic 4PCF, ~1M lognormal-Poisson data (w=+1) + 1M uniform randoms (w=-1), "
            "periodic box 1000, 10 linear bins over [20,160], lmax=5")
# the arithmetic each precision runs the path in (pair stage / coupling)
DTYPES = {"fp32": "f32", "fp64": "f64", "mixed_bf16x3": "f32 pairs, bf16x3 tensor-core coupling",
          "mixed_tf32x3": "f32 pairs, tf32x3 tensor-core coupling"}
SM_COUNT_NOMINAL = 152
FP32_LANES_PER_SM = 128


def _args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default="d3n4")
    ap.add_argument("--cpu-seconds", type=float, default=15.0, help="target CPU time of the oracle baseline")
    ap.add_argument("--scale", type=float, default=1.0, help="shrink the workload (profiling)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-autotune", action="store_true", help="keep the built-in launch shapes")
    ap.add_argument("--no-mixed-arm", action="store_true",
                    help="skip the split-precision (tensor-core) coupling comparison on the D=2 4PCF workload")
    ap.add_argument("--precision", default=None,
                    help="fp32 | fp64 | mixed_bf16x3 | mixed_tf32x3 (default: the workload's own, fp32 or fp64)")
    return ap.parse_args()


# ------------------------------------------------------------ counting helpers
def pair_flops_per_pair(D: int, lmax: int) -> int:
    """Algorithmic FP32 operations of one pair (FMA = 2): separation and r^2,
    the direction, the harmonic recurrence and the accumulation, counted from
    the recurrence of the pair kernel: D=3 counts the powers (x - iy)^m, the first step z P_m of
    each column, the three-term steps (one multiply by the recurrence constant and one FMA per
    real part) and one add per accumulated component."""
    sep = 3 * D  # D subtractions, D multiply-adds for r^2 (2 each) -> 3D
    direction = 2 + D  # rsqrt, r, D scalings
    if D == 3:
        powers = 6 * lmax  # complex multiply by (x - iy): 2 FMA + 2 MUL
        first = 1 + 2 * lmax  # z * P_m (real for m = 0, complex after)
        rec = 0
        for m in range(lmax + 1):
            for _ in range(m + 2, lmax + 1):
                rec += 3 if m == 0 else 5  # A*z, then one FMA per real component
        acc = (lmax + 1) ** 2
        return sep + direction + powers + first + rec + acc
    if D == 2:
        return sep + direction + 6 * lmax + (2 * lmax + 1)
    nq = sum((l + 1) ** 2 for l in range(lmax + 1))
    return sep + direction + 6 * lmax + 5 * lmax * lmax + 2 * nq


# the 2-sphere's pair beyond the D=2 one: a third separation component (3), the tangent vector
# chord + (chord^2 / 2) n_j (1 + 3 FMA = 7) and its two frame components (2 x 3 FMA = 12), less the
# D=2 direction's scalings it replaces (no change): 22
SPHERE_EXTRA_FLOPS = 22


# algorithmic FP32 operations per coupling term: N=3 a complex product and its accumulation, N=4 the
# complex triple product (8, as counted for the 4PCF), N=5 one more complex multiplication
COUPLING_FLOPS_PER_TERM = {3: 4, 4: 8, 5: 14}


def coupling_terms_per_primary(D: int, N: int, lmax: int, nbins: int) -> int:
    """Non-zero (Lambda, m1, m2) coupling terms summed over the bin tuples of one primary."""
    if N == 3:
        per = sum(2 * l + 1 for l in range(lmax + 1)) if D == 3 else (lmax + 1)
        return per * nbins * (nbins + 1) // 2
    if N == 5:  # D=3: (l1, l2, l12, l3, l4) even parity, (m1, m2, m3) with |m1 + m2| <= l12, |m4| <= l4
        t = 0
        for l1 in range(lmax + 1):
            for l2 in range(lmax + 1):
                for l12 in range(abs(l1 - l2), l1 + l2 + 1):
                    for l3 in range(lmax + 1):
                        for l4 in range(abs(l12 - l3), min(l12 + l3, lmax) + 1):
                            if (l1 + l2 + l3 + l4) % 2:
                                continue
                            for m1 in range(-l1, l1 + 1):
                                for m2 in range(-l2, l2 + 1):
                                    if abs(m1 + m2) <= l12:
                                        t += sum(1 for m3 in range(-l3, l3 + 1) if abs(m1 + m2 + m3) <= l4)
        return math.comb(nbins, 4) * t
    ntrip = math.comb(nbins, 3)
    if D == 2:
        return ntrip * sum(1 for a in range(lmax + 1) for b in range(-lmax, lmax + 1) if abs(a + b) <= lmax)
    t = 0
    for l1 in range(lmax + 1):
        for l2 in range(lmax + 1):
            for l3 in range(abs(l1 - l2), min(l1 + l2, lmax) + 1):
                for m1 in range(-l1, l1 + 1):
                    for m2 in range(-l2, l2 + 1):
                        if abs(m1 + m2) <= l3:
                            t += 1
    return ntrip * t


def adjoint_flops_per_pair(D: int, lmax: int) -> int:
    """Algorithmic FP32 operations of one pair in the adjoint pair kernel: the
    separation and direction, the harmonics carried as dual numbers (value and
    D partials: every product costs 2D + 1 operations, every FMA with the
    c-coefficients D + 1 FMAs), and the tangential projection."""
    fwd = pair_flops_per_pair(D, lmax)
    return 3 * D + 2 + D + (2 * D + 1) * fwd + 6 * D


def count_pairs_numpy(pos, edges, box, primaries, geometry="box"):
    """Ordered pairs (j, k != j, r in [e0, e_nb), minimum image) of the given primaries; on the
    2-sphere, cos theta in [e0, e_nb) between the normalised directions."""
    if geometry == "sphere":
        u = pos / np.linalg.norm(pos, axis=1, keepdims=True)
        tot = 0
        for j in range(*primaries):
            c = u @ u[j]
            tot += int(np.count_nonzero((c >= edges[0]) & (c < edges[-1])))
        return tot
    lo, hi = edges[0] ** 2, edges[-1] ** 2
    tot = 0
    for j in range(*primaries):
        d = pos - pos[j]
        d -= box * np.round(d / box)
        r2 = np.einsum("ij,ij->i", d, d)
        tot += int(np.count_nonzero((r2 >= lo) & (r2 < hi) & (r2 > 0)))
    return tot


# --------------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id=None):
        self.proc = None
        self.path = tempfile.mktemp(prefix="npcf_clocks_", suffix=".csv")
        cmd = ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "200"]
        if gpu_id:
            cmd += ["-i", gpu_id]
        try:
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(cmd, stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"unavailable": "nvidia-smi not runnable"}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append((float(parts[1]), float(parts[2]), parts[5:9]))
            except ValueError:
                continue
        os.unlink(self.path)
        if not rows:
            return {"unavailable": "no samples"}
        sm = [r[0] for r in rows]
        mx = max(r[1] for r in rows)
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i, v in enumerate(r[2]) if v.lower().startswith("active")})
        loaded = [s for s in sm if s > 0.5 * mx] or sm
        return {"sm_mhz": float(np.median(loaded)), "sm_max_mhz": mx, "reasons": reasons, "samples": len(rows)}


def _peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


def kernel_source_sha16() -> str:
    """Hash of the pair kernel's sources (the kernel, its harmonics and shared structures): a
    committed ncu traffic figure is used only while it matches."""
    import hashlib

    h = hashlib.sha256()
    for f in ("npcf_pairs.cuh", "npcf_device.cuh", "npcf_internal.h", "npcf_math.h"):
        h.update(open(os.path.join(ROOT, "paper_2106_10278_gb300", "csrc", f), "rb").read())
    return h.hexdigest()[:16]


def _traffic_from_profiles(workload: str):
    """Per-launch DRAM bytes of the pair kernel from the committed ncu summary, if it was taken on the
    current kernel sources (its kernel_sha16 line matches); else None."""
    path = os.path.join(ROOT, "profiles", f"k_pairs_{workload}.md")
    vals = {}
    try:
        for line in open(path):
            for key in ("traffic_bytes_per_launch:", "kernel_sha16:"):
                if line.startswith(key):
                    vals[key] = line.split(":", 1)[1].strip()
    except OSError:
        return None
    v = vals.get("traffic_bytes_per_launch:")
    if v in (None, "", "null") or vals.get("kernel_sha16:") != kernel_source_sha16():
        return None
    return float(v)


# ---------------------------------------------------------------------- arms
_ORACLE_INPUT = {}


def _oracle_worker_init(path):
    """Spawned worker: load the workload saved by the parent (memory-mapped) and build nothing."""
    import oracle

    oracle.build()
    d = np.load(path, allow_pickle=True)
    _ORACLE_INPUT.update({k: d[k] for k in d.files})


def _oracle_worker_block(prims):
    """The oracle, as it stands, on one block of primaries; returns (coefficients, seconds)."""
    import oracle

    x = _ORACLE_INPUT
    t0 = time.perf_counter()
    if str(x.get("geometry", "box")) == "sphere":
        _, z = oracle.estimate_sphere(int(x["N"]), int(x["lmax"]), x["edges"], x["pos"], x["w"], primaries=prims)
    else:
        _, z = oracle.estimate(int(x["D"]), int(x["N"]), int(x["lmax"]), x["edges"], x["box"], x["pos"], x["w"],
                               primaries=prims)
    return z, time.perf_counter() - t0


def _oracle_estimate(wl, primaries):
    """The oracle's estimate of a workload on a range of primaries (Euclidean or 2-sphere)."""
    import oracle

    if wl.geometry == "sphere":
        return oracle.estimate_sphere(wl.N, wl.lmax, wl.edges, wl.pos, wl.w, primaries=primaries)
    return oracle.estimate(wl.D, wl.N, wl.lmax, wl.edges, wl.box, wl.pos, wl.w, primaries=primaries)


def _cpu_baseline(wl, target_s, gpu_range_fn=None):
    """The FP64 oracle (as it stands) on a bounded sample of primaries: single-threaded, then the same
    program in one spawned process per host core over disjoint primary blocks.  When gpu_range_fn is
    given, the GPU's coefficients of the single-threaded sample's primaries are compared with the
    oracle's (the per-result error of this run)."""
    import multiprocessing as mp

    import oracle

    oracle.build()
    t0 = time.perf_counter()
    _oracle_estimate(wl, (0, 1))
    t1 = time.perf_counter() - t0
    nprim = int(max(1, min(256, round(target_s / max(t1, 1e-3)))))
    t0 = time.perf_counter()
    keys, ref = _oracle_estimate(wl, (0, nprim))
    dt = time.perf_counter() - t0
    pairs = count_pairs_numpy(wl.pos, wl.edges, wl.box, (0, nprim), wl.geometry)
    host = os.cpu_count() or 1
    out = {"value": pairs / dt, "unit": "pairs/s", "cores": 1, "host_cores": host, "kind": "oracle",
           "sample": f"primaries [0,{nprim}) of the {wl.n}-particle workload, all secondaries, "
                     f"{pairs} pairs in {dt:.2f} s (FP64 C oracle, single thread)"}
    if gpu_range_fn is not None:
        got, plan_keys = gpu_range_fn(0, nprim)
        index = {tuple(int(v) for v in k): i for i, k in enumerate(keys)}
        r = ref[np.array([index[tuple(int(v) for v in k)] for k in plan_keys])]
        out["rel_err_vs_oracle"] = {"value": float(np.linalg.norm(got - r) / np.linalg.norm(r)),
                                    "primaries": [0, nprim],
                                    "measure": "||gpu - oracle||_2 / ||oracle||_2 over all coefficients"}
    if host > 1:
        # the same oracle in `host` spawned processes, each on its own block of m primaries
        m = nprim
        blocks = [(nprim + i * m, nprim + (i + 1) * m) for i in range(host)]
        if blocks[-1][1] <= wl.n:
            fd, path = tempfile.mkstemp(suffix=".npz")
            os.close(fd)
            try:
                np.savez(path, D=wl.D, N=wl.N, lmax=wl.lmax, edges=wl.edges, box=wl.box, pos=wl.pos, w=wl.w,
                         geometry=wl.geometry)
                ctx = mp.get_context("spawn")
                with ctx.Pool(host, initializer=_oracle_worker_init, initargs=(path,)) as pool:
                    pool.map(_oracle_worker_block, [(i, i + 1) for i in range(host)])  # warm every worker
                    t0 = time.perf_counter()
                    res = pool.map(_oracle_worker_block, blocks)
                    wall = time.perf_counter() - t0
                ppairs = sum(count_pairs_numpy(wl.pos, wl.edges, wl.box, b, wl.geometry) for b in blocks)
                out["all_cores"] = {"value": ppairs / wall, "unit": "pairs/s", "cores": host,
                                    "sample": f"{host} processes x {m} primaries ([{nprim},{blocks[-1][1]})), "
                                              f"{ppairs} pairs in {wall:.2f} s wall (the same oracle, one spawned "
                                              "process per host core)"}
            finally:
                os.unlink(path)
    return out


def _reference_per_step(args, t_one):
    """Primaries per reference step: about min(20 s, 150 s / (steps + warmup)) of oracle time, so that the
    whole run ends within a few minutes."""
    return max(1, int(round(min(20.0, 150.0 / max(args.steps + args.warmup, 1)) / max(t_one, 1e-3))))


def _reference_line(args, metric, workload, n, v, total_t, sample):
    return {
        "impl": "reference", "metric": metric, "value": v, "unit": "pairs/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total_t / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": workload, "n": n},
        "cpu_baseline": {"value": v, "unit": "pairs/s", "cores": 1, "kind": "oracle", "sample": sample},
        "e2e": {"value": v, "unit": "pairs/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }


def _reference_batch64(args):
    """The oracle on the batched workload: every step runs the 3PCF (lmax 10) and the 4PCF (lmax 4) on a
    block of primaries of one catalogue (catalogue k mod 64 at step k); pairs are counted once, as in the
    GPU arm."""
    from paper_2106_10278_gb300 import catalogs
    import oracle

    bw = catalogs.batch64()

    def one(i, a, m):
        p, w, box = bw.catalogue(i)
        t0 = time.perf_counter()
        oracle.estimate(3, 3, 10, bw.edges, box, p, w, primaries=(a, a + m))
        oracle.estimate(3, 4, 4, bw.edges, box, p, w, primaries=(a, a + m))
        return time.perf_counter() - t0

    per_step = _reference_per_step(args, one(0, 0, 1))
    for k in range(args.warmup):
        one(k % bw.ncat, 0, 1)
    total_pairs, total_t, sizes = 0, 0.0, []
    for k in range(args.steps):
        i = k % bw.ncat
        p, w, box = bw.catalogue(i)
        m = min(per_step, len(p))
        a = (k * m) % max(len(p) - m + 1, 1)
        total_t += one(i, a, m)
        total_pairs += count_pairs_numpy(p, bw.edges, box, (a, a + m))
        sizes.append(m)
    v = total_pairs / total_t
    sample = (f"{max(sizes)} primaries per step (catalogue k mod {bw.ncat} at step k, all its secondaries), "
              "3PCF lmax 10 + 4PCF lmax 4")
    print(json.dumps(_reference_line(args, BATCH_METRIC, batch_workload(bw.ncat, len(bw.pos)), len(bw.pos), v,
                                     total_t, sample)), flush=True)


def _reference_grad(args):
    """The oracle on the gradient workload: every step runs the forward estimate and the analytic gradient
    (the addition-theorem form, bins held fixed) on a block of primaries, with the chi^2 upstream gradient
    2 (zeta - t); t is the seed-104 catalogue's estimate on the same block, computed once outside the
    timing (its values do not change the work)."""
    from paper_2106_10278_gb300 import catalogs
    import oracle

    wl = catalogs.workload("d4n3", seed=4)
    tgt = catalogs.workload("d4n3", seed=104)

    def one(a, m, t):
        t0 = time.perf_counter()
        _, z = oracle.estimate(4, 3, 4, wl.edges, wl.box, wl.pos, wl.w, primaries=(a, a + m))
        oracle.estimate_n3_closed(4, 4, wl.edges, wl.box, wl.pos, wl.w, primaries=(a, a + m),
                                  grad_coeffs=2.0 * (z - t))
        return time.perf_counter() - t0

    _, t1 = oracle.estimate(4, 3, 4, tgt.edges, tgt.box, tgt.pos, tgt.w, primaries=(0, 1))
    per_step = min(_reference_per_step(args, one(0, 1, t1)), wl.n)
    _, t = oracle.estimate(4, 3, 4, tgt.edges, tgt.box, tgt.pos, tgt.w, primaries=(0, per_step))
    for k in range(args.warmup):
        one(k, 1, t1)
    total_pairs, total_t = 0, 0.0
    for k in range(args.steps):
        a = (k * per_step) % max(wl.n - per_step + 1, 1)
        total_t += one(a, per_step, t)
        total_pairs += count_pairs_numpy(wl.pos, wl.edges, wl.box, (a, a + per_step))
    v = total_pairs / total_t
    sample = f"{per_step} primaries per step of the {wl.n}-particle catalogue: forward + analytic gradient"
    print(json.dumps(_reference_line(args, GRAD_METRIC, GRAD_WORKLOAD, wl.n, v, total_t, sample)), flush=True)


def run_reference(args, rank, world):
    from paper_2106_10278_gb300 import catalogs

    if rank != 0:
        return
    import oracle

    oracle.build()
    if args.workload == "batch64":
        return _reference_batch64(args)
    if args.workload == "d4n3-grad":
        return _reference_grad(args)
    wl = catalogs.workload(args.workload)
    import multiprocessing as mp

    # size one step at ~ (a few minutes / steps) of CPU time; every step runs the oracle, as it stands,
    # in one spawned process per host core, each on its own block of primaries
    host = os.cpu_count() or 1
    t0 = time.perf_counter()
    _oracle_estimate(wl, (0, 1))
    t1 = time.perf_counter() - t0
    per_proc = max(1, min(_reference_per_step(args, t1), wl.n // max(host, 1)))
    fd, path = tempfile.mkstemp(suffix=".npz")
    os.close(fd)
    total_pairs, total_t = 0, 0.0
    try:
        np.savez(path, D=wl.D, N=wl.N, lmax=wl.lmax, edges=wl.edges, box=wl.box, pos=wl.pos, w=wl.w,
                         geometry=wl.geometry)
        with mp.get_context("spawn").Pool(host, initializer=_oracle_worker_init, initargs=(path,)) as pool:
            for k in range(args.warmup):
                pool.map(_oracle_worker_block, [(i, i + 1) for i in range(host)])
            span = per_proc * host
            for k in range(args.steps):
                a = (k * span) % max(wl.n - span + 1, 1)
                blocks = [(a + i * per_proc, a + (i + 1) * per_proc) for i in range(host)]
                t0 = time.perf_counter()
                pool.map(_oracle_worker_block, blocks)
                total_t += time.perf_counter() - t0
                total_pairs += sum(count_pairs_numpy(wl.pos, wl.edges, wl.box, b, wl.geometry) for b in blocks)
    finally:
        os.unlink(path)
    v = total_pairs / total_t
    sample = (f"{host} processes x {per_proc} primaries per step of the {wl.n}-particle workload, all secondaries "
              "(the FP64 oracle, one spawned process per host core)")
    metric = METRIC if args.workload == "d3n4" else f"pairs/s and coupling terms/s, {args.workload}"
    workload = WORKLOAD if args.workload == "d3n4" else args.workload
    line = _reference_line(args, metric, workload, wl.n, v, total_t, sample)
    line["cpu_baseline"]["cores"] = host
    line["host_cores"] = host
    print(json.dumps(line), flush=True)


def run_ours(args, rank, world):
    import torch

    from paper_2106_10278_gb300 import build as pbuild
    from paper_2106_10278_gb300 import catalogs
    from paper_2106_10278_gb300.npcf import Plan

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if rank == 0:
        pbuild.build()
    if world > 1:
        torch.distributed.barrier()
    base_seed = {"d3n4": 2, "d2n3": 1, "d2n4": 1, "d4n3": 4, "d3n3_fp64": 0, "d3n5": 5, "s2n4": 6}[args.workload]
    wl = catalogs.workload(args.workload, seed=base_seed + 1000 * rank, scale=args.scale)
    prec = args.precision or ("fp64" if wl.precision == "fp64" else "fp32")
    tdt = torch.float64 if prec == "fp64" else torch.float32
    plan = Plan(wl.D, wl.N, wl.lmax, wl.edges, wl.box, precision=prec, sync_check=False, timing=True,
                geometry=wl.geometry)
    pos = torch.tensor(wl.pos, dtype=tdt, device=dev)
    w = torch.tensor(wl.w, dtype=tdt, device=dev)
    out = torch.empty(2 * plan.ncoeff, dtype=torch.float64, device=dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)  # 256 MB > L2
    stream = torch.cuda.current_stream(dev)
    # launch shapes chosen by the library's autotuner on a sample of this input (outside the timing)
    tuned = plan.tuned_config() if args.no_autotune else plan.autotune(pos, w)

    for _ in range(args.warmup):
        plan.compute(pos, w, out=out)
    torch.cuda.synchronize()
    st = plan.stats()
    counters = plan.counters()
    pairs_per_step = st["pairs"]
    nprim = st["primaries"]
    cand_per_step = st["candidates"]

    clocks = ClockSampler()
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    step_ms, pair_ms, couple_ms, cells_ms, launches = [], [], [], [], 0
    wall0 = time.perf_counter()
    for _ in range(args.steps):
        flush.fill_(1.0)  # evict L2 between timed steps (outside the events)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        plan.compute(pos, w, out=out)
        e1.record(stream)
        e1.synchronize()
        step_ms.append(e0.elapsed_time(e1))
        pr = plan.profile()
        pair_ms.append(pr["pairs_ms"])
        couple_ms.append(pr["couple_ms"])
        cells_ms.append(pr["cells_ms"])
        launches += pr["launches"]
    torch.cuda.synchronize()
    wall = time.perf_counter() - wall0
    if world > 1:
        torch.distributed.barrier()
    clk = clocks.stop()

    t_total = sum(step_ms) / 1e3
    if world > 1:
        tt = torch.tensor([t_total, float(pairs_per_step * args.steps)], dtype=torch.float64, device=dev)
        mx = tt.clone()
        torch.distributed.all_reduce(mx[:1], op=torch.distributed.ReduceOp.MAX)
        torch.distributed.all_reduce(tt[1:], op=torch.distributed.ReduceOp.SUM)
        t_max, all_pairs = float(mx[0]), float(tt[1])
    else:
        t_max, all_pairs = t_total, float(pairs_per_step * args.steps)
    value = all_pairs / t_max
    terms = coupling_terms_per_primary(wl.D, wl.N, wl.lmax, len(wl.edges) - 1)
    coeffs_per_s = world * nprim * terms * args.steps / t_max

    # roofline of the dominant kernel: the pair kernel, or the coupling where it takes longer
    # (both FP32 ALU bound)
    fpp = pair_flops_per_pair(wl.D, wl.lmax) + (SPHERE_EXTRA_FLOPS if wl.geometry == "sphere" else 0)
    pk_s = float(np.mean(pair_ms)) / 1e3
    ck_s = float(np.mean(couple_ms)) / 1e3
    sm_clock = 2070.0
    peak = SM_COUNT_NOMINAL * FP32_LANES_PER_SM * 2 * sm_clock * 1e6 / 1e12
    note = "152 SMs x 128 FP32 lanes x 2 flop x 2070 MHz (derived, FP32 CUDA cores)"
    if ck_s <= pk_s:
        achieved = fpp * pairs_per_step / pk_s / 1e12
        roofline = {"bound": "alu", "kernel": "k_pairs", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                    "frac": achieved / peak, "traffic": _traffic_from_profiles(args.workload),
                    "traffic_source": "ncu dram__bytes_read.sum + dram__bytes_write.sum per launch, committed in "
                                      f"profiles/k_pairs_{args.workload}.md for kernel sources {kernel_source_sha16()} "
                                      "(null when that summary was taken on other sources)", "peak_note": note,
                    "flops_per_pair": fpp, "pairs_per_launch": pairs_per_step,
                    "pair_kernel_ms": float(np.mean(pair_ms))}
    elif wl.N == 5:
        # the factored 5PCF coupling: its algorithmic work is the contraction over (primary, m12) of
        # X(row) Z(column) for every key, a complex multiply-add (8 flops) per key and m12 value
        k = plan.keys()
        macs = int(sum(2 * int(row[4 + 2]) + 1 for row in k))
        achieved = 8 * macs * nprim / ck_s / 1e12
        roofline = {"bound": "alu", "kernel": "k_d3n5_form + k_d3n5_contract (factored 5PCF)", "achieved": achieved,
                    "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak, "traffic": None, "peak_note": note,
                    "flops_per_primary": 8 * macs, "flops_note": "8 per key and m12 (complex multiply-add)",
                    "couple_kernel_ms": float(np.mean(couple_ms))}
        if prec == "mixed_bf16x3":
            roofline.update(d3n5_tensor_roofline(wl, ck_s))
    else:
        fpt = COUPLING_FLOPS_PER_TERM[wl.N]
        achieved = fpt * terms * nprim / ck_s / 1e12
        roofline = {"bound": "alu", "kernel": "k_couple (N=%d)" % wl.N, "achieved": achieved, "peak": peak,
                    "unit": "TFLOP/s", "frac": achieved / peak, "traffic": None, "peak_note": note,
                    "flops_per_term": fpt, "terms_per_launch": terms * nprim,
                    "couple_kernel_ms": float(np.mean(couple_ms))}

    # end to end through the public host-buffer entry point (pinned inputs)
    e2e = None
    if not args.no_e2e:
        hp = torch.tensor(wl.pos, dtype=tdt).pin_memory()
        hw = torch.tensor(wl.w, dtype=tdt).pin_memory()
        plan.compute_host(hp.numpy(), hw.numpy())  # warm
        e2e_t = []
        for _ in range(max(2, min(args.steps, 5))):
            flush.fill_(1.0)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            plan.compute_host(hp.numpy(), hw.numpy())
            e2e_t.append(time.perf_counter() - t0)
        e2e = {"value": world * pairs_per_step / float(np.mean(e2e_t)), "unit": "pairs/s",
               "h2d_bytes_per_step": int(hp.numel() * hp.element_size() + hw.numel() * hw.element_size()),
               "d2h_bytes_per_step": int(2 * plan.ncoeff * 8)}

    line = {
        "metric": METRIC if args.workload == "d3n4" else f"pairs/s and coupling terms/s, {args.workload}",
        "value": value, "unit": "pairs/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t_max * 1e3 / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": DTYPES[prec], "data": "synthetic",
        "config": {"workload": WORKLOAD if args.workload == "d3n4" else args.workload, "n": wl.n, "precision": prec,
                   "primaries": nprim, "pairs_per_step": pairs_per_step, "candidates_per_step": cand_per_step,
                   "ncoeff": plan.ncoeff,
                   "l2": "256 MB buffer written before every timed step (outside the events)"},
        "coeffs_per_s": coeffs_per_s, "coupling_terms_per_primary": terms, "pair_counters": counters,
        "tuned": tuned,
        "stages_ms": {"cells": float(np.mean(cells_ms)), "pairs": float(np.mean(pair_ms)),
                      "couple": float(np.mean(couple_ms))},
        "roofline": roofline, "e2e": e2e, "gpu_launches": launches, "clocks": clk,
        "wall_s_timed_region": wall,
    }
    if args.scale != 1.0:
        line["config"]["scale"] = args.scale
    if rank == 0 and args.workload == "d3n4" and not args.no_mixed_arm:
        # the D=3 4PCF has no tensor-core coupling (its contraction over primaries would need a
        # per-primary operand of 58,320 complex products, as costly as its CUDA-core kernel); the
        # metric's mixed-vs-FP32 comparison is measured on the D=2 4PCF, whose coupling runs there
        line["mixed_vs_fp32"] = mixed_arm(dev, "d2n4")
        line["mixed_vs_fp32_5pcf"] = mixed_arm(dev, "d3n5", oracle_prims=24)
    if rank == 0 and args.workload == "d3n5" and not args.no_mixed_arm and prec != "mixed_bf16x3":
        line["mixed_vs_fp32"] = mixed_arm(dev, "d3n5", oracle_prims=24)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        def gpu_range(a, b):  # the GPU's coefficients of primaries [a, b), for the per-result error
            z = plan.compute(pos, w, primaries=(a, b)).cpu().numpy()
            return z, plan.keys()

        cb = _cpu_baseline(wl, args.cpu_seconds, gpu_range)
        line["rel_err_vs_oracle"] = cb.pop("rel_err_vs_oracle", None)
        line["host_cores"] = cb["host_cores"]
        line["cpu_baseline"] = cb
    if rank == 0:
        print(json.dumps(line), flush=True)


def d3n5_tc_tiles(lmax, nbins):
    """The tiles of the tensor-core 5PCF contraction, as (l12, rows, columns): 128 rows x 64
    columns of one parity, rows (b2, b1, label pair) of the bin pairs b1 < b2 and label pairs
    (l1, l2) that couple to l12, columns (b3, b4, label pair) likewise for (l3, l4), each in
    ascending order; a tile is kept when its first row's b2 is below its last column's b3 (the
    plan's own tiling, restated)."""
    p12 = [(b1, b2) for b2 in range(1, nbins - 2) for b1 in range(b2)]
    p34 = [(b3, b4) for b3 in range(2, nbins - 1) for b4 in range(b3 + 1, nbins)]
    tiles = []
    for l12 in range(2 * lmax + 1):
        lx = [(a, b) for a in range(lmax + 1) for b in range(lmax + 1) if abs(a - b) <= l12 <= a + b]
        lz = [(a, b) for a in range(lmax + 1) for b in range(lmax + 1) if abs(l12 - a) <= b <= l12 + a]
        for par in (0, 1):
            rows = sorted((p[1], p[0], ab) for p in p12 for ab in lx if sum(ab) % 2 == par)
            cols = sorted((p[0], p[1], ab) for p in p34 for ab in lz if sum(ab) % 2 == par)
            for r0 in range(0, len(rows), 128):
                for c0 in range(0, len(cols), 64):
                    tr, tc = rows[r0:r0 + 128], cols[c0:c0 + 64]
                    if tr[0][0] < tc[-1][0]:
                        tiles.append((l12, tr, tc))
    return tiles


def d3n5_tc_k1_sum(lmax, nbins):
    """Sum over the tensor-core tiles of K per primary (2 l12 + 1)."""
    return sum(2 * l12 + 1 for l12, _, _ in d3n5_tc_tiles(lmax, nbins))


def d3n5_tensor_roofline(wl, couple_s):
    """Tensor-pipe rate of the BF16x3 5PCF contraction: MMA flops issued (6 MMAs of 128 x 128 per
    16 K elements: 2 x 128 x 128 x 6 flops per K element and tile, padding included) over the
    coupling stage (formation + contraction)."""
    mma = 6 * 2 * 128 * 128 * d3n5_tc_k1_sum(wl.lmax, len(wl.edges) - 1) * wl.n
    bf = _peaks().get("bf16_tflops")
    out = {"tensor_bound": "tensor", "tensor_kernel": "k_d3n5_contract_tc (bf16x3)",
           "tensor_achieved": mma / couple_s / 1e12, "tensor_peak": bf, "tensor_unit": "TFLOP/s",
           "tensor_peak_note": "MEASURED_PEAKS.json bf16_tflops (of measured)",
           "tensor_flops_note": "MMA flops issued per launch over the coupling stage (formation included)"}
    if bf:
        out["tensor_frac"] = out["tensor_achieved"] / bf
    return out


def mixed_arm(dev, name="d2n4", steps=5, oracle_prims=100):
    """The split-precision tensor-core coupling against the FP32 CUDA-core coupling, on the D=2 4PCF
    workload (200k points, 16 bins, lmax 10) or the paper's 5PCF example (10^4 points, 10 bins,
    lmax 4): coupling-stage times (CUDA events, median of `steps` after a warm-up), the speed-up,
    the error of each split against the FP32 result (every primary) and against the FP64 oracle
    (primaries [0, oracle_prims)), and the tensor pipe's rate."""
    import torch

    from paper_2106_10278_gb300 import catalogs
    from paper_2106_10278_gb300.npcf import Plan
    import oracle

    wl = catalogs.workload(name)
    pos = torch.tensor(wl.pos, dtype=torch.float32, device=dev)
    w = torch.tensor(wl.w, dtype=torch.float32, device=dev)
    keys, ref = oracle.estimate(wl.D, wl.N, wl.lmax, wl.edges, wl.box, wl.pos, wl.w, primaries=(0, oracle_prims))
    index = {tuple(int(x) for x in k): i for i, k in enumerate(keys)}
    desc = {"d2n4": "d2n4: D=2 4PCF, 200k points (100k uniform + 100k in 400 Gaussian blobs), 16 bins over "
                    "[0.002,0.05], lmax 10",
            "d3n5": "d3n5: D=3 5PCF, 10^4 uniform points in the periodic unit cube, 10 bins over [0.1,0.4], lmax 4"}
    out = {"workload": desc[name], "couple_ms": {}, "rel_err_vs_fp32": {}, "rel_err_vs_oracle": {},
           "oracle_primaries": oracle_prims}
    z32 = None
    precs = ("fp32", "mixed_bf16x3", "mixed_tf32x3") if name == "d2n4" else ("fp32", "mixed_bf16x3")
    for prec in precs:
        plan = Plan(wl.D, wl.N, wl.lmax, wl.edges, wl.box, precision=prec, sync_check=False, timing=True)
        plan.autotune(pos, w)
        z = plan.compute(pos, w).cpu().numpy()
        ms = []
        for _ in range(steps):
            plan.compute(pos, w)
            ms.append(plan.profile()["couple_ms"])
        zs = plan.compute(pos, w, primaries=(0, oracle_prims)).cpu().numpy()
        r = ref[np.array([index[tuple(int(x) for x in k)] for k in plan.keys()])]
        out["couple_ms"][prec] = float(np.median(ms))
        out["rel_err_vs_oracle"][prec] = float(np.linalg.norm(zs - r) / np.linalg.norm(r))
        if prec == "fp32":
            z32 = z
        else:
            out["rel_err_vs_fp32"][prec] = float(np.linalg.norm(z - z32) / np.linalg.norm(z32))
        if prec == "mixed_bf16x3":
            out["tuned_bf16x3"] = plan.tuned_config()
    t32 = out["couple_ms"]["fp32"]
    out["speedup_vs_fp32"] = {k: t32 / v for k, v in out["couple_ms"].items() if k != "fp32"}
    if name == "d3n5":
        out["tensor_roofline"] = d3n5_tensor_roofline(wl, out["couple_ms"]["mixed_bf16x3"] * 1e-3)
        return out
    # tensor-pipe rate of the BF16x3 kernel: MMA flops issued (3 split products over M=128 rows x N=32
    # columns x K=2 per primary and label set, padding included) over its time
    nprim, nlam = wl.n, 176
    mma_flops = 3 * 2 * 128 * 32 * 2 * nprim * nlam
    peaks = _peaks()
    bf = peaks.get("bf16_tflops")
    out["tensor_roofline"] = {"bound": "tensor", "kernel": "k_couple_d2n4_tc (bf16x3)",
                              "achieved": mma_flops / (out["couple_ms"]["mixed_bf16x3"] * 1e-3) / 1e12,
                              "peak": bf, "unit": "TFLOP/s", "peak_note": "MEASURED_PEAKS.json bf16_tflops (of measured)",
                              "flops_note": "MMA flops issued: 3 split products x 2 x 128 x 32 x 2 per primary and "
                                            "label set (176 label sets), padding included"}
    if bf:
        out["tensor_roofline"]["frac"] = out["tensor_roofline"]["achieved"] / bf
    return out


def _timed(args, world, step, flush, stream, after=None):
    """W untimed steps, then K steps each bracketed by CUDA events on `stream`
    (L2 flushed before each, outside the events); clocks sampled meanwhile.
    Returns (per-step ms, max over ranks of the summed seconds, wall s, clocks)."""
    import torch

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    clocks = ClockSampler()
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    ms = []
    wall0 = time.perf_counter()
    for _ in range(args.steps):
        flush.fill_(1.0)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        step()
        e1.record(stream)
        e1.synchronize()
        ms.append(e0.elapsed_time(e1))
        if after is not None:
            after()
    torch.cuda.synchronize()
    wall = time.perf_counter() - wall0
    if world > 1:
        torch.distributed.barrier()
    clk = clocks.stop()
    t = sum(ms) / 1e3
    if world > 1:
        tt = torch.tensor([t], dtype=torch.float64, device="cuda")
        torch.distributed.all_reduce(tt, op=torch.distributed.ReduceOp.MAX)
        t = float(tt[0])
    return ms, t, wall, clk


def _alu_peak():
    return SM_COUNT_NOMINAL * FP32_LANES_PER_SM * 2 * 2070.0 * 1e6 / 1e12


def run_batch64(args, rank, world):
    """The batched workload: 64 catalogues (sizes log-uniform in [5e4, 5e5], periodic cubes of side
    500-1000, half uniform and half lognormal-Poisson, 8 bins over [10, 120]); one step is the 3PCF at
    lmax 10 and the 4PCF at lmax 4 of every catalogue, one npcf_compute_batched call each."""
    import torch

    from paper_2106_10278_gb300 import build as pbuild
    from paper_2106_10278_gb300 import catalogs
    from paper_2106_10278_gb300.npcf import Plan

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if rank == 0:
        pbuild.build()
    if world > 1:
        torch.distributed.barrier()
    bw = catalogs.batch64(ncat=max(1, int(round(64 * min(1.0, args.scale)))))
    pos = torch.tensor(bw.pos, dtype=torch.float32, device=dev)
    w = torch.tensor(bw.w, dtype=torch.float32, device=dev)
    plans = [Plan(3, N, L, bw.edges, np.full(3, 1000.0), precision="fp32", sync_check=False, timing=True)
             for N, L in ((3, 10), (4, 4))]
    outs = [torch.empty(bw.ncat * 2 * p.ncoeff, dtype=torch.float64, device=dev) for p in plans]
    # launch shapes tuned on the largest catalogue (outside the timing); the batched calls use them
    big = int(np.argmax(np.diff(bw.offsets)))
    a0, a1 = int(bw.offsets[big]), int(bw.offsets[big + 1])
    tuned = [p.tuned_config() if args.no_autotune else p.autotune(pos[a0:a1], w[a0:a1]) for p in plans]
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev)
    prof = []

    def step():
        for p, o in zip(plans, outs):
            p.compute_batched(pos, w, bw.offsets, bw.boxes, out=o)

    def after():  # stage times of the step just timed (each plan reports its last call)
        prof.append([p.profile() for p in plans])

    ms, t_max, wall, clk = _timed(args, world, step, flush, stream, after)
    pairs = plans[0].stats()["pairs"]
    prof = prof[-args.steps:]
    pair_ms = [float(np.mean([pp[i]["pairs_ms"] for pp in prof])) for i in range(2)]
    couple_ms = [float(np.mean([pp[i]["couple_ms"] for pp in prof])) for i in range(2)]
    launches = sum(pp[i]["launches"] for pp in prof for i in range(2))
    fpp = pair_flops_per_pair(3, 10)
    achieved = fpp * pairs / (pair_ms[0] / 1e3) / 1e12
    value = world * pairs * args.steps / t_max
    line = {
        "metric": BATCH_METRIC, "value": value,
        "unit": "pairs/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": t_max * 1e3 / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32", "data": "synthetic",
        "config": {"workload": batch_workload(bw.ncat, len(bw.pos)),
                   "pairs_per_step": pairs, "ncoeff": [p.ncoeff for p in plans],
                   "l2": "256 MB buffer written before every timed step (outside the events)"},
        "stages_ms": {"pairs_3pcf_l10": pair_ms[0], "couple_3pcf": couple_ms[0], "pairs_4pcf_l4": pair_ms[1],
                      "couple_4pcf": couple_ms[1]},
        "roofline": {"bound": "alu", "kernel": "k_pairs (lmax 10)", "achieved": achieved, "peak": _alu_peak(),
                     "unit": "TFLOP/s", "frac": achieved / _alu_peak(), "traffic": None,
                     "flops_per_pair": fpp, "pairs_per_launch": pairs, "pair_kernel_ms": pair_ms[0]},
        "gpu_launches": launches, "clocks": clk, "wall_s_timed_region": wall, "tuned": tuned,
    }
    if rank == 0:
        print(json.dumps(line), flush=True)


def run_grad(args, rank, world):
    """One gradient step of the D=4 3PCF workload (n=100k in the unit 4-cube, 8 bins over [0.01, 0.12],
    lmax 4, FP32): coefficients, the chi^2 upstream gradient 2 (zeta - t) against the seed-104 catalogue's
    coefficients, and dL/dpos, dL/dw through npcf_backward."""
    import torch

    from paper_2106_10278_gb300 import build as pbuild
    from paper_2106_10278_gb300 import catalogs
    from paper_2106_10278_gb300.npcf import Plan

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if rank == 0:
        pbuild.build()
    if world > 1:
        torch.distributed.barrier()
    wl = catalogs.workload("d4n3", seed=4 + 1000 * rank, scale=args.scale)
    tgt = catalogs.workload("d4n3", seed=104, scale=args.scale)
    plan = Plan(4, 3, 4, wl.edges, wl.box, precision="fp32", sync_check=False, timing=True)
    pos = torch.tensor(wl.pos, dtype=torch.float32, device=dev)
    w = torch.tensor(wl.w, dtype=torch.float32, device=dev)
    t = plan.compute(torch.tensor(tgt.pos, dtype=torch.float32, device=dev),
                     torch.tensor(tgt.w, dtype=torch.float32, device=dev)).clone()
    out = torch.empty(2 * plan.ncoeff, dtype=torch.float64, device=dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev)
    tuned = plan.tuned_config() if args.no_autotune else plan.autotune(pos, w)
    ev = {}
    bwd_ms, bwd_launches = [], []

    def step():
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        z = plan.compute(pos, w, out=out)
        g = torch.view_as_real(2.0 * (z - t)).reshape(-1)
        a.record(stream)
        plan.backward(pos, w, g)
        b.record(stream)
        ev["bwd"] = (a, b)

    bwd_stages = []

    def after():
        bwd_ms.append(ev["bwd"][0].elapsed_time(ev["bwd"][1]))
        pr = plan.profile()  # the backward call's stages
        bwd_launches.append(pr["launches"])
        bwd_stages.append([pr["cells_ms"], pr["pairs_ms"], pr["couple_ms"], pr["reduce_ms"]])

    ms, t_max, wall, clk = _timed(args, world, step, flush, stream, after)
    torch.cuda.synchronize()
    pairs = plan.stats()["pairs"]
    plan.compute(pos, w, out=out)  # one more forward (untimed) for its stage times and launch count
    fwd = plan.profile()
    bwd_ms = float(np.mean(bwd_ms))
    value = world * pairs * args.steps / t_max
    line = {
        "metric": GRAD_METRIC, "value": value, "unit": "pairs/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_max * 1e3 / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": GRAD_WORKLOAD, "n": wl.n, "pairs_per_step": pairs,
                   "l2": "256 MB buffer written before every timed step (outside the events)"},
        "stages_ms": {"forward_pairs": fwd["pairs_ms"], "forward_couple": fwd["couple_ms"], "backward": bwd_ms,
                      "backward_stages": dict(zip(("cells", "pair_recompute", "couple_adjoint", "pair_adjoint"),
                                                  np.mean(bwd_stages, axis=0).tolist()))},
        "roofline": {"bound": "alu", "kernel": "npcf_backward (cell list, pair recompute, adjoint kernels)",
                     "achieved": adjoint_flops_per_pair(4, 4) * pairs / (bwd_ms / 1e3) / 1e12, "peak": _alu_peak(),
                     "unit": "TFLOP/s", "traffic": None, "flops_per_pair": adjoint_flops_per_pair(4, 4),
                     "note": "achieved counts the adjoint pair work only, over the whole backward call"},
        "gpu_launches": args.steps * fwd["launches"] + sum(bwd_launches), "clocks": clk,
        "wall_s_timed_region": wall, "tuned": tuned,
    }
    line["roofline"]["frac"] = line["roofline"]["achieved"] / line["roofline"]["peak"]
    if args.scale != 1.0:
        line["config"]["scale"] = args.scale
    if rank == 0:
        print(json.dumps(line), flush=True)


def main():
    args = _args()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    if world > 1:
        import torch

        torch.distributed.init_process_group("nccl")
    try:
        if args.workload == "batch64":
            run_batch64(args, rank, world)
        elif args.workload == "d4n3-grad":
            run_grad(args, rank, world)
        else:
            run_ours(args, rank, world)
    finally:
        if world > 1:
            import torch

            torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
