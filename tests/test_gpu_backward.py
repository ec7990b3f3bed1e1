"""The adjoint (npcf_backward) against the FP64 gradient oracle, through the C ABI.

The loss is L = sum_c Re(g_c) Re(zeta_c) + Im(g_c) Im(zeta_c) for a seeded
upstream gradient g; the oracle differentiates the closed-form N=3 estimator
(addition theorem for D >= 3, relative-angle exponential for D = 2) with the
radial bins held fixed.  Tolerances: FP64 plans max |gpu - oracle| <= 1e-10 *
max |oracle|; FP32 plans ||gpu - oracle||_2 <= 1e-5 ||oracle||_2 (the
estimator's own bounds).  Pair sets agree exactly (the adjoint decides bins
with the forward kernel's routine).
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


def _plan(D, lmax, edges, box, precision, **kw):
    from paper_2106_10278_gb300.npcf import Plan

    return Plan(D, 3, lmax, edges, box, precision=precision, **kw)


def _catalog(D, n, seed, fp32=True):
    """Half uniform, half in Gaussian blobs; FP32-representable, or with a full FP64 mantissa for FP64 plans."""
    pos = np.concatenate([catalogs.uniform(n // 2, D, 1.0, seed, fp32=fp32),
                          catalogs.gaussian_blobs(n - n // 2, D, 1.0, 5, 0.04, seed + 1, fp32=fp32)])
    w = catalogs.normal_weights(n, 1.0, 0.3, seed + 2, fp32=fp32)
    return pos, w


def _upstream(plan, keys, seed):
    """A seeded complex upstream gradient over the oracle's keys and the same one in the plan's order."""
    g = np.random.default_rng(seed)
    gk = g.normal(size=len(keys)) + 1j * g.normal(size=len(keys))
    index = {tuple(int(x) for x in k): i for i, k in enumerate(keys)}
    order = np.array([index[tuple(int(x) for x in k)] for k in plan.keys()])
    gp = np.empty(2 * len(order))
    gp[0::2] = gk[order].real
    gp[1::2] = gk[order].imag
    return gk, gp


def _gpu_backward(plan, pos, w, gflat, primaries=None):
    dt = torch.float64 if plan.precision == "fp64" else torch.float32
    tp = torch.tensor(pos, dtype=dt, device="cuda")
    tw = torch.tensor(w, dtype=dt, device="cuda")
    tg = torch.tensor(gflat, dtype=torch.float64, device="cuda")
    gp, gw = plan.backward(tp, tw, tg, primaries=primaries)
    torch.cuda.synchronize()
    return gp.double().cpu().numpy(), gw.double().cpu().numpy()


def _check(precision, got, ref, what):
    if precision == "fp64":
        err = np.max(np.abs(got - ref))
        scale = np.max(np.abs(ref))
        assert err <= TOL64 * scale, f"{what}: max err {err:.3e} vs scale {scale:.3e}"
    else:
        err = np.linalg.norm(got - ref)
        scale = np.linalg.norm(ref)
        assert err <= TOL32 * scale, f"{what}: rel err {err / scale:.3e}"
    assert scale > 0


def _compare(D, lmax, edges, box, pos, w, precision, primaries=None, periodic=True, seed=0):
    plan = _plan(D, lmax, edges, box, precision, periodic=periodic)
    keys, _ = oracle.estimate_n3_closed(D, lmax, edges, box, pos, w, periodic=periodic, primaries=primaries)
    gk, gflat = _upstream(plan, keys, seed)
    _, _, rp, rw = oracle.estimate_n3_closed(D, lmax, edges, box, pos, w, periodic=periodic, primaries=primaries,
                                             grad_coeffs=gk)
    gp, gw = _gpu_backward(plan, pos, w, gflat, primaries)
    _check(precision, gp, rp, "grad_pos")
    _check(precision, gw, rw, "grad_w")
    return plan, gp, gw


CASES = [
    # D, lmax, nbins, n, r_max
    (2, 6, 8, 1500, 0.2),
    (2, 10, 6, 1200, 0.15),
    (3, 5, 10, 1500, 0.2),
    (3, 3, 4, 1500, 0.25),
    (4, 3, 6, 1200, 0.3),
    (4, 2, 3, 1000, 0.3),
]


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("D,lmax,nbins,n,rmax", CASES)
def test_backward_small(D, lmax, nbins, n, rmax, precision):
    pos, w = _catalog(D, n, 10 * D + lmax, fp32=precision == "fp32")
    edges = np.linspace(0.02, rmax, nbins + 1)
    _compare(D, lmax, edges, np.ones(D), pos, w, precision, seed=D + lmax)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_backward_primary_range_and_open_box(precision):
    pos, w = _catalog(3, 1500, 77, fp32=precision == "fp32")
    pos = pos * 0.96 + 0.02
    if precision == "fp32":
        pos = pos.astype(np.float32).astype(np.float64)
    edges = np.linspace(0.03, 0.22, 7)
    _compare(3, 4, edges, np.ones(3), pos, w, precision, primaries=(200, 900), seed=5)
    _compare(3, 4, edges, np.ones(3), pos, w, precision, periodic=False, seed=6)


def test_backward_full_size_sampled():
    """The 1M-galaxy + 1M-random D=3 catalogue (box 1000, 10 bins over [20, 160], lmax 5, FP32),
    sampled one primary at a time.  For a single primary j the coefficients are linear in w_j and
    quadratic in every secondary weight, so dL/dw_j = L/w_j and a central difference in w_k with
    any step is exact; position derivatives are checked by central differences away from bin
    edges.  All values come from the FP64 oracle's coefficients."""
    wl = catalogs.workload("d3n4")
    pos, w, edges, box = wl.pos, wl.w, wl.edges, wl.box
    plan = _plan(3, 5, edges, box, "fp32")
    tp = torch.tensor(pos, dtype=torch.float32, device="cuda")
    tw = torch.tensor(w, dtype=torch.float32, device="cuda")
    rng = np.random.default_rng(17)
    for j in (123456, 1500001):
        prims = (j, j + 1)
        keys, z0 = oracle.estimate(3, 3, 5, edges, box, pos, w, primaries=prims)
        gk, gflat = _upstream(plan, keys, j)

        def loss(p, ww):
            _, zz = oracle.estimate(3, 3, 5, edges, box, p, ww, primaries=prims)
            return float(np.sum(gk.real * zz.real + gk.imag * zz.imag))

        L0 = float(np.sum(gk.real * z0.real + gk.imag * z0.imag))
        gp, gw = plan.backward(tp, tw, torch.tensor(gflat, device="cuda"), primaries=prims)
        gp = gp.double().cpu().numpy()
        gw = gw.double().cpu().numpy()
        assert abs(gw[j] - L0 / w[j]) <= TOL32 * abs(L0 / w[j])
        sec = np.flatnonzero(gw)
        sec = sec[sec != j]
        assert len(sec) > 1000
        wscale = np.max(np.abs(gw[sec]))
        for k in rng.choice(sec, 2, replace=False):
            wp = w.copy(); wp[k] += 1.0
            wm = w.copy(); wm[k] -= 1.0
            fd = (loss(pos, wp) - loss(pos, wm)) / 2.0
            assert abs(gw[k] - fd) <= TOL32 * wscale, (k, gw[k], fd)
        # a secondary whose separation is far from every edge
        d = pos[sec] - pos[j]
        d -= box * np.round(d / box)
        r = np.linalg.norm(d, axis=1)
        far = sec[np.min(np.abs(r[:, None] - edges[None, :]), axis=1) > 0.5]
        k = int(rng.choice(far))
        pscale = np.max(np.abs(gp[sec]))
        h = 1e-2
        for a in range(3):
            pp = pos.copy(); pp[k, a] += h
            pm = pos.copy(); pm[k, a] -= h
            fd = (loss(pp, w) - loss(pm, w)) / (2 * h)
            assert abs(gp[k, a] - fd) <= TOL32 * pscale, (k, a, gp[k, a], fd)
        # the primary's position gradient balances its secondaries' (translation invariance)
        np.testing.assert_allclose(gp[j], gp[j] - gp.sum(axis=0), rtol=0, atol=1e-6 * np.abs(gp).sum())
    # every particle, 20000 primaries: translation invariance and cubic weight homogeneity
    prims = (0, 20000)
    z = plan.compute(tp, tw, primaries=prims)
    g = torch.randn(2 * plan.ncoeff, dtype=torch.float64, device="cuda", generator=torch.Generator("cuda").manual_seed(3))
    L = float((torch.view_as_real(z).reshape(-1) * g).sum())
    gp, gw = plan.backward(tp, tw, g, primaries=prims)
    gp, gw = gp.double(), gw.double()
    assert gp.sum(dim=0).abs().max().item() <= 1e-6 * gp.abs().sum().item()
    hom = float((tw.double() * gw).sum())
    assert abs(hom - 3 * L) <= TOL32 * float((tw.double() * gw).abs().sum())


@pytest.mark.parametrize("D", [2, 3, 4])
def test_backward_identities_at_scale(D):
    """Properties that hold at any size: sum_i dL/dy_i = 0 (translation invariance of a periodic
    catalogue) and sum_i w_i dL/dw_i = 3 L (zeta is cubic in the weights), with L from the forward."""
    n = {2: 60000, 3: 60000, 4: 40000}[D]
    pos, w = _catalog(D, n, 300 + D, fp32=False)
    lmax = {2: 8, 3: 5, 4: 3}[D]
    edges = np.linspace(0.005, {2: 0.03, 3: 0.06, 4: 0.12}[D], 9)
    plan = _plan(D, lmax, edges, np.ones(D), "fp64")
    tp = torch.tensor(pos, dtype=torch.float64, device="cuda")
    tw = torch.tensor(w, dtype=torch.float64, device="cuda")
    z = plan.compute(tp, tw)
    g = torch.randn(2 * plan.ncoeff, dtype=torch.float64, device="cuda", generator=torch.Generator("cuda").manual_seed(D))
    L = float((torch.view_as_real(z).reshape(-1) * g).sum())
    gp, gw = plan.backward(tp, tw, g)
    torch.cuda.synchronize()
    s = gp.sum(dim=0).abs().max().item()
    assert s <= 1e-10 * gp.abs().sum().item()
    hom = float((tw * gw).sum())
    assert abs(hom - 3 * L) <= 1e-10 * float((tw * gw).abs().sum())


def test_autograd_function_matches_backward():
    pos, w = _catalog(3, 1200, 9, fp32=False)
    edges = np.linspace(0.02, 0.2, 6)
    plan = _plan(3, 4, edges, np.ones(3), "fp64")
    tp = torch.tensor(pos, dtype=torch.float64, device="cuda", requires_grad=True)
    tw = torch.tensor(w, dtype=torch.float64, device="cuda", requires_grad=True)
    fn = plan.function()
    out = fn(tp, tw)
    assert out.shape == (plan.ncoeff, 2)
    G = torch.randn(plan.ncoeff, 2, dtype=torch.float64, device="cuda")
    (out * G).sum().backward()
    gp, gw = plan.backward(tp.detach(), tw.detach(), G.reshape(-1))
    torch.cuda.synchronize()
    assert torch.equal(out, torch.view_as_real(plan.compute(tp.detach(), tw.detach())))
    np.testing.assert_allclose(tp.grad.cpu().numpy(), gp.cpu().numpy(), rtol=0, atol=1e-12 * gp.abs().max().item())
    np.testing.assert_allclose(tw.grad.cpu().numpy(), gw.cpu().numpy(), rtol=0, atol=1e-12 * gw.abs().max().item())


def test_backward_rejections_and_empty():
    from paper_2106_10278_gb300.npcf import NpcfError

    edges = np.linspace(0.02, 0.2, 5)
    p4 = _plan(3, 2, edges, np.ones(3), "fp64")
    pos = torch.rand(100, 3, dtype=torch.float64, device="cuda")
    w = torch.ones(100, dtype=torch.float64, device="cuda")
    g = torch.zeros(2 * p4.ncoeff, dtype=torch.float64, device="cuda")
    with pytest.raises(NpcfError) as e:
        p4.backward(pos, w, g, want_pos=False, want_w=False)
    assert e.value.status == -1
    with pytest.raises(NpcfError) as e:
        p4.backward(pos, w, g, primaries=(50, 120))
    assert e.value.status == -1
    from paper_2106_10278_gb300.npcf import Plan

    n4 = Plan(3, 4, 2, edges, np.ones(3), precision="fp64")
    with pytest.raises(NpcfError) as e:
        n4.backward(pos, w, torch.zeros(2 * n4.ncoeff, dtype=torch.float64, device="cuda"))
    assert e.value.status == -2
    gp, gw = p4.backward(pos[:0], w[:0], g)
    assert gp.shape == (0, 3) and gw.shape == (0,)
    # a single particle has no pair: zero gradient
    gp, gw = p4.backward(pos[:1], w[:1], g)
    torch.cuda.synchronize()
    assert float(gp.abs().sum()) == 0.0 and float(gw.abs().sum()) == 0.0


def _d4_chi2_inputs(primaries):
    """The D=4 3PCF gradient workload (n=100k in the unit 4-cube: 50k uniform + 50k in 200 Gaussian blobs,
    8 bins over [0.01, 0.12], lmax 4) and a chi^2 loss against the coefficients of the seed-104 catalogue."""
    wl = catalogs.workload("d4n3")
    tgt = catalogs.workload("d4n3", seed=104)
    keys, z = oracle.estimate_n3_closed(4, 4, wl.edges, wl.box, wl.pos, wl.w, primaries=primaries)
    _, t = oracle.estimate_n3_closed(4, 4, tgt.edges, tgt.box, tgt.pos, tgt.w, primaries=primaries)
    return wl, keys, 2.0 * (z - t)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_backward_d4_chi2_workload_sampled(precision):
    prims = (0, 400)
    wl, keys, gk = _d4_chi2_inputs(prims)
    _, _, rp, rw = oracle.estimate_n3_closed(4, 4, wl.edges, wl.box, wl.pos, wl.w, primaries=prims, grad_coeffs=gk)
    plan = _plan(4, 4, wl.edges, wl.box, precision)
    index = {tuple(int(x) for x in k): i for i, k in enumerate(keys)}
    order = np.array([index[tuple(int(x) for x in k)] for k in plan.keys()])
    gflat = np.zeros(2 * plan.ncoeff)
    gflat[0::2] = gk[order].real
    gflat[1::2] = gk[order].imag
    w = wl.w if precision == "fp64" else wl.w.astype(np.float32).astype(np.float64)
    if precision == "fp32":  # the oracle sees the weights the FP32 plan sees
        _, _, rp, rw = oracle.estimate_n3_closed(4, 4, wl.edges, wl.box, wl.pos, w, primaries=prims, grad_coeffs=gk)
    gp, gw = _gpu_backward(plan, wl.pos, w, gflat, prims)
    _check(precision, gp, rp, "grad_pos")
    _check(precision, gw, rw, "grad_w")


def test_backward_d4_chi2_central_differences():
    """Every primary of the D=4 workload in FP64: the adjoint against central differences (h=1e-5) of the
    forward chi^2 loss on 64 coordinates (of particles with no pair within 2h of an edge) and 64 weights."""
    wl = catalogs.workload("d4n3")
    tgt = catalogs.workload("d4n3", seed=104)
    plan = _plan(4, 4, wl.edges, wl.box, "fp64")
    dev = lambda a: torch.tensor(a, dtype=torch.float64, device="cuda")
    t = plan.compute(dev(tgt.pos), dev(tgt.w)).clone()

    def loss(p, ww):
        z = plan.compute(dev(p), dev(ww))
        return float((z - t).abs().pow(2).sum())

    tp, tw = dev(wl.pos), dev(wl.w)
    z = plan.compute(tp, tw)
    g = torch.view_as_real(2.0 * (z - t)).reshape(-1).contiguous()
    gp, gw = plan.backward(tp, tw, g)
    gp, gw = gp.cpu().numpy(), gw.cpu().numpy()
    rng = np.random.default_rng(23)
    h = 1e-5
    safe = []
    for i in rng.permutation(wl.n):
        d = wl.pos - wl.pos[i]
        d -= np.round(d)
        r = np.linalg.norm(d, axis=1)
        r[i] = 1.0
        if np.min(np.abs(r[:, None] - wl.edges[None, :])) > 2 * h:
            safe.append(int(i))
        if len(safe) == 16:
            break
    pscale = np.max(np.abs(gp))
    for i in safe:
        for a in range(4):
            pp = wl.pos.copy(); pp[i, a] += h
            pm = wl.pos.copy(); pm[i, a] -= h
            fd = (loss(pp, wl.w) - loss(pm, wl.w)) / (2 * h)
            assert abs(fd - gp[i, a]) <= 1e-6 * pscale, (i, a, fd, gp[i, a])
    wscale = np.max(np.abs(gw))
    for i in rng.choice(wl.n, 64, replace=False):
        wp = wl.w.copy(); wp[i] += h
        wm = wl.w.copy(); wm[i] -= h
        fd = (loss(wl.pos, wp) - loss(wl.pos, wm)) / (2 * h)
        assert abs(fd - gw[i]) <= 1e-6 * wscale, (i, fd, gw[i])
