"""FP64 CPU oracle for the isotropic NPCF estimator (arXiv:2106.10278).

TEST INFRASTRUCTURE ONLY.  Only the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  It shares no code
with the CUDA library in ``paper_2106_10278_gb300`` and imports nothing from it.

The arithmetic lives in ``npcf_oracle.c`` (plain C, FP64, no fused
multiply-add); this module compiles it with gcc and exposes it through ctypes.
Every function below states the passage of the paper it follows; see the C
file for the readings taken where the paper is silent.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "npcf_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

_i32 = ctypes.c_int
_i64 = ctypes.c_int64
_f64 = ctypes.c_double
_pd = ctypes.POINTER(ctypes.c_double)
_pi = ctypes.POINTER(ctypes.c_int)


def build(force: bool = False) -> str:
    """Compile the oracle into ``oracle/_build/liboracle.so`` (gcc, -O2, no FMA contraction)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build())
        lib.npcf_oracle_nstates.argtypes = [_i32, _i32]
        lib.npcf_oracle_states.argtypes = [_i32, _i32, _pi]
        lib.npcf_oracle_harmonics.argtypes = [_i32, _i32, _pd, _i64, _pd]
        lib.npcf_oracle_wigner3j.argtypes = [_i32] * 6
        lib.npcf_oracle_wigner3j.restype = _f64
        lib.npcf_oracle_cg_d3.argtypes = [_i32] * 6
        lib.npcf_oracle_cg_d3.restype = _f64
        lib.npcf_oracle_ferrers_int.argtypes = [_i32, _i32, _f64]
        lib.npcf_oracle_ferrers_int.restype = _f64
        lib.npcf_oracle_ferrers_half.argtypes = [_i32, _i32, _f64]
        lib.npcf_oracle_ferrers_half.restype = _f64
        lib.npcf_oracle_nkeys.argtypes = [_i32, _i32, _i32, _i32, _i32]
        lib.npcf_oracle_keys.argtypes = [_i32, _i32, _i32, _i32, _i32, _pi]
        lib.npcf_oracle_coupling.argtypes = [_i32, _i32, _i32, _i32, _pi, _pd]
        lib.npcf_oracle_estimate.argtypes = [_i32, _i32, _i32, _i32, _i32, _pd, _pd, _i32, _pd, _pd, _i64,
                                             _i64, _i64, _i32, _pd]
        lib.npcf_oracle_estimate_ex.argtypes = [_i32, _i32, _i32, _i32, _i32, _pd, _pd, _i32, _pd, _pd, _i64,
                                                _i64, _i64, _i32, _i32, _pd]
        lib.npcf_oracle_n3_closed.argtypes = [_i32, _i32, _i32, _i32, _pd, _pd, _i32, _pd, _pd, _i64, _i64,
                                              _i64, _pd, _pd, _pd, _pd]
        lib.npcf_oracle_sphere_estimate.argtypes = [_i32, _i32, _i32, _i32, _pd, _pd, _pd, _i64, _i64, _i64, _i32,
                                                    _pd]
        lib.npcf_oracle_aniso_nkeys.argtypes = [_i32, _i32, _i32, _i32]
        lib.npcf_oracle_aniso_keys.argtypes = [_i32, _i32, _i32, _i32, _pi]
        lib.npcf_oracle_aniso_estimate.argtypes = [_i32, _i32, _i32, _i32, _pd, _pd, _i32, _pd, _pd, _i64, _i64, _i64,
                                                   _i32, _pd]
        lib.npcf_oracle_grid_alm.argtypes = [_i32, _i32, _i32, _pd, _pd, _pi, _pd, _pd]
        lib.npcf_oracle_grid_estimate.argtypes = [_i32, _i32, _i32, _i32, _i32, _pd, _pd, _pi, _pd, _pd]
        _lib = lib
        return lib


def _dp(a: np.ndarray):
    return a.ctypes.data_as(_pd)


def _ip(a: np.ndarray):
    return a.ctypes.data_as(_pi)


def states(D: int, lmax: int) -> np.ndarray:
    """Index vectors (l_1, .., l_{D-1}) obeying eq. selection-rules, in the oracle's order (padded to 3)."""
    lib = _load()
    ns = lib.npcf_oracle_nstates(D, lmax)
    out = np.zeros((ns, 3), dtype=np.int32)
    lib.npcf_oracle_states(D, lmax, _ip(out))
    return out


def harmonics(D: int, lmax: int, dirs: np.ndarray) -> np.ndarray:
    """Y_l(d/|d|) of eq. hypersph-def for every state and direction: complex (nd, nstates)."""
    lib = _load()
    d = np.ascontiguousarray(dirs, dtype=np.float64).reshape(-1, D)
    ns = lib.npcf_oracle_nstates(D, lmax)
    out = np.zeros((d.shape[0], ns, 2))
    lib.npcf_oracle_harmonics(D, lmax, _dp(d), d.shape[0], _dp(out))
    return out[..., 0] + 1j * out[..., 1]


def wigner3j(j1, j2, j3, m1, m2, m3) -> float:
    """Wigner 3j symbol by the Racah formula (DLMF 34.2.4)."""
    return _load().npcf_oracle_wigner3j(j1, j2, j3, m1, m2, m3)


def cg_d3(l1, m1, l2, m2, L, M) -> float:
    """D=3 Clebsch-Gordan coefficient as printed in eq. CG-examples."""
    return _load().npcf_oracle_cg_d3(l1, m1, l2, m2, L, M)


def ferrers_int(n: int, mu: int, x: float) -> float:
    """Ferrers function P^mu_n(x), integer degree and order (DLMF 14.6.1, 14.9.3)."""
    return _load().npcf_oracle_ferrers_int(n, mu, x)


def ferrers_half(L: int, k: int, theta: float) -> float:
    """Ferrers function P^{-(k+1/2)}_{L+1/2}(cos theta) (DLMF 14.5.11-12, 14.10.1)."""
    return _load().npcf_oracle_ferrers_half(L, k, theta)


def keys(D: int, N: int, lmax: int, nbins: int, bin_lt: bool = False) -> np.ndarray:
    """Output keys in the oracle's order: (b1, b2, b3, l1, l2, l3) for N <= 4 (unused bins -1,
    unused ells 0); (b1, b2, b3, b4, l1, l2, l12, l3, l4) for N = 5."""
    lib = _load()
    nk = lib.npcf_oracle_nkeys(D, N, lmax, nbins, int(bin_lt))
    if nk < 0:
        raise ValueError(f"unsupported (D={D}, N={N}, lmax={lmax}, nbins={nbins})")
    out = np.zeros((max(nk, 1), 9), dtype=np.int32)
    lib.npcf_oracle_keys(D, N, lmax, nbins, int(bin_lt), _ip(out))
    out = out[:nk]
    return out if N == 5 else out[:, [0, 1, 2, 4, 5, 6]].copy()


def coupling_terms(D: int, N: int, lmax: int, lam_index: int):
    """Non-zero terms (state indices, C^{Lambda;0}) of eq. Coupling-C for one Lambda."""
    lib = _load()
    nt = lib.npcf_oracle_coupling(D, N, lmax, lam_index, None, None)
    if nt < 0:
        raise ValueError("bad lambda")
    s = np.zeros((max(nt, 1), 4), dtype=np.int32)
    c = np.zeros(max(nt, 1))
    lib.npcf_oracle_coupling(D, N, lmax, lam_index, _ip(s), _dp(c))
    return (s[:nt] if N == 5 else s[:nt, :3].copy()), c[:nt]


def _prep(pos, w, edges, box):
    pos = np.ascontiguousarray(pos, dtype=np.float64)
    w = np.ascontiguousarray(w, dtype=np.float64)
    edges = np.ascontiguousarray(edges, dtype=np.float64)
    box = np.ascontiguousarray(box, dtype=np.float64)
    return pos, w, edges, box


def estimate(D, N, lmax, edges, box, pos, w, *, periodic=True, primaries=None, brute=False, bin_lt=False,
             remove_self=False):
    """The isotropic NPCF coefficients zeta^{0,b}_Lambda (N = 3: D = 2..4; N = 4: D = 2, 3;
    N = 5: D = 3, lmax <= 6).

    brute=False: the separable estimator, eq. NPCF-estimator-discrete.
    brute=True:  the naive sum over N-tuplets, eq. NPCF-estimator-intro-discrete
                 with the basis of eq. B-hypersph.
    primaries: (begin, end) range of primary particles (all particles are secondaries).
    remove_self: exclude the tuples whose secondaries coincide (only N=3 keys with b1 = b2 have
                 them); by default they are kept, as in the naive N-tuplet sum.
    Returns (keys, complex coefficients) in the oracle's key order.
    """
    lib = _load()
    pos, w, edges, box = _prep(pos, w, edges, box)
    n = pos.shape[0]
    pb, pe = (0, n) if primaries is None else primaries
    nbins = len(edges) - 1
    k = keys(D, N, lmax, nbins, bin_lt)
    out = np.zeros((k.shape[0], 2))
    rc = lib.npcf_oracle_estimate_ex(D, N, lmax, nbins, int(bin_lt), _dp(edges), _dp(box), int(periodic),
                                     _dp(pos), _dp(w), n, pb, pe, int(brute), int(remove_self), _dp(out))
    if rc < 0:
        raise ValueError(f"oracle estimate failed ({rc})")
    return k, out[:, 0] + 1j * out[:, 1]


def estimate_n3_closed(D, lmax, edges, box, pos, w, *, periodic=True, primaries=None, bin_lt=False,
                       grad_coeffs=None):
    """N=3 coefficients through the addition theorem (D in {3, 4}) or the plain
    exponential of the relative angle (D = 2).

    With grad_coeffs (complex array over keys, or real) also returns the
    gradient of L = sum_c Re(grad_c) Re(zeta_c) + Im(grad_c) Im(zeta_c) in
    positions and weights (radial bins held fixed).
    Returns (keys, zeta) or (keys, zeta, grad_pos, grad_w).
    """
    lib = _load()
    pos, w, edges, box = _prep(pos, w, edges, box)
    n = pos.shape[0]
    pb, pe = (0, n) if primaries is None else primaries
    nbins = len(edges) - 1
    k = keys(D, 3, lmax, nbins, bin_lt)
    out = np.zeros((k.shape[0], 2))
    if grad_coeffs is None:
        rc = lib.npcf_oracle_n3_closed(D, lmax, nbins, int(bin_lt), _dp(edges), _dp(box), int(periodic), _dp(pos),
                                       _dp(w), n, pb, pe, None, _dp(out), None, None)
        if rc < 0:
            raise ValueError(f"oracle failed ({rc})")
        return k, out[:, 0] + 1j * out[:, 1]
    g = np.zeros((k.shape[0], 2))
    gc = np.asarray(grad_coeffs)
    g[:, 0] = np.real(gc)
    g[:, 1] = np.imag(gc) if np.iscomplexobj(gc) else 0.0
    gpos = np.zeros((n, D))
    gw = np.zeros(n)
    rc = lib.npcf_oracle_n3_closed(D, lmax, nbins, int(bin_lt), _dp(edges), _dp(box), int(periodic), _dp(pos),
                                   _dp(w), n, pb, pe, _dp(g), _dp(out), _dp(gpos), _dp(gw))
    if rc < 0:
        raise ValueError(f"oracle failed ({rc})")
    return k, out[:, 0] + 1j * out[:, 1], gpos, gw


def _prep_grid(X, edges, box):
    X = np.ascontiguousarray(X, dtype=np.float64)
    D = X.ndim
    box = np.ascontiguousarray(np.broadcast_to(np.asarray(box, dtype=np.float64), (D,)))
    dims = np.ascontiguousarray(X.shape, dtype=np.int32)
    return X, np.ascontiguousarray(edges, dtype=np.float64), box, dims


def grid_alm(lmax, edges, box, X):
    """a^b_l(s) of eq. alm-bin-def at every node of a periodic grid field X (a D-dimensional
    array over a box of sides `box`), as the direct sum over node offsets (Sec. "Application to
    Gridded Data", reading R16).  Returns complex (ncell, nbins, nstates), nodes in row-major
    order, states in the order of states()."""
    lib = _load()
    X, edges, box, dims = _prep_grid(X, edges, box)
    D, nbins = X.ndim, len(edges) - 1
    ns = lib.npcf_oracle_nstates(D, lmax)
    out = np.zeros((X.size, nbins, ns, 2))
    rc = lib.npcf_oracle_grid_alm(D, lmax, nbins, _dp(edges), _dp(box), _ip(dims), _dp(X), _dp(out))
    if rc < 0:
        raise ValueError(f"oracle failed ({rc})")
    return out[..., 0] + 1j * out[..., 1]


def estimate_grid(N, lmax, edges, box, X, *, bin_lt=False):
    """The isotropic NPCF coefficients of a periodic grid field X (eq. NPCF-mult-estimator with the
    spatial integral as a sum over nodes, Sec. "Application to Gridded Data"): keys as in keys(),
    coefficients complex."""
    lib = _load()
    X, edges, box, dims = _prep_grid(X, edges, box)
    D, nbins = X.ndim, len(edges) - 1
    k = keys(D, N, lmax, nbins, bin_lt)
    out = np.zeros((k.shape[0], 2))
    rc = lib.npcf_oracle_grid_estimate(D, N, lmax, nbins, int(bin_lt), _dp(edges), _dp(box), _ip(dims), _dp(X),
                                       _dp(out))
    if rc < 0:
        raise ValueError(f"oracle failed ({rc})")
    return k, out[:, 0] + 1j * out[:, 1]


def estimate_sphere(N, lmax, cos_edges, pos, w, *, primaries=None, brute=False, bin_lt=False):
    """The isotropic NPCF of points on the unit 2-sphere (Sec. "Cosmic Microwave Background"):
    the D = 2 basis about every primary, radial bins [c_b, c_{b+1}) in cos(theta) (reading R17),
    1/(4 pi) in place of 1/V.  pos: (n, 3) directions (normalised by the oracle).  Keys as in
    keys(2, N, ...); N = 3 or 4."""
    lib = _load()
    pos = np.ascontiguousarray(pos, dtype=np.float64).reshape(-1, 3)
    w = np.ascontiguousarray(w, dtype=np.float64)
    cos_edges = np.ascontiguousarray(cos_edges, dtype=np.float64)
    n = pos.shape[0]
    pb, pe = (0, n) if primaries is None else primaries
    nbins = len(cos_edges) - 1
    k = keys(2, N, lmax, nbins, bin_lt)
    out = np.zeros((k.shape[0], 2))
    rc = lib.npcf_oracle_sphere_estimate(N, lmax, nbins, int(bin_lt), _dp(cos_edges), _dp(pos), _dp(w), n, pb, pe,
                                         int(brute), _dp(out))
    if rc < 0:
        raise ValueError(f"oracle failed ({rc})")
    return k, out[:, 0] + 1j * out[:, 1]


def aniso_keys(N: int, lmax: int, nbins: int, bin_lt: bool = False) -> np.ndarray:
    """Labels of the anisotropic basis about the x_3 line of sight (reading R18), one row per
    coefficient: (b1, b2, b3, l1, l2, L, 0, 0) for N = 3 (b3 = -1) and
    (b1, b2, b3, l1, l2, l12, l3, L) for N = 4."""
    lib = _load()
    nk = lib.npcf_oracle_aniso_nkeys(N, lmax, nbins, int(bin_lt))
    if nk < 0:
        raise ValueError("unsupported anisotropic configuration")
    out = np.zeros((nk, 8), dtype=np.int32)
    lib.npcf_oracle_aniso_keys(N, lmax, nbins, int(bin_lt), _ip(out))
    return out


def estimate_aniso(N, lmax, edges, box, pos, w, *, periodic=True, primaries=None, brute=False, bin_lt=False):
    """The D = 3 NPCF coefficients zeta^{0L}_Lambda of the basis invariant under rotations about the
    x_3 axis (Sec. "Large-Scale Structure": the redshift-space 3PCF and its extension to N = 4),
    keys as in aniso_keys()."""
    lib = _load()
    pos, w, edges, box = _prep(pos, w, edges, box)
    box = np.ascontiguousarray(np.broadcast_to(box, (3,)))
    n = pos.shape[0]
    pb, pe = (0, n) if primaries is None else primaries
    nbins = len(edges) - 1
    k = aniso_keys(N, lmax, nbins, bin_lt)
    out = np.zeros((k.shape[0], 2))
    rc = lib.npcf_oracle_aniso_estimate(N, lmax, nbins, int(bin_lt), _dp(edges), _dp(box), int(periodic), _dp(pos),
                                        _dp(w), n, pb, pe, int(brute), _dp(out))
    if rc < 0:
        raise ValueError(f"oracle failed ({rc})")
    return k, out[:, 0] + 1j * out[:, 1]
