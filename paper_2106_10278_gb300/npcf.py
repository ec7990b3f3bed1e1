"""Thin ctypes binding of libnpcf (include/npcf.h).

Every step of the estimator runs in the CUDA library; this module only checks
arguments, passes pointers and sizes through the C ABI and wraps results in
torch tensors (PyTorch is used for device memory and streams only).  It fails
loudly when the library has not been built: there is no fallback.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.environ.get("NPCF_LIBRARY") or os.path.join(_HERE, "_build", "libnpcf.so")

NPCF_OK = 0
NPCF_FP64, NPCF_FP32, NPCF_MIXED_BF16X3, NPCF_MIXED_TF32X3 = 0, 1, 2, 3
PRECISIONS = {"fp64": NPCF_FP64, "fp32": NPCF_FP32, "mixed_bf16x3": NPCF_MIXED_BF16X3,
              "mixed_tf32x3": NPCF_MIXED_TF32X3}
NPCF_BINS_LE, NPCF_BINS_LT = 0, 1
PARITIES = {"all": 0, "even": 1, "odd": 2}
BASES = {"isotropic": 0, "los": 1}
GEOMETRIES = {"box": 0, "sphere": 1}
STATUS = {0: "NPCF_OK", -1: "NPCF_ERR_ARG", -2: "NPCF_ERR_UNSUPPORTED", -3: "NPCF_ERR_CUDA",
          -4: "NPCF_ERR_WORKSPACE", -5: "NPCF_ERR_DEVICE_TIMEOUT", -6: "NPCF_ERR_NONFINITE"}

# every entry point declared in include/npcf.h
EXPORTS = ("npcf_default_opts", "npcf_plan_create", "npcf_num_coeffs", "npcf_coeff_index", "npcf_compute",
           "npcf_compute_host", "npcf_device_status", "npcf_last_stats", "npcf_last_profile", "npcf_last_error",
           "npcf_plan_destroy", "npcf_compute_noalloc", "npcf_last_counters", "npcf_backward",
           "npcf_compute_batched", "npcf_selftest_tc", "npcf_autotune", "npcf_tuned_config", "npcf_compute_grid")


class NpcfError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS.get(status, status)}: {message}")
        self.status = status


class Opts(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("periodic", ctypes.c_int), ("bin_order", ctypes.c_int),
                ("sync_check", ctypes.c_int), ("timing", ctypes.c_int), ("remove_self", ctypes.c_int),
                ("parity", ctypes.c_int), ("basis", ctypes.c_int), ("geometry", ctypes.c_int)]


_lib = None
_lock = threading.Lock()


def load_library(path: str = LIB_PATH):
    """Load libnpcf.so (raises if it is missing: build it with paper_2106_10278_gb300.build)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(path):
            raise RuntimeError(f"libnpcf is not built ({path} missing); run python -m paper_2106_10278_gb300.build")
        lib = ctypes.CDLL(path)
        P = ctypes.c_void_p
        i32, i64 = ctypes.c_int, ctypes.c_int64
        lib.npcf_default_opts.argtypes = [ctypes.POINTER(Opts)]
        lib.npcf_default_opts.restype = None
        lib.npcf_plan_create.argtypes = [ctypes.POINTER(P), i32, i32, i32, ctypes.POINTER(ctypes.c_double), i32,
                                         ctypes.POINTER(ctypes.c_double), ctypes.POINTER(Opts)]
        lib.npcf_plan_create.restype = i32
        lib.npcf_num_coeffs.argtypes = [P, ctypes.POINTER(i64)]
        lib.npcf_num_coeffs.restype = i32
        lib.npcf_coeff_index.argtypes = [P, i64, ctypes.POINTER(i32), ctypes.POINTER(i32)]
        lib.npcf_coeff_index.restype = i32
        lib.npcf_compute.argtypes = [P, P, P, i64, P, i64, i64, P]
        lib.npcf_compute.restype = i32
        lib.npcf_compute_noalloc.argtypes = [P, P, P, i64, P, i64, i64, P]
        lib.npcf_compute_noalloc.restype = i32
        lib.npcf_compute_host.argtypes = [P, P, P, i64, P, i64, i64, P]
        lib.npcf_compute_host.restype = i32
        lib.npcf_device_status.argtypes = [P]
        lib.npcf_device_status.restype = i32
        lib.npcf_last_stats.argtypes = [P, ctypes.POINTER(i64), ctypes.POINTER(i64), ctypes.POINTER(i64)]
        lib.npcf_last_stats.restype = i32
        lib.npcf_last_profile.argtypes = [P, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(i32)]
        lib.npcf_last_profile.restype = i32
        lib.npcf_last_counters.argtypes = [P, ctypes.POINTER(i64), i32]
        lib.npcf_last_counters.restype = i32
        lib.npcf_compute_batched.argtypes = [P, P, P, ctypes.POINTER(i64), ctypes.POINTER(ctypes.c_double), i32, P,
                                             P]
        lib.npcf_compute_batched.restype = i32
        lib.npcf_backward.argtypes = [P, P, P, i64, P, i64, i64, P, P, P]
        lib.npcf_backward.restype = i32
        lib.npcf_autotune.argtypes = [P, P, P, i64, P]
        lib.npcf_autotune.restype = i32
        lib.npcf_tuned_config.argtypes = [P, ctypes.POINTER(i32), i32]
        lib.npcf_tuned_config.restype = i32
        lib.npcf_selftest_tc.argtypes = [i32, i32, i32, P, P, P, P]
        lib.npcf_selftest_tc.restype = i32
        lib.npcf_compute_grid.argtypes = [P, P, ctypes.POINTER(i32), P, P]
        lib.npcf_compute_grid.restype = i32
        lib.npcf_last_error.argtypes = []
        lib.npcf_last_error.restype = ctypes.c_char_p
        lib.npcf_plan_destroy.argtypes = [P]
        lib.npcf_plan_destroy.restype = None
        _lib = lib
        return lib


def _check(status: int):
    if status != NPCF_OK:
        msg = load_library().npcf_last_error().decode(errors="replace")
        raise NpcfError(status, msg)


def selftest_tc(a, b, tf32=False, stream=None):
    """The split-precision tensor-core contraction on caller data: a (128, k) and b (n, k) float32
    CUDA tensors -> a b^T (128, n) float32, through npcf_selftest_tc (a diagnostic of the MMA path
    the mixed couplings use)."""
    import torch
    lib = load_library()
    if not (a.is_cuda and b.is_cuda) or a.dtype != torch.float32 or b.dtype != torch.float32:
        raise TypeError("a and b must be float32 CUDA tensors")
    a = a.contiguous()
    b = b.contiguous()
    if a.dim() != 2 or b.dim() != 2 or a.shape[0] != 128 or a.shape[1] != b.shape[1]:
        raise ValueError("a must be (128, k) and b (n, k)")
    d = torch.empty(128, b.shape[0], dtype=torch.float32, device=a.device)
    s = stream if stream is not None else torch.cuda.current_stream(a.device)
    with torch.cuda.device(a.device):
        _check(lib.npcf_selftest_tc(int(bool(tf32)), b.shape[0], a.shape[1], ctypes.c_void_p(a.data_ptr()),
                                    ctypes.c_void_p(b.data_ptr()), ctypes.c_void_p(d.data_ptr()),
                                    ctypes.c_void_p(s.cuda_stream)))
    return d


class Plan:
    """A plan for one (D, N, lmax, bins, box) estimator configuration.

    remove_self: subtract the tuples whose secondaries coincide (N=3 keys with b1 = b2).
    parity: "all", "even" or "odd" components (odd ones exist for the D=3 4PCF only).
    basis: "isotropic" or "los" (D=3, N=3 or 4: the basis about the x_3 line of sight, labels
    (l1, l2, L) or (l1, l2, l12, l3, L)).
    geometry: "box" (Euclidean) or "sphere" (points on the unit 2-sphere: D=2, N=3 or 4, positions
    (n, 3) directions, edges in cos theta, box ignored -- pass None).
    precision: "fp32" (positions/weights float32; FP32 pair and coupling
    arithmetic, FP64 sums over primaries), "fp64" (double throughout), or
    "mixed_bf16x3" / "mixed_tf32x3" (float32 inputs and pair stage; the coupling
    on the tensor cores with every operand split into BF16 or TF32 hi + lo
    pairs, FP32 accumulation, FP64 sums across spans of primaries).
    """

    def __init__(self, D, N, lmax, edges, box, *, precision="fp32", periodic=True, bin_lt=False, sync_check=True,
                 timing=False, remove_self=False, parity="all", basis="isotropic", geometry="box"):
        if precision not in PRECISIONS:
            raise ValueError(f"precision must be one of {sorted(PRECISIONS)}, not {precision!r}")
        lib = load_library()
        self.D, self.N, self.lmax = int(D), int(N), int(lmax)
        self.edges = np.ascontiguousarray(edges, dtype=np.float64)
        if geometry not in GEOMETRIES:
            raise ValueError(f"geometry must be one of {sorted(GEOMETRIES)}, not {geometry!r}")
        self.geometry = geometry
        self.Dp = 3 if geometry == "sphere" else self.D  # components of a position
        if box is None and geometry == "sphere":
            box = 1.0
        self.box = np.ascontiguousarray(np.broadcast_to(np.asarray(box, dtype=np.float64), (self.D,)))
        self.nbins = len(self.edges) - 1
        self.precision = precision
        o = Opts()
        lib.npcf_default_opts(ctypes.byref(o))
        o.precision = PRECISIONS[precision]
        o.periodic = int(bool(periodic))
        o.bin_order = NPCF_BINS_LT if bin_lt else NPCF_BINS_LE
        o.sync_check = int(bool(sync_check))
        o.timing = int(bool(timing))
        o.remove_self = int(bool(remove_self))
        if parity not in PARITIES:
            raise ValueError(f"parity must be one of {sorted(PARITIES)}, not {parity!r}")
        o.parity = PARITIES[parity]
        if basis not in BASES:
            raise ValueError(f"basis must be one of {sorted(BASES)}, not {basis!r}")
        o.basis = BASES[basis]
        self.basis = basis
        o.geometry = GEOMETRIES[geometry]
        h = ctypes.c_void_p()
        _check(lib.npcf_plan_create(ctypes.byref(h), self.D, self.N, self.lmax,
                                    self.edges.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), self.nbins,
                                    self.box.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), ctypes.byref(o)))
        self._h = h
        n = ctypes.c_int64()
        _check(lib.npcf_num_coeffs(self._h, ctypes.byref(n)))
        self.ncoeff = int(n.value)
        self._keys = None

    # ------------------------------------------------------------------
    def keys(self) -> np.ndarray:
        """Output labels, one row per coefficient: (b1, b2, b3, l1, l2, l3) for N <= 4 (b3 = -1 and
        l2 = l3 = 0 when unused); (b1, b2, b3, b4, l1, l2, l12, l3, l4) for N = 5; with the
        line-of-sight basis (b1, b2, b3, l1, l2, L, 0, 0) for N = 3 and (b1, b2, b3, l1, l2, l12,
        l3, L) for N = 4."""
        if self._keys is None:
            lib = load_library()
            los = getattr(self, "basis", "isotropic") == "los"
            if los:
                nb, ne, nl = 3, 5, (3 if self.N == 3 else 5)
            else:
                nb, ne = (4, 5) if self.N == 5 else (3, 3)
                nl = {3: 1, 4: 3, 5: 5}[self.N]
            k = np.zeros((self.ncoeff, nb + ne), dtype=np.int32)
            k[:, nb - 1] = -1
            bins = (ctypes.c_int * 4)()
            ells = (ctypes.c_int * 5)()
            for i in range(self.ncoeff):
                _check(lib.npcf_coeff_index(self._h, i, bins, ells))
                for a in range(self.N - 1):
                    k[i, a] = bins[a]
                for a in range(nl):
                    k[i, nb + a] = ells[a]
            self._keys = k
        return self._keys

    def _dtype(self):
        import torch
        return torch.float64 if self.precision == "fp64" else torch.float32

    def compute(self, pos, w, primaries=None, out=None, stream=None):
        """Coefficients on the device for device tensors pos (n, D) (n, 3 on the sphere) and w (n).

        Returns a complex128 tensor of ncoeff entries (a view of `out`, a float64
        tensor of 2*ncoeff, allocated if not given)."""
        import torch
        lib = load_library()
        dt = self._dtype()
        if not (pos.is_cuda and w.is_cuda):
            raise ValueError("pos and w must be CUDA tensors (use compute_host for host arrays)")
        if pos.dtype != dt or w.dtype != dt:
            raise TypeError(f"pos and w must be {dt} for a {self.precision} plan")
        if pos.dim() != 2 or pos.shape[1] != self.Dp or w.shape != (pos.shape[0],):
            raise ValueError("pos must be (n, D) and w (n,)")
        pos = pos.contiguous()
        w = w.contiguous()
        n = pos.shape[0]
        if out is None:
            out = torch.empty(2 * self.ncoeff, dtype=torch.float64, device=pos.device)
        pb, pe = (0, n) if primaries is None else (int(primaries[0]), int(primaries[1]))
        s = stream if stream is not None else torch.cuda.current_stream(pos.device)
        with torch.cuda.device(pos.device):
            _check(lib.npcf_compute(self._h, ctypes.c_void_p(pos.data_ptr()), ctypes.c_void_p(w.data_ptr()), n,
                                    ctypes.c_void_p(out.data_ptr()), pb, pe, ctypes.c_void_p(s.cuda_stream)))
        return torch.view_as_complex(out.view(-1, 2))

    def compute_batched(self, pos, w, offsets, boxes, out=None, stream=None):
        """Coefficients of several catalogues in one pass.

        pos (n, D) and w (n) are the catalogues concatenated on the device;
        offsets (ncat + 1) delimits them and boxes (ncat, D) gives each one's box.
        Returns a complex128 tensor (ncat, ncoeff)."""
        import torch
        lib = load_library()
        dt = self._dtype()
        if not (pos.is_cuda and w.is_cuda):
            raise ValueError("pos and w must be CUDA tensors")
        if pos.dtype != dt or w.dtype != dt:
            raise TypeError(f"pos and w must be {dt} for a {self.precision} plan")
        off = np.ascontiguousarray(offsets, dtype=np.int64)
        ncat = len(off) - 1
        bx = np.ascontiguousarray(np.broadcast_to(np.asarray(boxes, dtype=np.float64), (ncat, self.D)))
        if pos.dim() != 2 or pos.shape[1] != self.Dp or w.shape != (pos.shape[0],) or off[-1] != pos.shape[0]:
            raise ValueError("pos must be (n, D), w (n,) and offsets[-1] == n")
        pos = pos.contiguous()
        w = w.contiguous()
        if out is None:
            out = torch.empty(ncat * 2 * self.ncoeff, dtype=torch.float64, device=pos.device)
        s = stream if stream is not None else torch.cuda.current_stream(pos.device)
        with torch.cuda.device(pos.device):
            _check(lib.npcf_compute_batched(self._h, ctypes.c_void_p(pos.data_ptr()), ctypes.c_void_p(w.data_ptr()),
                                            off.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                                            bx.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), ncat,
                                            ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(s.cuda_stream)))
        return torch.view_as_complex(out.view(ncat, -1, 2))

    def compute_grid(self, field, out=None, stream=None):
        """Coefficients of a periodic grid field (a D-dimensional CUDA tensor of the plan's precision
        over the plan's box, row-major) by the FFT form of the estimator (npcf_compute_grid).
        Returns a complex128 tensor of ncoeff entries."""
        import torch
        lib = load_library()
        dt = self._dtype()
        if not field.is_cuda or field.dtype != dt:
            raise TypeError(f"field must be a {dt} CUDA tensor")
        if field.dim() != self.D:
            raise ValueError(f"field must have {self.D} axes")
        field = field.contiguous()
        dims = np.ascontiguousarray(field.shape, dtype=np.int32)
        if out is None:
            out = torch.empty(2 * self.ncoeff, dtype=torch.float64, device=field.device)
        s = stream if stream is not None else torch.cuda.current_stream(field.device)
        with torch.cuda.device(field.device):
            _check(lib.npcf_compute_grid(self._h, ctypes.c_void_p(field.data_ptr()),
                                         dims.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                                         ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(s.cuda_stream)))
        return torch.view_as_complex(out.view(-1, 2))

    def backward(self, pos, w, grad_coeffs, primaries=None, stream=None, want_pos=True, want_w=True):
        """dL/dpos (n, D) and dL/dw (n) for device tensors, given dL/dcoeff.

        grad_coeffs: float64 device tensor of 2*ncoeff entries (dL/dRe, dL/dIm
        interleaved) or a complex128 tensor of ncoeff entries.  N=3 plans only."""
        import torch
        lib = load_library()
        dt = self._dtype()
        if not (pos.is_cuda and w.is_cuda and grad_coeffs.is_cuda):
            raise ValueError("pos, w and grad_coeffs must be CUDA tensors")
        if pos.dtype != dt or w.dtype != dt:
            raise TypeError(f"pos and w must be {dt} for a {self.precision} plan")
        if pos.dim() != 2 or pos.shape[1] != self.Dp or w.shape != (pos.shape[0],):
            raise ValueError("pos must be (n, D) and w (n,)")
        g = torch.view_as_real(grad_coeffs).reshape(-1) if grad_coeffs.is_complex() else grad_coeffs.reshape(-1)
        g = g.to(torch.float64).contiguous()
        if g.numel() != 2 * self.ncoeff:
            raise ValueError(f"grad_coeffs must hold {2 * self.ncoeff} doubles")
        pos = pos.contiguous()
        w = w.contiguous()
        n = pos.shape[0]
        gp = torch.empty_like(pos) if want_pos else None
        gw = torch.empty_like(w) if want_w else None
        pb, pe = (0, n) if primaries is None else (int(primaries[0]), int(primaries[1]))
        s = stream if stream is not None else torch.cuda.current_stream(pos.device)
        ptr = lambda t: ctypes.c_void_p(None if t is None else t.data_ptr())
        with torch.cuda.device(pos.device):
            _check(lib.npcf_backward(self._h, ptr(pos), ptr(w), n, ptr(g), pb, pe, ptr(gp), ptr(gw),
                                     ctypes.c_void_p(s.cuda_stream)))
        return gp, gw

    def compute_host(self, pos, w, primaries=None, stream=None) -> np.ndarray:
        """Coefficients for host arrays (copied in and out by the library)."""
        lib = load_library()
        dt = np.float64 if self.precision == "fp64" else np.float32
        pos = np.ascontiguousarray(pos, dtype=dt)
        w = np.ascontiguousarray(w, dtype=dt)
        n = pos.shape[0]
        out = np.zeros(2 * self.ncoeff)
        pb, pe = (0, n) if primaries is None else (int(primaries[0]), int(primaries[1]))
        sptr = ctypes.c_void_p(None if stream is None else stream.cuda_stream)
        _check(lib.npcf_compute_host(self._h, pos.ctypes.data_as(ctypes.c_void_p), w.ctypes.data_as(ctypes.c_void_p),
                                     n, out.ctypes.data_as(ctypes.c_void_p), pb, pe, sptr))
        return out[0::2] + 1j * out[1::2]

    def autotune(self, pos, w, stream=None) -> dict:
        """Time candidate launch shapes on a sample of these device tensors' primaries and keep the
        fastest (npcf_autotune); returns the shapes chosen (tuned_config)."""
        import torch
        lib = load_library()
        dt = self._dtype()
        if not (pos.is_cuda and w.is_cuda) or pos.dtype != dt or w.dtype != dt:
            raise TypeError(f"pos and w must be {dt} CUDA tensors")
        pos = pos.contiguous()
        w = w.contiguous()
        s = stream if stream is not None else torch.cuda.current_stream(pos.device)
        with torch.cuda.device(pos.device):
            _check(lib.npcf_autotune(self._h, ctypes.c_void_p(pos.data_ptr()), ctypes.c_void_p(w.data_ptr()),
                                     pos.shape[0], ctypes.c_void_p(s.cuda_stream)))
        return self.tuned_config()

    def tuned_config(self) -> dict:
        """The launch shapes in use (npcf_tuned_config)."""
        lib = load_library()
        v = (ctypes.c_int * 6)()
        _check(lib.npcf_tuned_config(self._h, v, 6))
        names = ("pair_warps", "pair_batch", "couple_ctas_per_sm", "tc_span", "d5_chunk", "tuned")
        return dict(zip(names, (int(x) for x in v)))

    def stats(self) -> dict:
        """Pairs accumulated, primaries and candidate secondaries of the last call."""
        lib = load_library()
        a, b, c = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
        _check(lib.npcf_last_stats(self._h, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)))
        return {"pairs": a.value, "primaries": b.value, "candidates": c.value}

    def profile(self) -> dict:
        """Stage times (ms, CUDA events; -1 unless timing=True) and kernel launches of the last call."""
        lib = load_library()
        ms = (ctypes.c_double * 4)()
        nl = ctypes.c_int()
        _check(lib.npcf_last_profile(self._h, ms, ctypes.byref(nl)))
        return {"cells_ms": ms[0], "pairs_ms": ms[1], "couple_ms": ms[2], "reduce_ms": ms[3], "launches": nl.value}

    def counters(self) -> dict:
        """Pair-kernel work counters of the last call (profiling)."""
        lib = load_library()
        c = (ctypes.c_int64 * 8)()
        _check(lib.npcf_last_counters(self._h, c, 8))
        names = ("pairs", "candidates", "rounds", "busy_lanes", "chunks", "batches", "flagged", "exact")
        return dict(zip(names, (int(x) for x in c)))

    def function(self, primaries=None):
        """A torch.autograd.Function-backed callable (pos, w) -> coefficients as an
        (ncoeff, 2) float64 tensor (re, im), differentiable in pos and w (N=3)."""
        plan = self

        import torch

        class _Estimate(torch.autograd.Function):
            @staticmethod
            def forward(ctx, pos, w):
                ctx.save_for_backward(pos, w)
                return torch.view_as_real(plan.compute(pos.detach(), w.detach(), primaries=primaries)).clone()

            @staticmethod
            def backward(ctx, grad_out):
                pos, w = ctx.saved_tensors
                gp, gw = plan.backward(pos, w, grad_out.reshape(-1), primaries=primaries,
                                       want_pos=ctx.needs_input_grad[0], want_w=ctx.needs_input_grad[1])
                return gp, gw

        return _Estimate.apply

    def close(self):
        if getattr(self, "_h", None):
            load_library().npcf_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
