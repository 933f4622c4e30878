"""Thin Python binding of libgmp (include/gmp.h): argument marshalling only.

Every step of the featurization runs in the CUDA library; this module only
checks shapes and dtypes, passes pointers and the current CUDA stream, and
turns status codes into exceptions.  There is no CPU fallback: if the
library is missing or fails to load, an ImportError / RuntimeError is
raised.

Naming follows GMP-Featurizer (arXiv 2303.12980, Examples): "orders" are the
MCSH angular probe orders (-1 = local density), "sigmas" the Gaussian radial
probe widths; features are ordered order-major; the position derivatives are
"feature_primes" (here: a CSR Jacobian) or, for training, a vector-Jacobian
product.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libgmp.so")

GMP_OK = 0
GMP_ERR_CAPACITY = 4
_STATUS = {1: "GMP_ERR_INVALID_ARG", 2: "GMP_ERR_CUDA", 3: "GMP_ERR_OOM", 4: "GMP_ERR_CAPACITY",
           5: "GMP_ERR_TIMEOUT", 6: "GMP_ERR_DEVICE"}
EXPORTS = ("gmp_create", "gmp_num_features", "gmp_featurize", "gmp_featurize_vjp", "gmp_featurize_vjp_virial",
           "gmp_featurize_grad", "gmp_featurize_grad_centers", "gmp_featurize_points", "gmp_neighbors", "gmp_cutoff", "gmp_set_graph", "gmp_tune", "gmp_tuning_get", "gmp_tuning_set",
           "gmp_sync", "gmp_profile", "gmp_profile_read",
           "gmp_probe_peaks", "gmp_probe_contraction", "gmp_probe_backward_contraction", "gmp_last_error",
           "gmp_kernel_launches", "gmp_destroy")
TUNING_CACHE = os.environ.get("GMP_TUNING_CACHE",
                              os.path.join(os.path.expanduser("~"), ".cache", "gmp_gb300", "tuning.json"))

_lib = None
_lock = threading.Lock()


class GMPError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{_STATUS.get(status, status)}: {msg}")
        self.status = status


class _Params(C.Structure):
    _fields_ = [
        ("n_elements", C.c_int32),
        ("n_gauss", C.c_void_p),
        ("gauss_coef", C.c_void_p),
        ("gauss_exp", C.c_void_p),
        ("n_orders", C.c_int32),
        ("orders", C.c_void_p),
        ("n_sigmas", C.c_int32),
        ("sigmas", C.c_void_p),
        ("cutoff", C.c_double),
        ("flags", C.c_uint32),
        ("overlap_threshold", C.c_double),
    ]


def load_library(path: str = LIB_PATH):
    """Load libgmp.so (built by paper_2303_12980_gb300.build.build())."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(path):
            raise ImportError(f"libgmp.so not found at {path}; build it with "
                              "paper_2303_12980_gb300.build.build() (needs nvcc)")
        L = C.CDLL(path)
        vp, i32, i64 = C.c_void_p, C.c_int32, C.c_int64
        L.gmp_create.argtypes = [C.POINTER(_Params), C.c_int, C.POINTER(vp)]
        L.gmp_num_features.argtypes = [vp, C.POINTER(i32)]
        common = [vp, i32, vp, vp, vp, vp, vp]
        L.gmp_featurize.argtypes = common + [vp, vp]
        L.gmp_featurize_vjp.argtypes = common + [vp, vp, vp, vp]
        L.gmp_featurize_vjp_virial.argtypes = common + [vp, vp, vp, vp, vp]
        L.gmp_featurize_grad.argtypes = common + [vp, vp, vp, vp, i64, C.POINTER(i64), vp]
        L.gmp_featurize_grad_centers.argtypes = common + [i64, i64, vp, vp, vp, vp, i64, C.POINTER(i64), vp]
        L.gmp_neighbors.argtypes = common + [vp, vp, vp, i64, C.POINTER(i64), vp]
        L.gmp_featurize_points.argtypes = common + [vp, vp, vp, vp]
        L.gmp_set_graph.argtypes = [vp, C.c_int]
        L.gmp_cutoff.argtypes = [vp, C.POINTER(C.c_double)]
        L.gmp_tune.argtypes = common + [i32, C.POINTER(i64), vp]
        L.gmp_tuning_get.argtypes = [vp, C.POINTER(i32), i32]
        L.gmp_tuning_set.argtypes = [vp, C.POINTER(i32), i32]
        L.gmp_sync.argtypes = [vp, vp, C.c_double]
        L.gmp_profile.argtypes = [vp, C.c_int]
        L.gmp_profile_read.argtypes = [vp, C.POINTER(C.c_double), C.POINTER(i64), C.c_int]
        L.gmp_last_error.argtypes = [vp]
        L.gmp_last_error.restype = C.c_char_p
        L.gmp_kernel_launches.argtypes = [vp]
        L.gmp_kernel_launches.restype = i64
        L.gmp_probe_peaks.argtypes = [C.c_int, C.POINTER(C.c_double), C.POINTER(C.c_double), C.POINTER(C.c_double)]
        L.gmp_probe_contraction.argtypes = [C.c_int, C.POINTER(C.c_double), i32]
        L.gmp_probe_backward_contraction.argtypes = [C.c_int, C.POINTER(C.c_double), i32]
        L.gmp_destroy.argtypes = [vp]
        L.gmp_destroy.restype = None
        for name in EXPORTS[:-3]:
            getattr(L, name).restype = C.c_int
        _lib = L
        return _lib


def _torch():
    import torch
    return torch


def _ptr(x):
    if x is None:
        return None
    if isinstance(x, np.ndarray):
        return x.ctypes.data
    return x.data_ptr()


def _stream_ptr(stream, on_device: bool):
    if not on_device:
        return None
    torch = _torch()
    s = stream if stream is not None else torch.cuda.current_stream()
    return s.cuda_stream


class GMPFeaturizer:
    """Handle on a GMP probe set + density tables on one CUDA device.

    orders: MCSH orders (each -1..6), sigmas: radial widths (A), cutoff (A),
    n_gauss/gauss_coef/gauss_exp: per-element Gaussian densities
    rho_e(r) = sum_k c_k exp(-alpha_k r^2).
    """

    def __init__(self, orders, sigmas, cutoff, n_gauss, gauss_coef, gauss_exp, device: int = 0,
                 flags: int = 0, overlap_threshold: float = 1e-16):
        self._L = load_library()
        self.orders = [int(o) for o in orders]
        self.sigmas = [float(s) for s in sigmas]
        self.cutoff = float(cutoff) if cutoff else 0.0
        self.device = int(device)
        self._keep = dict(
            n_gauss=np.ascontiguousarray(n_gauss, np.int32),
            coef=np.ascontiguousarray(gauss_coef, np.float64),
            expo=np.ascontiguousarray(gauss_exp, np.float64),
            orders=np.ascontiguousarray(self.orders, np.int32),
            sigmas=np.ascontiguousarray(self.sigmas if self.sigmas else [1.0], np.float64),
        )
        k = self._keep
        p = _Params(n_elements=k["n_gauss"].size, n_gauss=k["n_gauss"].ctypes.data,
                    gauss_coef=k["coef"].ctypes.data, gauss_exp=k["expo"].ctypes.data,
                    n_orders=len(self.orders), orders=k["orders"].ctypes.data,
                    n_sigmas=len(self.sigmas), sigmas=k["sigmas"].ctypes.data,
                    cutoff=self.cutoff, flags=int(flags), overlap_threshold=float(overlap_threshold))
        h = C.c_void_p()
        st = self._L.gmp_create(C.byref(p), self.device, C.byref(h))
        if st != GMP_OK:
            raise GMPError(st, "gmp_create rejected the parameters (see stderr)")
        self._h = h
        rc = C.c_double()
        self._check(self._L.gmp_cutoff(self._h, C.byref(rc)))
        self.cutoff = float(rc.value)  # derived from overlap_threshold when cutoff was not given
        F = C.c_int32()
        self._check(self._L.gmp_num_features(self._h, C.byref(F)))
        self.num_features = int(F.value)
        # output rows of the last featurize_grad / neighbors call: the next
        # call allocates that many first and re-runs only when it needs more
        self._rows = {"grad": 0, "neighbors": 0}

    @classmethod
    def from_workload(cls, w, device: int = 0):
        return cls(w.orders, w.sigmas, w.cutoff, w.n_gauss, w.gauss_coef, w.gauss_exp, device)

    def close(self):
        if getattr(self, "_h", None):
            self._L.gmp_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, st):
        if st != GMP_OK:
            msg = self._L.gmp_last_error(self._h)
            raise GMPError(st, msg.decode() if msg else "")

    @property
    def kernel_launches(self) -> int:
        return int(self._L.gmp_kernel_launches(self._h))

    # ---------------------------------------------------------------- inputs
    @staticmethod
    def _struct(atom_off, cell, pbc):
        off = np.ascontiguousarray(atom_off, np.int64)
        S = off.size - 1
        cell = np.ascontiguousarray(np.asarray(cell, np.float64).reshape(S, 3, 3))
        pbc = np.ascontiguousarray(np.asarray(pbc, np.uint8).reshape(S, 3))
        return off, cell, pbc

    def _inputs(self, pos, species):
        torch = _torch()
        on_dev = isinstance(pos, torch.Tensor) and pos.is_cuda
        if isinstance(pos, torch.Tensor):
            if pos.dtype != torch.float64 or not pos.is_contiguous() or pos.dim() != 2 or pos.shape[1] != 3:
                raise ValueError("pos must be a contiguous float64 [N,3] tensor")
            if species.dtype != torch.int32 or not species.is_contiguous() or species.is_cuda != on_dev:
                raise ValueError("species must be a contiguous int32 tensor on the same device as pos")
            if not on_dev:
                pos, species = pos.numpy(), species.numpy()
        else:
            pos = np.ascontiguousarray(pos, np.float64)
            species = np.ascontiguousarray(species, np.int32)
        return pos, species, on_dev

    def _alloc(self, shape, dtype, on_dev, like=None):
        torch = _torch()
        if on_dev:
            return torch.empty(shape, dtype=dtype, device=like.device)
        return torch.empty(shape, dtype=dtype).pin_memory() if torch.cuda.is_available() else \
            torch.empty(shape, dtype=dtype)

    # ----------------------------------------------------------------- calls
    def featurize(self, pos, species, atom_off, cell, pbc, out=None, stream=None):
        """features [N, F] float32 (device tensor for device inputs)."""
        torch = _torch()
        off, cell, pbc = self._struct(atom_off, cell, pbc)
        pos, species, on_dev = self._inputs(pos, species)
        N = int(off[-1])
        feat = out if out is not None else self._alloc((N, self.num_features), torch.float32, on_dev, pos)
        self._check(self._L.gmp_featurize(self._h, off.size - 1, off.ctypes.data, _ptr(pos), cell.ctypes.data,
                                          pbc.ctypes.data, _ptr(species), _ptr(feat),
                                          _stream_ptr(stream, on_dev)))
        return feat

    def featurize_vjp(self, pos, species, atom_off, cell, pbc, grad_feat, want_features=True,
                      stream=None, out=None):
        """(features or None, grad_pos [N,3] float32) with
        grad_pos[j] = sum_{i,f} grad_feat[i,f] d features[i,f] / d pos[j]."""
        torch = _torch()
        off, cell, pbc = self._struct(atom_off, cell, pbc)
        pos, species, on_dev = self._inputs(pos, species)
        N = int(off[-1])
        if isinstance(grad_feat, np.ndarray):
            grad_feat = torch.from_numpy(np.ascontiguousarray(grad_feat, np.float32))
        if grad_feat.dtype != torch.float32 or tuple(grad_feat.shape) != (N, self.num_features):
            raise ValueError("grad_feat must be float32 [N, F]")
        grad_feat = grad_feat.contiguous()
        if out is not None:
            feat, gp = out
        else:
            feat = self._alloc((N, self.num_features), torch.float32, on_dev, pos) if want_features else None
            gp = self._alloc((N, 3), torch.float32, on_dev, pos)
        self._check(self._L.gmp_featurize_vjp(self._h, off.size - 1, off.ctypes.data, _ptr(pos), cell.ctypes.data,
                                              pbc.ctypes.data, _ptr(species), _ptr(grad_feat), _ptr(feat),
                                              _ptr(gp), _stream_ptr(stream, on_dev)))
        return feat, gp

    def featurize_vjp_virial(self, pos, species, atom_off, cell, pbc, grad_feat, stream=None):
        """(features, grad_pos [N,3] float32, virial [S,3,3] float64): the
        VJP plus, per structure, dL/d(strain) = sum over pairs of (dL/dd) d^T."""
        torch = _torch()
        off, cell, pbc = self._struct(atom_off, cell, pbc)
        pos, species, on_dev = self._inputs(pos, species)
        N = int(off[-1])
        if isinstance(grad_feat, np.ndarray):
            grad_feat = torch.from_numpy(np.ascontiguousarray(grad_feat, np.float32))
        if grad_feat.dtype != torch.float32 or tuple(grad_feat.shape) != (N, self.num_features):
            raise ValueError("grad_feat must be float32 [N, F]")
        grad_feat = grad_feat.contiguous()
        feat = self._alloc((N, self.num_features), torch.float32, on_dev, pos)
        gp = self._alloc((N, 3), torch.float32, on_dev, pos)
        vir = self._alloc((off.size - 1, 3, 3), torch.float64, on_dev, pos)
        self._check(self._L.gmp_featurize_vjp_virial(self._h, off.size - 1, off.ctypes.data, _ptr(pos),
                                                     cell.ctypes.data, pbc.ctypes.data, _ptr(species),
                                                     _ptr(grad_feat), _ptr(feat), _ptr(gp), _ptr(vir),
                                                     _stream_ptr(stream, on_dev)))
        return feat, gp, vir

    def featurize_grad(self, pos, species, atom_off, cell, pbc, stream=None, centers=None):
        """(features [N,F], jac_off [N+1] int64, jac_j [nnz] int32, jac [nnz,F,3] float32):
        jac[r] = d features[i] / d pos[jac_j[r]] for r in jac_off[i]:jac_off[i+1].
        centers=(begin, end): only those centers (gmp_featurize_grad_centers);
        features, jac_off and rows are then relative to the range."""
        torch = _torch()
        off, cell, pbc = self._struct(atom_off, cell, pbc)
        pos, species, on_dev = self._inputs(pos, species)
        N = int(off[-1])
        b, e = (0, N) if centers is None else (int(centers[0]), int(centers[1]))
        if not 0 <= b <= e <= N:
            raise ValueError("centers must satisfy 0 <= begin <= end <= number of atoms")
        feat = self._alloc((e - b, self.num_features), torch.float32, on_dev, pos)
        joff = self._alloc((e - b + 1,), torch.int64, on_dev, pos)
        nnz = C.c_int64()
        cap = self._rows["grad"]
        while True:
            jj = self._alloc((max(cap, 1),), torch.int32, on_dev, pos)
            jac = self._alloc((max(cap, 1), self.num_features, 3), torch.float32, on_dev, pos)
            head = (self._h, off.size - 1, off.ctypes.data, _ptr(pos), cell.ctypes.data, pbc.ctypes.data,
                    _ptr(species))
            tail = (_ptr(feat), _ptr(joff), _ptr(jj), _ptr(jac), max(cap, 1), C.byref(nnz),
                    _stream_ptr(stream, on_dev))
            if centers is None:
                st = self._L.gmp_featurize_grad(*head, *tail)
            else:
                st = self._L.gmp_featurize_grad_centers(*head, b, e, *tail)
            n = int(nnz.value)
            if st == GMP_ERR_CAPACITY and n > max(cap, 1):
                cap = n  # the call reported the rows it needs
                continue
            self._check(st)
            break
        self._rows["grad"] = n
        return feat, joff, jj[:n], jac[:n]

    def featurize_points(self, pos, species, atom_off, cell, pbc, points, point_off, stream=None):
        """Features [n_points, F] float32 with the probes centred on reference
        points (float64 [n_points, 3], same device as pos); structure s owns
        points point_off[s]:point_off[s+1]."""
        torch = _torch()
        off, cell, pbc = self._struct(atom_off, cell, pbc)
        pos, species, on_dev = self._inputs(pos, species)
        poff = np.ascontiguousarray(point_off, np.int64)
        if poff.size != off.size:
            raise ValueError("point_off needs one entry per structure plus one")
        if isinstance(points, torch.Tensor):
            if points.dtype != torch.float64 or not points.is_contiguous() or points.is_cuda != on_dev:
                raise ValueError("points must be a contiguous float64 tensor on the same device as pos")
            if not on_dev:
                points = points.numpy()
        else:
            points = np.ascontiguousarray(points, np.float64)
        NP = int(poff[-1])
        if tuple(points.shape) != (NP, 3):
            raise ValueError("points must be [point_off[-1], 3]")
        feat = self._alloc((NP, self.num_features), torch.float32, on_dev, pos)
        self._check(self._L.gmp_featurize_points(self._h, off.size - 1, off.ctypes.data, _ptr(pos), cell.ctypes.data,
                                                 pbc.ctypes.data, _ptr(species), poff.ctypes.data, _ptr(points),
                                                 _ptr(feat), _stream_ptr(stream, on_dev)))
        return feat

    def neighbors(self, pos, species, atom_off, cell, pbc, stream=None):
        """Exact neighbor images: (nbr_off [N+1], nbr_j [P], nbr_shift [P,3])."""
        torch = _torch()
        off, cell, pbc = self._struct(atom_off, cell, pbc)
        pos, species, on_dev = self._inputs(pos, species)
        N = int(off[-1])
        noff = self._alloc((N + 1,), torch.int64, on_dev, pos)
        nnz = C.c_int64()
        cap = self._rows["neighbors"]
        while True:
            nj = self._alloc((max(cap, 1),), torch.int32, on_dev, pos)
            ns = self._alloc((max(cap, 1), 3), torch.int32, on_dev, pos)
            st = self._L.gmp_neighbors(self._h, off.size - 1, off.ctypes.data, _ptr(pos), cell.ctypes.data,
                                       pbc.ctypes.data, _ptr(species), _ptr(noff), _ptr(nj), _ptr(ns), max(cap, 1),
                                       C.byref(nnz), _stream_ptr(stream, on_dev))
            n = int(nnz.value)
            if st == GMP_ERR_CAPACITY and n > max(cap, 1):
                cap = n
                continue
            self._check(st)
            break
        self._rows["neighbors"] = n
        return noff, nj[:n], ns[:n]

    def profile(self, enable: bool = True):
        """Per-stage CUDA-event timing on the caller's stream (diagnostics)."""
        self._check(self._L.gmp_profile(self._h, int(enable)))

    def profile_read(self):
        """{stage: (ms, count)} since the last read, stages 'neighbors',
        'features' (forward / Jacobian kernel), 'backward', 'refine'."""
        ms = (C.c_double * 4)()
        cnt = (C.c_int64 * 4)()
        self._check(self._L.gmp_profile_read(self._h, ms, cnt, 4))
        names = ("neighbors", "features", "backward", "refine")
        return {n: (ms[k], cnt[k]) for k, n in enumerate(names)}

    def set_graph(self, enable: bool = True):
        """CUDA-graph replay of repeated calls on the same buffers and a
        non-default stream (gmp_set_graph)."""
        self._check(self._L.gmp_set_graph(self._h, int(enable)))

    # ---------------------------------------------------------------- tuning
    def tuning_key(self, atom_off) -> str:
        """Signature of a problem for the tuning cache: probe set, tables
        and the batch's size class."""
        off = np.asarray(atom_off)
        N, S = int(off[-1]), off.size - 1
        ng = tuple(int(x) for x in self._keep["n_gauss"])
        return (f"o{self.orders}_s{len(self.sigmas)}_g{max(ng)}x{len(ng)}_rc{self.cutoff:g}"
                f"_N{int(np.log2(max(N, 1)))}_S{int(np.log2(max(S, 1)))}")

    def tuning(self):
        n = 6 * 64
        buf = (C.c_int32 * n)()
        st = self._L.gmp_tuning_get(self._h, buf, n)
        self._check(st)
        vals = list(buf)
        npass = max(1, (len(self.sigmas) + 15) // 16) if any(o >= 0 for o in self.orders) else 1
        return vals[:6 * npass]

    def set_tuning(self, values):
        arr = (C.c_int32 * len(values))(*[int(v) for v in values])
        self._check(self._L.gmp_tuning_set(self._h, arr, len(values)))

    def tune(self, pos, species, atom_off, cell, pbc, reps: int = 3, cache: bool = True, stream=None):
        """Pick the fastest launch shapes on this batch (gmp_tune), reusing
        and updating a JSON cache keyed by tuning_key()."""
        import json
        key = self.tuning_key(atom_off)
        if cache and os.path.exists(TUNING_CACHE):
            try:
                with open(TUNING_CACHE) as f:
                    known = json.load(f)
                if key in known:
                    self.set_tuning(known[key])
                    return {"key": key, "values": known[key], "cached": True}
            except (OSError, ValueError, GMPError):
                pass
        off, cell, pbc = self._struct(atom_off, cell, pbc)
        pos, species, on_dev = self._inputs(pos, species)
        pairs = C.c_int64()
        self._check(self._L.gmp_tune(self._h, off.size - 1, off.ctypes.data, _ptr(pos), cell.ctypes.data,
                                     pbc.ctypes.data, _ptr(species), int(reps), C.byref(pairs),
                                     _stream_ptr(stream, on_dev)))
        vals = self.tuning()
        if cache:
            try:
                os.makedirs(os.path.dirname(TUNING_CACHE), exist_ok=True)
                known = {}
                if os.path.exists(TUNING_CACHE):
                    with open(TUNING_CACHE) as f:
                        known = json.load(f)
                known[key] = vals
                tmp = TUNING_CACHE + f".tmp{os.getpid()}"
                with open(tmp, "w") as f:
                    json.dump(known, f, indent=1)
                os.replace(tmp, TUNING_CACHE)
            except (OSError, ValueError):
                pass
        return {"key": key, "values": vals, "cached": False, "pairs": int(pairs.value)}

    def sync(self, stream=None, timeout_s: float = 0.0):
        torch = _torch()
        s = (stream if stream is not None else torch.cuda.current_stream()).cuda_stream
        self._check(self._L.gmp_sync(self._h, s, float(timeout_s)))


def _make_function():
    torch = _torch()

    class GMPFeatures(torch.autograd.Function):
        """features = GMPFeatures.apply(pos, featurizer, species, atom_off, cell, pbc).

        Forward: gmp_featurize.  Backward: gmp_featurize_vjp (recomputes the
        per-neighbor terms from the saved positions; no per-pair storage)."""

        @staticmethod
        def forward(ctx, pos, featurizer, species, atom_off, cell, pbc):
            ctx.featurizer = featurizer
            ctx.meta = (species, atom_off, cell, pbc)
            ctx.save_for_backward(pos)
            return featurizer.featurize(pos.detach(), species, atom_off, cell, pbc)

        @staticmethod
        def backward(ctx, grad_out):
            (pos,) = ctx.saved_tensors
            species, atom_off, cell, pbc = ctx.meta
            _, gp = ctx.featurizer.featurize_vjp(pos.detach(), species, atom_off, cell, pbc,
                                                 grad_out.contiguous().float(), want_features=False)
            return gp.to(pos.dtype), None, None, None, None, None

    return GMPFeatures


_fn_cache = {}


def probe_peaks(device: int = 0) -> dict:
    """Measured FP32 FMA (scalar, packed pairs) and ex2 throughput of a GPU
    at its present clocks (gmp_probe_peaks)."""
    L = load_library()
    a, b, c = C.c_double(), C.c_double(), C.c_double()
    st = L.gmp_probe_peaks(int(device), C.byref(a), C.byref(b), C.byref(c))
    if st != GMP_OK:
        raise GMPError(st, "gmp_probe_peaks failed")
    return {"fp32_fma_tflops": a.value, "fp32_fma2_tflops": b.value, "ex2_tops": c.value}


def probe_contraction(device: int = 0) -> dict:
    """The moment contraction as the forward kernel runs it (packed FP32)
    against a TF32x3 tensor-core version (gmp_probe_contraction): pairs/s,
    error relative to the cancellation-free scale, registers."""
    L = load_library()
    r = (C.c_double * 12)()
    st = L.gmp_probe_contraction(int(device), r, 12)
    if st != GMP_OK:
        raise GMPError(st, "gmp_probe_contraction failed")
    names = ("fp32", "tf32x3_16w", "tf32x3_8w", "tf32x3_presplit_16w")
    return {n: {"gpairs_per_s": r[k], "max_rel_err": r[4 + k], "registers": int(r[8 + k])}
            for k, n in enumerate(names)}


def probe_backward_contraction(device: int = 0) -> dict:
    """The backward kernel's per-pair adjoint contraction, FP32 as the
    kernel runs it against a tcgen05 (kind::tf32, hi/lo split) version
    (gmp_probe_backward_contraction): pairs/s, errors relative to the
    cancellation-free scale, registers."""
    L = load_library()
    r = (C.c_double * 9)()
    st = L.gmp_probe_backward_contraction(int(device), r, 9)
    if st != GMP_OK:
        raise GMPError(st, "gmp_probe_backward_contraction failed")
    return {"fp32": {"gpairs_per_s": r[0], "max_rel_err_lam": r[2], "max_rel_err_lamd": r[3], "registers": int(r[6])},
            "tcgen05_tf32x3": {"gpairs_per_s": r[1], "max_rel_err_lam": r[4], "max_rel_err_lamd": r[5],
                               "registers": int(r[7]), "wait_timed_out": bool(r[8])}}


def gmp_features(pos, featurizer, species, atom_off, cell, pbc):
    """Differentiable features (torch.autograd.Function around the C ABI)."""
    if "f" not in _fn_cache:
        _fn_cache["f"] = _make_function()
    return _fn_cache["f"].apply(pos, featurizer, species, atom_off, cell, pbc)
