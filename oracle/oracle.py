"""Python driver for the FP64 CPU oracle (gmp_oracle.c).

TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the
benchmark's CPU-baseline leg may import this module; the product path
(the CUDA library and its binding) never does, and this module imports
nothing from the product package.

The C core implements the GMP definitions step by step (neighbor images,
MCSH polynomials from differentiating 1/r, Gaussian overlap integrals from
1-D moments, the weighted sum of squares per (order, sigma), and the
position derivatives); see the header of gmp_oracle.c for the steps and the
readings they take where the paper (GMP-Featurizer, arXiv 2303.12980) defers
to its GMP reference.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gmp_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

CFLAGS = ["-O2", "-fopenmp", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
          "-std=c11", "-D_DEFAULT_SOURCE", "-Wall"]


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no FMA contraction) into oracle/_build."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.run(["gcc", *CFLAGS, _SRC, "-o", tmp, "-lm"], check=True)
        os.replace(tmp, _LIB)
    return _LIB


class _Problem(C.Structure):
    _fields_ = [
        ("n_struct", C.c_int32),
        ("atom_off", C.c_void_p),
        ("pos", C.c_void_p),
        ("cell", C.c_void_p),
        ("pbc", C.c_void_p),
        ("species", C.c_void_p),
        ("n_elements", C.c_int32),
        ("gauss_off", C.c_void_p),
        ("gauss_coef", C.c_void_p),
        ("gauss_exp", C.c_void_p),
        ("n_orders", C.c_int32),
        ("orders", C.c_void_p),
        ("n_sigmas", C.c_int32),
        ("sigmas", C.c_void_p),
        ("cutoff", C.c_double),
    ]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = C.CDLL(build())
            P = C.POINTER(_Problem)
            vp = C.c_void_p
            L.oracle_mcsh_poly.argtypes = [C.c_int, C.c_int, C.c_int, vp]
            L.oracle_num_features.argtypes = [P]
            L.oracle_num_moment_columns.argtypes = [P]
            L.oracle_neighbor_counts.argtypes = [P, C.c_int64, vp, vp]
            L.oracle_neighbor_lists.argtypes = [P, C.c_int64, vp, vp, vp, vp, vp]
            L.oracle_features.argtypes = [P, C.c_int64, vp, vp, vp, vp]
            L.oracle_point_features.argtypes = [P, C.c_int64, vp, vp, vp, vp]
            L.oracle_virial.argtypes = [P, vp, vp, vp]
            L.oracle_jacobian_counts.argtypes = [P, C.c_int64, vp, vp]
            L.oracle_jacobian_rows.argtypes = [P, C.c_int64, vp, vp, vp, vp, vp]
            L.oracle_pair_terms.argtypes = [P, C.c_int64, C.c_int64, vp, vp]
            _lib = L
    return _lib


def num_threads() -> int:
    return int(lib().oracle_num_threads())


def mcsh_poly(a: int, b: int, c: int) -> dict:
    """Integer coefficients {(p, q, s): coef} of S_abc (x^p y^q z^s)."""
    l = a + b + c
    out = np.zeros((l + 1) * (l + 1), np.int64)
    if lib().oracle_mcsh_poly(a, b, c, out.ctypes.data) != 0:
        raise ValueError("order out of range")
    res = {}
    for p in range(l + 1):
        for q in range(l + 1 - p):
            k = int(out[p * (l + 1) + q])
            if k:
                res[(p, q, l - p - q)] = k
    return res


def components(l: int):
    """Component order inside one order l (a descending, then b descending)."""
    return [(a, b, l - a - b) for a in range(l, -1, -1) for b in range(l - a, -1, -1)]


class Problem:
    """Keeps the numpy arrays alive behind the C struct."""

    def __init__(self, w):
        self.w = w
        self._arrs = dict(
            atom_off=np.ascontiguousarray(w.atom_off, np.int64),
            pos=np.ascontiguousarray(w.positions, np.float64),
            cell=np.ascontiguousarray(w.cells, np.float64),
            pbc=np.ascontiguousarray(w.pbc, np.uint8),
            species=np.ascontiguousarray(w.species, np.int32),
            gauss_off=np.ascontiguousarray(w.gauss_off, np.int32),
            gauss_coef=np.ascontiguousarray(w.gauss_coef, np.float64),
            gauss_exp=np.ascontiguousarray(w.gauss_exp, np.float64),
            orders=np.ascontiguousarray(w.orders, np.int32),
            sigmas=np.ascontiguousarray(w.sigmas, np.float64),
        )
        a = self._arrs
        self.s = _Problem(
            n_struct=w.n_struct, atom_off=a["atom_off"].ctypes.data, pos=a["pos"].ctypes.data,
            cell=a["cell"].ctypes.data, pbc=a["pbc"].ctypes.data,
            species=a["species"].ctypes.data, n_elements=w.n_elements,
            gauss_off=a["gauss_off"].ctypes.data, gauss_coef=a["gauss_coef"].ctypes.data,
            gauss_exp=a["gauss_exp"].ctypes.data, n_orders=len(w.orders),
            orders=a["orders"].ctypes.data, n_sigmas=len(w.sigmas),
            sigmas=a["sigmas"].ctypes.data, cutoff=float(w.cutoff),
        )
        self.F = lib().oracle_num_features(C.byref(self.s))
        if self.F < 0:
            raise ValueError("unsupported orders")
        self.ncol = lib().oracle_num_moment_columns(C.byref(self.s))


def _centers(w, centers):
    if centers is None:
        return np.arange(w.n_atoms, dtype=np.int64)
    return np.ascontiguousarray(centers, np.int64)


def neighbors(w, centers=None):
    """Exact neighbor images: (offsets [nc+1], j [P], shift [P,3], d [P,3]),
    each center's list ordered by (j, n1, n2, n3)."""
    P = Problem(w)
    c = _centers(w, centers)
    counts = np.zeros(c.size, np.int64)
    if lib().oracle_neighbor_counts(C.byref(P.s), c.size, c.ctypes.data, counts.ctypes.data):
        raise ValueError("singular periodic cell")
    off = np.concatenate([[0], np.cumsum(counts)]).astype(np.int64)
    j = np.zeros(off[-1], np.int32)
    sh = np.zeros((off[-1], 3), np.int32)
    d = np.zeros((off[-1], 3), np.float64)
    if lib().oracle_neighbor_lists(C.byref(P.s), c.size, c.ctypes.data, off.ctypes.data,
                                   j.ctypes.data, sh.ctypes.data, d.ctypes.data):
        raise RuntimeError("neighbor listing failed")
    return off, j, sh, d


def features(w, centers=None, want_abs=False, want_mu=False):
    """FP64 features [nc, F]; optionally the cancellation-free scale F_abs
    (same reduction of sums of |per-pair contribution|) and raw moments."""
    P = Problem(w)
    c = _centers(w, centers)
    f = np.zeros((c.size, P.F), np.float64)
    fa = np.zeros((c.size, P.F), np.float64) if want_abs else None
    mu = np.zeros((c.size, P.ncol), np.float64) if want_mu else None
    rc = lib().oracle_features(C.byref(P.s), c.size, c.ctypes.data, f.ctypes.data,
                               fa.ctypes.data if want_abs else None,
                               mu.ctypes.data if want_mu else None)
    if rc:
        raise ValueError("oracle_features failed")
    out = [f]
    if want_abs:
        out.append(fa)
    if want_mu:
        out.append(mu)
    return out[0] if len(out) == 1 else tuple(out)


def point_features(w, points, point_struct, want_abs=False):
    """FP64 features at reference points [n,3] of structures point_struct [n]."""
    P = Problem(w)
    pts = np.ascontiguousarray(points, np.float64)
    ps = np.ascontiguousarray(point_struct, np.int32)
    f = np.zeros((ps.size, P.F), np.float64)
    fa = np.zeros((ps.size, P.F), np.float64) if want_abs else None
    if lib().oracle_point_features(C.byref(P.s), ps.size, pts.ctypes.data, ps.ctypes.data, f.ctypes.data,
                                   fa.ctypes.data if want_abs else None):
        raise ValueError("oracle_point_features failed")
    return (f, fa) if want_abs else f


def virial(w, g, want_abs=False):
    """Per-structure strain derivative W[s,a,b] = dL/d eps_ab of
    L = sum_i sum_f g[i,f] f_i (positions and lattice vectors strained
    alike), i.e. the sum over the structure's pairs of (dL/dd)_a d_b."""
    P = Problem(w)
    gg = np.ascontiguousarray(g, np.float64)
    W = np.zeros((w.n_struct, 3, 3), np.float64)
    Wa = np.zeros((w.n_struct, 3, 3), np.float64) if want_abs else None
    if lib().oracle_virial(C.byref(P.s), gg.ctypes.data, W.ctypes.data, Wa.ctypes.data if want_abs else None):
        raise ValueError("oracle_virial failed")
    return (W, Wa) if want_abs else W


def pair_terms(w, center):
    """Per-pair moment contributions of one center, in the order of
    neighbors(w, [center]): t [m, ncol] and dt [m, ncol, 3] = d t / d d, the
    columns ordered (order slot, sigma, component) as the moments of
    features(..., want_mu=True)."""
    P = Problem(w)
    c = np.array([center], np.int64)
    counts = np.zeros(1, np.int64)
    if lib().oracle_neighbor_counts(C.byref(P.s), 1, c.ctypes.data, counts.ctypes.data):
        raise ValueError("singular periodic cell")
    m = int(counts[0])
    t = np.zeros((m, P.ncol), np.float64)
    dt = np.zeros((m, P.ncol, 3), np.float64)
    if lib().oracle_pair_terms(C.byref(P.s), int(center), m, t.ctypes.data, dt.ctypes.data):
        raise RuntimeError("pair terms failed")
    return t, dt


def jacobian_rows(w, centers=None, want_abs=False):
    """d f_i / d x_j for the listed centers: (offsets [nc+1], j [nnz],
    jac [nnz, F, 3]); j ascending within each center's row.  With want_abs,
    also jac_abs [nnz, F]: the cancellation-free scale of each block (sum of
    2 w_c A_c |d t_c / d d| over its pairs, A_c = sum of |t_c|)."""
    P = Problem(w)
    c = _centers(w, centers)
    counts = np.zeros(c.size, np.int64)
    if lib().oracle_jacobian_counts(C.byref(P.s), c.size, c.ctypes.data, counts.ctypes.data):
        raise ValueError("singular periodic cell")
    off = np.concatenate([[0], np.cumsum(counts)]).astype(np.int64)
    j = np.zeros(off[-1], np.int32)
    jac = np.zeros((off[-1], P.F, 3), np.float64)
    jab = np.zeros((off[-1], P.F), np.float64) if want_abs else None
    if lib().oracle_jacobian_rows(C.byref(P.s), c.size, c.ctypes.data, off.ctypes.data,
                                  j.ctypes.data, jac.ctypes.data,
                                  jab.ctypes.data if want_abs else None):
        raise RuntimeError("jacobian failed")
    if want_abs:
        return off, j, jac, jab
    return off, j, jac


def vjp_atoms(w, g, atoms, want_abs=False):
    """dL/dx_a = sum_i sum_f g[i,f] d f_i / d x_a for the listed atoms.
    The centers that see atom a are exactly the atoms in a's own neighbor
    list (the neighbor relation is symmetric), so only those rows are built.
    With want_abs also the scale sum_i sum_f |g[i,f]| jac_abs[i,f,a]."""
    atoms = np.ascontiguousarray(atoms, np.int64)
    off, j, _, _ = neighbors(w, atoms)
    need = np.unique(j.astype(np.int64))
    joff, jj, jac, jab = jacobian_rows(w, need, want_abs=True)
    row_of = {int(c): k for k, c in enumerate(need)}
    out = np.zeros((atoms.size, 3), np.float64)
    scale = np.zeros(atoms.size, np.float64)
    for t, a in enumerate(atoms):
        centers_a = np.unique(j[off[t]:off[t + 1]])
        for ci in centers_a:
            k = row_of[int(ci)]
            js = jj[joff[k]:joff[k + 1]]
            pos = np.searchsorted(js, a)
            if pos < js.size and js[pos] == a:
                gi = g[ci].astype(np.float64)
                out[t] += np.einsum("f,fk->k", gi, jac[joff[k] + pos])
                scale[t] += np.abs(gi) @ jab[joff[k] + pos]
    if want_abs:
        return out, scale
    return out
