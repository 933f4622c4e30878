"""The C ABI library loads and exports every symbol declared in include/gmp.h
(no compute call: this runs without a GPU)."""
import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    text = open(os.path.join(ROOT, "include", "gmp.h")).read()
    return sorted(set(re.findall(r"^\s*(?:gmp_status|const char|int64_t|void)\s*\*?\s*(gmp_\w+)\s*\(", text, re.M)))


def test_header_declares_the_boundary():
    names = _declared()
    for n in ("gmp_create", "gmp_featurize", "gmp_featurize_vjp", "gmp_featurize_grad",
              "gmp_neighbors", "gmp_sync", "gmp_last_error", "gmp_destroy"):
        assert n in names


def test_library_exports_every_declared_symbol():
    from paper_2303_12980_gb300 import build
    path = build.build()
    lib = ctypes.CDLL(path)
    for n in _declared():
        assert hasattr(lib, n), n


def test_binding_fails_loudly_without_device():
    import pytest
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_2303_12980_gb300.binding import GMPError, GMPFeaturizer
    with pytest.raises(GMPError):
        GMPFeaturizer([0], [0.5], 5.0, [1], [1.0], [1.0])


def test_generated_mcsh_header_is_current():
    import subprocess
    import sys
    import tempfile
    csrc = os.path.join(ROOT, "paper_2303_12980_gb300", "csrc")
    with tempfile.TemporaryDirectory() as d:
        out = os.path.join(d, "mcsh_gen.cuh")
        subprocess.run([sys.executable, os.path.join(csrc, "gen_mcsh.py"), out], check=True)
        assert open(out).read() == open(os.path.join(csrc, "mcsh_gen.cuh")).read()


def test_create_rejects_invalid_parameters_before_the_device():
    """Host-side validation of gmp_params runs before any CUDA call: these
    fail with GMP_ERR_INVALID_ARG on a machine without a GPU too."""
    import ctypes as C
    from paper_2303_12980_gb300 import build
    from paper_2303_12980_gb300.binding import _Params, load_library
    build.build()
    L = load_library()
    n_gauss = (C.c_int32 * 1)(1)
    coef = (C.c_double * 1)(1.0)
    expo = (C.c_double * 1)(1.0)
    orders = (C.c_int32 * 2)(0, 0)
    sig = (C.c_double * 1)(0.5)
    def create(**kw):
        args = dict(n_elements=1, n_gauss=C.addressof(n_gauss), gauss_coef=C.addressof(coef),
                    gauss_exp=C.addressof(expo), n_orders=1, orders=C.addressof(orders), n_sigmas=1,
                    sigmas=C.addressof(sig), cutoff=5.0, flags=0, overlap_threshold=1e-16)
        args.update(kw)
        h = C.c_void_p()
        return L.gmp_create(C.byref(_Params(**args)), 0, C.byref(h))
    INVALID = 1
    assert create(flags=1) == INVALID
    assert create(n_orders=2) == INVALID            # repeated order
    assert create(cutoff=float("inf")) == INVALID
    assert create(cutoff=0.0, overlap_threshold=0.0) == INVALID
    expo[0] = -1.0
    assert create() == INVALID                      # exponent <= 0


def test_entry_points_reject_a_null_handle():
    """Every featurize entry point returns GMP_ERR_INVALID_ARG for a null
    handle before touching the device (runs without a GPU)."""
    import ctypes as C
    from paper_2303_12980_gb300 import build
    from paper_2303_12980_gb300.binding import load_library
    build.build()
    L = load_library()
    nnz = C.c_int64(-1)
    off = (C.c_int64 * 2)(0, 1)
    INVALID = 1
    common = (None, 1, C.addressof(off), None, None, None, None)
    assert L.gmp_featurize(*common, None, None) == INVALID
    assert L.gmp_featurize_vjp(*common, None, None, None, None) == INVALID
    assert L.gmp_featurize_grad(*common, None, None, None, None, 0, C.byref(nnz), None) == INVALID
    assert L.gmp_featurize_grad_centers(*common, 0, 1, None, None, None, None, 0, C.byref(nnz), None) == INVALID
    assert L.gmp_neighbors(*common, None, None, None, 0, C.byref(nnz), None) == INVALID
