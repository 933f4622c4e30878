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
