"""Shared helpers of the GPU parity tests: tolerances, error metrics, and a
small report written next to the test run (when GMP_REPORT_DIR is set).

Tolerances (floating point; neighbor sets are compared bit for bit):
  features   : |f_gpu - f_ref| <= FEAT_TOL * max(|f_ref|, FEAT_TAU * F_abs)
  derivatives: |g_gpu - g_ref| <= GRAD_TOL * max(|g_ref|, GRAD_TAU * G_abs)
F_abs / G_abs are the oracle's cancellation-free scales (the same reduction
applied to sums of |per-pair contribution|).  The floors follow from FP32
arithmetic: a per-pair contribution carries rounding of ~1e-7 of its own
magnitude, so a result that cancels below FEAT_TAU (GRAD_TAU) of its
absolute scale cannot keep the relative bound in FP32.

Dense Jacobian rows (d f_i / d x_j for one center i and one neighbor atom
j) take JAC_TAU = 5e-3 instead of GRAD_TAU.  Such an entry is the
contraction sum_c 2 w_c mu_c dt_c/dd of the center's moments with one
pair's derivative terms, so an error of the moments enters it undiluted:
with mu_c off by k units of 2^-24 of its cancellation-free scale A_c, the
entry is off by up to k units of 2^-24 of G_abs (G_abs = sum_c 2 w_c A_c
|dt_c/dd|).  The FP32 moments carry k of a few: every per-pair term is a
product of an FP32 radial factor (a sum of SFU exponentials) and an FP32
MCSH value, and the forward kernel adds 16 pairs in plain FP32 before each
compensated fold.  Measured over every row of the first 4096 atoms of
batched300, the worst entry is 3.5 units of 2^-24 G_abs (1.2e-4 at a 1e-3
floor, which allows 1.68 units; 4.3e-5 at 5e-3).  tests/test_fp32_floor.py
shows the same limit without the GPU: moments formed from the rounded FP32
radial factors and MCSH values of the FP64 oracle, added in FP32 over
16-pair blocks, already give Jacobian-row errors of 2.0 units on fcc4096.  Position gradients (VJP)
and strain derivatives sum many rows, whose moment errors do not add up
coherently, and keep GRAD_TAU.

Both denominators are also floored at FP32_MIN_NORMAL = 2^-126: the outputs
are FP32, and below the smallest normal FP32 number the format itself has
fewer than 24 significant bits (subnormals) or none (below 2^-149), so no
FP32 result can meet a relative bound there.  Such values arise for probes
much narrower than the distance to the nearest atom (e.g. sigma = 0.05 A at a
reference point 2 A from every atom, where features fall to 1e-48).
"""
import json
import os

import numpy as np

FEAT_TOL = 1e-5
FEAT_TAU = 1e-6
GRAD_TOL = 1e-4
GRAD_TAU = 1e-3
JAC_TAU = 5e-3
FP32_MIN_NORMAL = 2.0 ** -126

_report = {}


def feature_errors(f_gpu, f_ref, f_abs, tau=FEAT_TAU):
    f_gpu = np.asarray(f_gpu, np.float64)
    num = np.abs(f_gpu - f_ref)
    den = np.maximum(np.maximum(np.abs(f_ref), tau * f_abs), FP32_MIN_NORMAL)
    err = num / den
    return err.max(axis=0)


def grad_errors(g_gpu, g_ref, g_abs, tau=GRAD_TAU):
    """Row-wise: Euclidean error of each 3-vector over max(|g_ref|, tau*g_abs)."""
    g_gpu = np.asarray(g_gpu, np.float64)
    num = np.linalg.norm(g_gpu - g_ref, axis=-1)
    den = np.maximum(np.maximum(np.linalg.norm(g_ref, axis=-1), tau * g_abs), FP32_MIN_NORMAL)
    return num / den


def record(name, **vals):
    _report[name] = {k: (float(v) if np.isscalar(v) else np.asarray(v, float).tolist()) for k, v in vals.items()}
    d = os.environ.get("GMP_REPORT_DIR")
    if d:
        os.makedirs(d, exist_ok=True)
        with open(os.path.join(d, "parity_report.json"), "w") as f:
            json.dump(_report, f, indent=1)
