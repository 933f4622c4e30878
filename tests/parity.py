"""Shared helpers of the GPU parity tests: tolerances, error metrics, and a
small report written next to the test run (when GMP_REPORT_DIR is set).

Tolerances (floating point; neighbor sets are compared bit for bit):
  features   : |f_gpu - f_ref| <= FEAT_TOL * max(|f_ref|, FEAT_TAU * F_abs)
  derivatives: |g_gpu - g_ref| <= GRAD_TOL * max(|g_ref|, GRAD_TAU * G_abs)
F_abs / G_abs are the oracle's cancellation-free scales (the same reduction
applied to sums of |per-pair contribution|).  See the design doc for how the
floors follow from FP32 arithmetic.
"""
import json
import os

import numpy as np

FEAT_TOL = 1e-5
FEAT_TAU = 1e-6
GRAD_TOL = 1e-4
GRAD_TAU = 1e-3

_report = {}


def feature_errors(f_gpu, f_ref, f_abs, tau=FEAT_TAU):
    f_gpu = np.asarray(f_gpu, np.float64)
    num = np.abs(f_gpu - f_ref)
    den = np.maximum(np.abs(f_ref), tau * f_abs)
    # an exactly zero feature with a zero scale (e.g. l >= 1 of an isolated
    # atom) must come out exactly zero
    err = np.where(num == 0.0, 0.0, num / np.where(den > 0.0, den, 1e-300))
    return err.max(axis=0)


def grad_errors(g_gpu, g_ref, g_abs, tau=GRAD_TAU):
    """Row-wise: Euclidean error of each 3-vector over max(|g_ref|, tau*g_abs)."""
    g_gpu = np.asarray(g_gpu, np.float64)
    num = np.linalg.norm(g_gpu - g_ref, axis=-1)
    den = np.maximum(np.linalg.norm(g_ref, axis=-1), tau * g_abs)
    return np.where(num == 0.0, 0.0, num / np.where(den > 0.0, den, 1e-300))


def record(name, **vals):
    _report[name] = {k: (float(v) if np.isscalar(v) else np.asarray(v, float).tolist()) for k, v in vals.items()}
    d = os.environ.get("GMP_REPORT_DIR")
    if d:
        os.makedirs(d, exist_ok=True)
        with open(os.path.join(d, "parity_report.json"), "w") as f:
            json.dump(_report, f, indent=1)
