"""Why dense Jacobian rows take the floor JAC_TAU and not GRAD_TAU
(tests/parity.py): an error of the FP32 moments enters a Jacobian entry
undiluted, and FP32 moments alone, however they are summed, carry a few
units of 2^-24 of their cancellation-free scale.

The test computes, with the FP64 oracle, the per-pair moment
contributions t = R_{l,sigma}(r^2) S_c(d) of some centers of fcc4096 and
their displacement derivatives, and forms the moments as an FP32 kernel
would at best: each term the rounded product of the rounded radial
factor and the rounded MCSH value, added in FP32 over blocks of 16 pairs,
the block sums combined exactly.  The resulting error of each Jacobian
row, d f_{l,sigma} / d x_j = sum_c 2 w_c mu_c sum_{images of j} dt_c / dd,
is measured in units of 2^-24 of the oracle's row scale jac_abs.  At the
parity tolerance GRAD_TOL a floor tau admits GRAD_TOL * tau / 2^-24 such
units: 1.68 at tau = 1e-3, 8.4 at tau = 5e-3.  The emulation exceeds the
first (no FP32-moment implementation can meet it) and stays inside the
second.  No GPU code is involved."""
import math

import numpy as np
import pytest

from paper_2303_12980_gb300 import synth
from parity import GRAD_TAU, GRAD_TOL, JAC_TAU

pytestmark = pytest.mark.timeout(600)


def _weight(a, b, c):
    return math.factorial(a + b + c) / (math.factorial(a) * math.factorial(b) * math.factorial(c))


def _radial(w, el, sig, l, r2):
    """R_{l,sigma}(r^2) of element el: the overlap of each Gaussian of the
    element's density with the order-l probe of width sigma, closed form."""
    beta = 1.0 / (2.0 * sig * sig)
    out = np.zeros_like(r2)
    for g in range(w.gauss_off[el], w.gauss_off[el + 1]):
        a, c = w.gauss_exp[g], w.gauss_coef[g]
        gam = a + beta
        out += (c * (2.0 * math.pi * sig * sig) ** -1.5 * (math.pi / gam) ** 1.5 * (a / gam) ** l
                * np.exp(-(a * beta / gam) * r2))
    return out


def test_fp32_moments_exceed_the_gradient_floor_in_jacobian_rows(oracle_mod):
    O = oracle_mod
    w = synth.workload("fcc4096")
    orders = [l for l in w.orders if l >= 0]
    assert orders == list(w.orders)  # no density column: moment columns start at 0
    cols = [(l, s, abc) for l in orders for s in range(len(w.sigmas)) for abc in O.components(l)]
    feats = [(l, s) for l in orders for s in range(len(w.sigmas))]
    W = np.array([_weight(*abc) for (_, _, abc) in cols])
    sel = [np.array([(cl, cs) == f for (cl, cs, _) in cols]) for f in feats]
    polys = [O.mcsh_poly(*abc) for (_, _, abc) in cols]
    units = []
    centers = np.random.default_rng(5).choice(w.n_atoms, 12, replace=False)
    for i in centers:
        t, dt = O.pair_terms(w, int(i))
        off, jj, _, d = O.neighbors(w, [int(i)])
        jj, d = jj[off[0]:off[1]], d[off[0]:off[1]]
        r2 = (d * d).sum(1)
        el = w.species[jj]
        S = np.stack([sum(co * d[:, 0] ** p * d[:, 1] ** q * d[:, 2] ** r for (p, q, r), co in poly.items())
                      for poly in polys], axis=1)
        R = np.zeros_like(S)
        for k, (l, s, _) in enumerate(cols):
            for e in np.unique(el):
                m = el == e
                R[m, k] = _radial(w, e, w.sigmas[s], l, r2[m])
        # the factorisation reproduces the oracle's terms
        assert np.abs(R * S - t).max() <= 1e-12 * np.abs(t).max()
        t32 = R.astype(np.float32) * S.astype(np.float32)
        mu32 = np.zeros(len(cols))
        for b0 in range(0, len(d), 16):
            part = np.zeros(len(cols), np.float32)
            for p in range(b0, min(len(d), b0 + 16)):
                part = part + t32[p]
            mu32 += part.astype(np.float64)
        dmu = mu32 - t.sum(0)
        jo, jrow, _, jabs = O.jacobian_rows(w, [int(i)], want_abs=True)
        for r, a in enumerate(jrow[jo[0]:jo[1]]):
            if a == i:
                continue  # the center's own row is minus the sum of the others
            g = dt[jj == a].sum(0)
            err = 2.0 * (W * dmu)[:, None] * g
            for fi, m in enumerate(sel):
                scale = jabs[jo[0] + r, fi]
                if scale > 0:
                    units.append(np.linalg.norm(err[m].sum(0)) / scale / 2.0 ** -24)
    worst = max(units)
    print("worst Jacobian-row error of FP32 moments: %.2f units of 2^-24 jac_abs" % worst)
    assert worst > GRAD_TOL * GRAD_TAU / 2.0 ** -24, worst   # 1.68 units: the VJP floor cannot hold
    assert worst < GRAD_TOL * JAC_TAU / 2.0 ** -24, worst    # 8.4 units: the Jacobian floor does
