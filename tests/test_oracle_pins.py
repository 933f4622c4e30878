"""Pins of the FP64 CPU oracle to facts that do not come from the oracle itself:
symbolic differentiation, exact polynomial identities, numerical quadrature of
the defining integral, a second closed-form route (Gaussian mean-value
property of harmonic polynomials), brute-force neighbor enumeration, symmetry
invariances, and central finite differences.

The method (GMP-Featurizer, arXiv 2303.12980): features = overlap of the
Gaussian electron density with MCSH angular x Gaussian radial probes, grouped
by (order, sigma) and reduced to rotation invariants; derivatives w.r.t.
positions (Examples).  The integral definitions are those written in the
header of oracle/gmp_oracle.c.
"""
import math
import os

import numpy as np
import pytest

from paper_2303_12980_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ------------------------------------------------------------ polynomials
def _laplacian(poly):
    out = {}
    for (p, q, s), k in poly.items():
        for ax, e in enumerate((p, q, s)):
            if e >= 2:
                m = [p, q, s]
                m[ax] -= 2
                out[tuple(m)] = out.get(tuple(m), 0) + k * e * (e - 1)
    return {m: v for m, v in out.items() if v}


def _pmul(a, b):
    out = {}
    for m1, v1 in a.items():
        for m2, v2 in b.items():
            m = (m1[0] + m2[0], m1[1] + m2[1], m1[2] + m2[2])
            out[m] = out.get(m, 0) + v1 * v2
    return {m: v for m, v in out.items() if v}


def _r2pow(n):
    p = {(0, 0, 0): 1}
    for _ in range(n):
        p = _pmul(p, {(2, 0, 0): 1, (0, 2, 0): 1, (0, 0, 2): 1})
    return p


def test_mcsh_matches_symbolic_differentiation(oracle_mod):
    sp = pytest.importorskip("sympy")
    x, y, z = sp.symbols("x y z")
    r = sp.sqrt(x * x + y * y + z * z)
    for l in range(0, 5):
        for (a, b, c) in oracle_mod.components(l):
            expr = sp.expand(sp.simplify((-1) ** l * r ** (2 * l + 1) * sp.diff(1 / r, x, a, y, b, z, c)))
            want = {}
            for term in sp.Add.make_args(expr):
                coef, mono = term.as_coeff_Mul()
                pw = sp.Poly(mono, x, y, z).monoms()[0] if mono != 1 else (0, 0, 0)
                want[tuple(int(t) for t in pw)] = int(coef)
            assert oracle_mod.mcsh_poly(a, b, c) == want, (a, b, c)


def test_mcsh_harmonic_and_sum_rule(oracle_mod):
    # Laplacian zero; sum_abc l!/(a!b!c!) S_abc^2 = l! (2l-1)!! r^(2l)
    for l in range(0, 7):
        total = {}
        for (a, b, c) in oracle_mod.components(l):
            P = oracle_mod.mcsh_poly(a, b, c)
            assert _laplacian(P) == {}, (a, b, c)
            w = math.factorial(l) // (math.factorial(a) * math.factorial(b) * math.factorial(c))
            for m, v in _pmul(P, P).items():
                total[m] = total.get(m, 0) + w * v
        dfact = 1
        for k in range(2 * l - 1, 0, -2):
            dfact *= k
        want = {m: v * math.factorial(l) * dfact for m, v in _r2pow(l).items()}
        assert total == want, l


def test_mcsh_golden_low_orders(oracle_mod):
    # tests/golden/mcsh_low_orders.txt: explicit polynomials of the
    # definition S_abc = (-1)^l r^(2l+1) d^abc (1/r), written out by hand
    with open(os.path.join(GOLDEN, "mcsh_low_orders.txt")) as f:
        for line in f:
            line = line.split("#")[0].strip()
            if not line:
                continue
            lhs, rhs = line.split(":")
            a, b, c = (int(t) for t in lhs.split())
            want = {}
            for tok in rhs.split(","):
                k, p, q, s = (int(t) for t in tok.split())
                want[(p, q, s)] = k
            assert oracle_mod.mcsh_poly(a, b, c) == want, line


# ------------------------------------------------------------ tiny systems
def _cluster(pos, species, orders, sigmas, coef, expo, n_gauss, cutoff=12.0):
    pos = np.asarray(pos, np.float64)
    return synth.Workload(
        name="tiny", positions=pos, cells=np.zeros((1, 3, 3)), pbc=np.zeros((1, 3), np.uint8),
        atom_off=np.array([0, len(pos)], np.int64), species=np.asarray(species, np.int32),
        n_gauss=np.asarray(n_gauss, np.int32), gauss_coef=np.asarray(coef, np.float64),
        gauss_exp=np.asarray(expo, np.float64), orders=list(orders), sigmas=list(sigmas), cutoff=cutoff)


def test_order0_single_pair_matches_1d_quadrature(oracle_mod):
    from scipy.integrate import quad
    d = np.array([0.7, -0.4, 1.1])
    alpha, c, sig = 1.3, 0.8, 0.45
    w = _cluster([[0, 0, 0], d], [0, 0], [0], [sig], [c], [alpha], [1])
    mu = oracle_mod.features(w, [0], want_mu=True)[1][0]
    beta = 1.0 / (2 * sig * sig)
    Ns = (2 * math.pi * sig * sig) ** -1.5

    def axis(dd):
        return quad(lambda t: math.exp(-beta * t * t - alpha * (t - dd) ** 2), -20, 20, epsabs=0, epsrel=1e-13)[0]

    want = c * Ns * (np.prod([axis(0.0)] * 3) + np.prod([axis(v) for v in d]))
    assert abs(mu[0] - want) <= 1e-12 * abs(want)


def test_moments_match_3d_quadrature(oracle_mod):
    # two atoms, one element with two Gaussians, orders 0..3, one sigma:
    # mu_{l,abc} = int N_s S_abc(r) exp(-beta r^2) rho(r) d^3r on a grid
    pos = np.array([[0.0, 0.0, 0.0], [0.9, -0.6, 0.5], [-0.5, 0.8, -0.7]])
    coef, expo = [0.7, 0.4], [1.6, 0.6]
    sig = 0.55
    w = _cluster(pos, [0, 0, 0], [0, 1, 2, 3], [sig], coef, expo, [2])
    mu = oracle_mod.features(w, [0], want_mu=True)[1][0]
    h = 0.05
    g = np.arange(-5.0, 5.0 + h / 2, h)
    X, Y, Z = np.meshgrid(g, g, g, indexing="ij")
    beta = 1.0 / (2 * sig * sig)
    Ns = (2 * math.pi * sig * sig) ** -1.5
    rho = np.zeros_like(X)
    for p in pos:
        R2 = (X - p[0]) ** 2 + (Y - p[1]) ** 2 + (Z - p[2]) ** 2
        for c, a in zip(coef, expo):
            rho += c * np.exp(-a * R2)
    base = Ns * np.exp(-beta * (X * X + Y * Y + Z * Z)) * rho * h ** 3
    col = 0
    for l in [0, 1, 2, 3]:
        for (a, b, c) in oracle_mod.components(l):
            P = oracle_mod.mcsh_poly(a, b, c)
            S = sum(k * X ** pp * Y ** qq * Z ** ss for (pp, qq, ss), k in P.items())
            want = float(np.sum(S * base))
            scale = float(np.sum(np.abs(S) * base))
            assert abs(mu[col] - want) <= 1e-9 * scale, (l, a, b, c, mu[col], want)
            col += 1


def _grid_moments(pos, coef, expo, sig, orders, center, h, half):
    """Moments mu_{l,abc} = sum over a grid of N_s S_abc(r) exp(-beta r^2)
    rho(r + center) h^3, every component of the listed orders, and the
    matching sums of |S| (the scale the comparison is relative to).  The
    trapezoid rule on these Gaussian integrands converges spectrally: at
    h = 0.2 A and alpha + beta <= 4.1 A^-2 the aliasing error is of the
    order of exp(-pi^2 / (h^2 (alpha + beta))) < 1e-26 of the integral."""
    import oracle.oracle as O
    g = np.arange(-half, half + h / 2, h)
    X, Y, Z = np.meshgrid(g, g, g, indexing="ij")
    beta = 1.0 / (2 * sig * sig)
    Ns = (2 * math.pi * sig * sig) ** -1.5
    rho = np.zeros_like(X)
    for p in np.asarray(pos) - center:
        R2 = (X - p[0]) ** 2 + (Y - p[1]) ** 2 + (Z - p[2]) ** 2
        for c, a in zip(coef, expo):
            rho += c * np.exp(-a * R2)
    base = Ns * np.exp(-beta * (X * X + Y * Y + Z * Z)) * rho * h ** 3
    lmax = max(orders)
    Xp, Yp, Zp = [np.ones_like(X)], [np.ones_like(X)], [np.ones_like(X)]
    for _ in range(lmax):
        Xp.append(Xp[-1] * X)
        Yp.append(Yp[-1] * Y)
        Zp.append(Zp[-1] * Z)
    mu, scale = [], []
    for l in orders:
        for (a, b, c) in O.components(l):
            S = np.zeros_like(X)
            for (pp, qq, ss), k in O.mcsh_poly(a, b, c).items():
                S += k * Xp[pp] * Yp[qq] * Zp[ss]
            mu.append(float(np.sum(S * base)))
            scale.append(float(np.sum(np.abs(S) * base)))
    return np.array(mu), np.array(scale)


@pytest.mark.parametrize("sig", [0.45, 0.8])
def test_high_order_moments_match_3d_quadrature(oracle_mod, sig):
    # orders 4, 5, 6 (every component): the oracle's 1-D moment route at the
    # orders the slab workload runs, against the defining integral on a grid
    pos = np.array([[0.0, 0.0, 0.0], [0.9, -0.6, 0.5], [-0.5, 0.8, -0.7], [1.2, 0.4, 1.0]])
    coef, expo = [0.7, 0.4], [1.6, 0.6]
    w = _cluster(pos, [0, 0, 0, 0], [4, 5, 6], [sig], coef, expo, [2])
    mu = oracle_mod.features(w, [0], want_mu=True)[1][0]
    want, scale = _grid_moments(pos, coef, expo, sig, [4, 5, 6], np.zeros(3), 0.2, 7.0)
    assert mu.shape == want.shape
    assert np.all(np.abs(mu - want) <= 1e-12 * scale), np.max(np.abs(mu - want) / scale)


def test_high_order_point_features_match_3d_quadrature(oracle_mod):
    # features (weighted sums of squares over all components) of orders 4-6
    # at a point that is not an atom
    pos = np.array([[0.0, 0.0, 0.0], [0.9, -0.6, 0.5], [-0.5, 0.8, -0.7]])
    coef, expo = [0.7, 0.4], [1.6, 0.6]
    sig = 0.6
    p = np.array([0.35, 0.2, -0.15])
    w = _cluster(pos, [0, 0, 0], [4, 5, 6], [sig], coef, expo, [2])
    f = oracle_mod.point_features(w, p[None, :], [0])[0]
    mu, mu_abs = _grid_moments(pos, coef, expo, sig, [4, 5, 6], p, 0.2, 7.0)
    k = 0
    for col, l in enumerate([4, 5, 6]):
        want = scale = 0.0
        for (a, b, c) in oracle_mod.components(l):
            wt = math.factorial(l) / (math.factorial(a) * math.factorial(b) * math.factorial(c))
            want += wt * mu[k] * mu[k]
            scale += wt * mu_abs[k] * mu_abs[k]
            k += 1
        assert abs(f[col] - want) <= 1e-11 * scale, (l, f[col], want)


@pytest.mark.parametrize("orders,sigmas", [
    ([0, 1, 2], None),
    # the slab's probe set: orders 0-6, 16 sigmas log-spaced in 0.05-1.5 A
    ([0, 1, 2, 3, 4, 5, 6], list(np.geomspace(0.05, 1.5, 16))),
])
def test_factorised_route_agrees(oracle_mod, orders, sigmas):
    # Mean-value property: the Gaussian average of a harmonic polynomial is
    # its value at the Gaussian's centre, so each overlap integral equals
    # c N_s (pi/g)^1.5 (alpha/g)^l exp(-(alpha beta/g) r^2) S_abc(d).
    # The oracle instead sums the polynomial's monomials against 1-D
    # Gaussian moments, and that sum cancels: for a narrow probe and a small
    # density exponent the product Gaussian's variance 1/(2g) dwarfs its
    # centre P = (alpha/g) d, the monomial moments are ~var^(l/2) while the
    # harmonic combination leaves ~|P|^l.  Its FP64 rounding error is then
    # bounded by a few units of 2^-53 times the sum of the magnitudes it
    # adds, K |coef| a_p a_q a_s with a_n the moments of the same recursion
    # taken with |P| (every term non-negative): the tolerance below is
    # 1e-12 of the factorised scale plus 2^-46 of that summation scale.
    w = synth.workload("random64_box").replace(orders=orders)
    if sigmas is not None:
        w = w.replace(sigmas=sigmas)
    centers = np.array([0, 5, 17, 40])
    f, mu = oracle_mod.features(w, centers, want_mu=True)
    off, j, sh, d = oracle_mod.neighbors(w, centers)
    go = w.gauss_off
    col = 0
    cols = []
    for l in w.orders:
        for s in range(len(w.sigmas)):
            for abc in oracle_mod.components(l):
                cols.append((l, s, abc))
    lmax = max(w.orders)
    for t in range(len(centers)):
        dd = d[off[t]:off[t + 1]]
        r2 = (dd * dd).sum(1)
        ee = w.species[j[off[t]:off[t + 1]]]
        # per (sigma, primitive): K per pair and the |P| moments a_n per axis
        cache = {}
        for s in range(len(w.sigmas)):
            sig = w.sigmas[s]
            beta = 1 / (2 * sig * sig)
            for e in range(w.n_elements):
                m = ee == e
                for k in range(go[e], go[e + 1]):
                    a, c = w.gauss_exp[k], w.gauss_coef[k]
                    gm = a + beta
                    K = c * (2 * math.pi * sig * sig) ** -1.5 * (math.pi / gm) ** 1.5 * np.exp(-(a * beta / gm) * r2[m])
                    Pa = np.abs(dd[m]) * (a / gm)
                    mom = [np.ones_like(Pa), Pa]
                    for n in range(1, lmax):
                        mom.append(Pa * mom[n] + n * (0.5 / gm) * mom[n - 1])
                    cache[(s, k)] = (m, a / gm, K, mom)
        for col, (l, s, abc) in enumerate(cols):
            P = oracle_mod.mcsh_poly(*abc)
            S = sum(k * dd[:, 0] ** p * dd[:, 1] ** q * dd[:, 2] ** r for (p, q, r), k in P.items())
            R = np.zeros_like(r2)
            cscale = 0.0
            for e in range(w.n_elements):
                for k in range(go[e], go[e + 1]):
                    m, ratio, K, mom = cache[(s, k)]
                    R[m] += K * ratio ** l
                    summed = sum(abs(kk) * mom[p][:, 0] * mom[q][:, 1] * mom[r][:, 2] for (p, q, r), kk in P.items())
                    cscale += float(np.sum(np.abs(K) * summed))
            want = float(np.sum(R * S))
            scale = float(np.sum(np.abs(R * S)))
            assert abs(mu[t, col] - want) <= 1e-12 * scale + 2.0 ** -46 * cscale + 1e-300, (t, l, s, abc)


def test_density_order_matches_direct_sum(oracle_mod):
    w = synth.workload("random64_box").replace(orders=[-1, 0])
    f = oracle_mod.features(w, [3, 9])
    off, j, sh, d = oracle_mod.neighbors(w, [3, 9])
    go = w.gauss_off
    for t in range(2):
        dd = d[off[t]:off[t + 1]]
        r2 = (dd * dd).sum(1)
        rho = 0.0
        for jj, rr in zip(j[off[t]:off[t + 1]], r2):
            e = w.species[jj]
            rho += sum(w.gauss_coef[k] * math.exp(-w.gauss_exp[k] * rr) for k in range(go[e], go[e + 1]))
        assert abs(f[t, 0] - rho) <= 1e-13 * rho


# ------------------------------------------------------------ neighbors
def test_neighbors_match_brute_force(oracle_mod):
    w = synth.workload("random64_box")
    off, j, sh, d = oracle_mod.neighbors(w)
    got = set()
    for i in range(w.n_atoms):
        for t in range(off[i], off[i + 1]):
            got.add((i, int(j[t]), *map(int, sh[t])))
    A = w.cells[0]
    rc2 = w.cutoff * w.cutoff
    want = set()
    x = w.positions
    rng = range(-3, 4)  # cell 10 A, cutoff 6 A: |n| <= 2 suffices
    for n1 in rng:
        for n2 in rng:
            for n3 in rng:
                shift = (n1 * A[0] + n2 * A[1]) + n3 * A[2]
                D = (x[None, :, :] - x[:, None, :]) + shift
                r2 = (D[..., 0] * D[..., 0] + D[..., 1] * D[..., 1]) + D[..., 2] * D[..., 2]
                for i, jj in zip(*np.nonzero(r2 < rc2)):
                    want.add((int(i), int(jj), n1, n2, n3))
    assert got == want
    # ordering: (j, n) ascending within each center
    for i in range(w.n_atoms):
        keys = [(int(j[t]), *map(int, sh[t])) for t in range(off[i], off[i + 1])]
        assert keys == sorted(keys)


def test_neighbors_cluster_has_no_images(oracle_mod):
    w = synth.batched10k(n_struct=6)
    off, j, sh, d = oracle_mod.neighbors(w)
    for s in range(w.n_struct):
        a0, a1 = w.atom_off[s], w.atom_off[s + 1]
        for i in range(a0, a1):
            js = j[off[i]:off[i + 1]]
            assert np.all((js >= a0) & (js < a1))
            if not w.pbc[s].any():
                assert np.all(sh[off[i]:off[i + 1]] == 0)
                # a cluster: exactly the atoms within the cutoff, self included
                r = np.linalg.norm(w.positions[a0:a1] - w.positions[i], axis=1)
                assert len(js) == int(np.sum(r < w.cutoff))


# ------------------------------------------------------------ invariances
def _rel(a, b, floor):
    return np.max(np.abs(a - b) / np.maximum(np.abs(b), floor))


def test_rotation_translation_permutation_invariance(oracle_mod):
    w = synth.workload("random64_box").replace(orders=[-1, 0, 1, 2, 3, 4])
    f0, fa = oracle_mod.features(w, want_abs=True)
    floor = 1e-9 * fa
    rng = np.random.default_rng(7)
    Q, _ = np.linalg.qr(rng.normal(size=(3, 3)))
    if np.linalg.det(Q) < 0:
        Q[:, 0] = -Q[:, 0]
    wr = w.replace(positions=w.positions @ Q.T + np.array([0.3, -1.7, 2.2]), cells=w.cells @ Q.T)
    assert _rel(oracle_mod.features(wr), f0, floor) < 1e-10
    perm = rng.permutation(w.n_atoms)
    wp = w.replace(positions=w.positions[perm], species=w.species[perm])
    assert _rel(oracle_mod.features(wp), f0[perm], floor[perm]) < 1e-12
    # moving one atom by a lattice vector changes nothing
    pos = w.positions.copy()
    pos[11] += 2 * w.cells[0][0] - w.cells[0][2]
    assert _rel(oracle_mod.features(w.replace(positions=pos)), f0, floor) < 1e-12


def test_supercell_replication(oracle_mod):
    w = synth.workload("random64_box")
    A = w.cells[0]
    reps = [(a, b, c) for a in range(2) for b in range(2) for c in range(2)]
    pos = np.concatenate([w.positions + a * A[0] + b * A[1] + c * A[2] for a, b, c in reps])
    ws = w.replace(positions=pos, species=np.tile(w.species, 8), cells=(2 * A)[None],
                   atom_off=np.array([0, 8 * w.n_atoms]))
    f0, fa = oracle_mod.features(w, want_abs=True)
    centers = np.array([0, 64 + 3, 5 * 64 + 30, 7 * 64 + 63])
    fs = oracle_mod.features(ws, centers)
    assert _rel(fs, f0[centers % 64], 1e-12 * fa[centers % 64]) < 1e-11


# ------------------------------------------------------------ gradients
@pytest.mark.parametrize("orders", [[-1, 0, 1, 2], [-1, 3, 4, 5, 6]])
def test_jacobian_matches_central_differences(oracle_mod, orders):
    w = synth.workload("random64_box").replace(orders=orders)
    atoms = [2, 33]
    h = 1e-4
    centers = np.arange(w.n_atoms)
    joff, jj, jac = oracle_mod.jacobian_rows(w, centers)
    off, j, sh, d = oracle_mod.neighbors(w)
    r = np.linalg.norm(d, axis=1)
    for a in atoms:
        for ax in range(3):
            pp = w.positions.copy()
            pm = w.positions.copy()
            pp[a, ax] += h
            pm[a, ax] -= h
            fp = oracle_mod.features(w.replace(positions=pp), centers)
            fm = oracle_mod.features(w.replace(positions=pm), centers)
            fd = (fp - fm) / (2 * h)
            for i in centers:
                # skip centers with a pair involving atom a within 2h of the cutoff
                seg = slice(off[i], off[i + 1])
                near = np.abs(r[seg] - w.cutoff) < 4 * h
                if near.any() and (i == a or np.any(j[seg][near] == a)):
                    continue
                row = np.searchsorted(jj[joff[i]:joff[i + 1]], a)
                an = np.zeros(w.n_features)
                if row < joff[i + 1] - joff[i] and jj[joff[i] + row] == a:
                    an = jac[joff[i] + row, :, ax]
                scale = np.max(np.abs(jac[joff[i]:joff[i + 1]]), axis=(0, 2)) + 1e-30
                assert np.all(np.abs(fd[i] - an) <= 1e-6 * scale), (a, ax, i)


def test_jacobian_translation_sum_rule(oracle_mod):
    w = synth.workload("random64_box")
    joff, jj, jac = oracle_mod.jacobian_rows(w, np.arange(10))
    for t in range(10):
        blk = jac[joff[t]:joff[t + 1]]
        assert np.all(np.abs(blk.sum(0)) <= 1e-11 * np.abs(blk).sum(0).max())


# ------------------------------------------------------------ reference points
def test_point_features_match_3d_quadrature(oracle_mod):
    # probes centred on a point that is not an atom: each moment is the
    # defining overlap integral on a grid around the point, the feature the
    # weighted sum of squares l!/(a!b!c!) mu_abc^2 over all components
    pos = np.array([[0.0, 0.0, 0.0], [0.9, -0.6, 0.5], [-0.5, 0.8, -0.7]])
    coef, expo = [0.7, 0.4], [1.6, 0.6]
    sig = 0.55
    p = np.array([0.35, 0.2, -0.15])
    w = _cluster(pos, [0, 0, 0], [-1, 0, 1, 2, 3], [sig], coef, expo, [2])
    f = oracle_mod.point_features(w, p[None, :], [0])[0]
    h = 0.05
    g = np.arange(-5.0, 5.0 + h / 2, h)
    X, Y, Z = np.meshgrid(g, g, g, indexing="ij")
    beta = 1.0 / (2 * sig * sig)
    Ns = (2 * math.pi * sig * sig) ** -1.5
    rho = np.zeros_like(X)
    for q in pos - p:
        R2 = (X - q[0]) ** 2 + (Y - q[1]) ** 2 + (Z - q[2]) ** 2
        for c, a in zip(coef, expo):
            rho += c * np.exp(-a * R2)
    base = Ns * np.exp(-beta * (X * X + Y * Y + Z * Z)) * rho * h ** 3
    dens = sum(c * math.exp(-a * float(np.sum((q - p) ** 2))) for q in pos for c, a in zip(coef, expo))
    assert abs(f[0] - dens) <= 1e-13 * dens
    for col, l in enumerate([0, 1, 2, 3], start=1):
        want = scale = 0.0
        for (a, b, c) in oracle_mod.components(l):
            P = oracle_mod.mcsh_poly(a, b, c)
            S = sum(k * X ** pp * Y ** qq * Z ** ss for (pp, qq, ss), k in P.items())
            wt = math.factorial(l) / (math.factorial(a) * math.factorial(b) * math.factorial(c))
            mu = float(np.sum(S * base))
            mu_abs = float(np.sum(np.abs(S) * base))
            want += wt * mu * mu
            scale += wt * mu_abs * mu_abs
        assert abs(f[col] - want) <= 1e-8 * scale, (l, f[col], want)


def test_point_density_matches_brute_force_images(oracle_mod):
    # order -1 at points anywhere (inside, outside, far outside the cell):
    # the density of every atom image within the cutoff, images enumerated
    # by brute force
    w = synth.workload("random64_box").replace(orders=[-1])
    rng = np.random.default_rng(11)
    pts = rng.uniform(-12.0, 22.0, (24, 3))
    f = oracle_mod.point_features(w, pts, np.zeros(24, np.int32))[:, 0]
    A = w.cells[0]
    go = w.gauss_off
    rc2 = w.cutoff * w.cutoff
    for t, p in enumerate(pts):
        rho = 0.0
        for n1 in range(-4, 5):
            for n2 in range(-4, 5):
                for n3 in range(-4, 5):
                    shift = (n1 * A[0] + n2 * A[1]) + n3 * A[2]
                    D = (w.positions - p) + shift
                    r2 = (D[:, 0] * D[:, 0] + D[:, 1] * D[:, 1]) + D[:, 2] * D[:, 2]
                    for jj in np.nonzero(r2 < rc2)[0]:
                        e = w.species[jj]
                        rho += sum(w.gauss_coef[k] * math.exp(-w.gauss_exp[k] * r2[jj]) for k in range(go[e], go[e + 1]))
        assert abs(f[t] - rho) <= 1e-12 * abs(rho), (t, f[t], rho)


def test_point_features_special_points(oracle_mod):
    # a point on an atom has that atom's features; a point beyond the cutoff
    # of every atom of a cluster has zero features
    w = synth.batched10k(n_struct=6)
    atoms = np.array([0, int(w.atom_off[3]) + 1, int(w.atom_off[5])])
    ps = np.searchsorted(w.atom_off, atoms, side="right") - 1
    fa = oracle_mod.features(w, atoms)
    fp = oracle_mod.point_features(w, w.positions[atoms], ps)
    assert np.array_equal(fa, fp)
    cl = next(s for s in range(w.n_struct) if not w.pbc[s].any())
    far = w.positions[w.atom_off[cl]:w.atom_off[cl + 1]].max(0) + w.cutoff + 0.01
    assert np.all(oracle_mod.point_features(w, far[None, :], [cl]) == 0.0)


# ------------------------------------------------------------ strain derivative
def _strained_loss(oracle_mod, w, g, eps):
    M = np.eye(3) + eps
    w2 = w.replace(positions=w.positions @ M.T, cells=w.cells @ M.T)
    return float((oracle_mod.features(w2) * g).sum())


@pytest.mark.parametrize("kind", ["periodic", "periodic_high", "cluster", "triclinic"])
def test_virial_matches_strained_central_differences(oracle_mod, kind):
    # W_ab = dL/d eps_ab with positions and lattice vectors strained alike,
    # against central differences of the oracle's own features (h = 1e-5;
    # the neighbor lists at +-h are checked to be the same)
    if kind == "periodic":
        w = synth.workload("random64_box").replace(orders=[-1, 0, 1, 2])
    elif kind == "periodic_high":
        w = synth.workload("random64_box").replace(orders=[0, 4, 5, 6])
    elif kind == "cluster":
        b = synth.batched10k(n_struct=2)
        a0, a1 = int(b.atom_off[1]), int(b.atom_off[2])
        w = b.replace(positions=b.positions[a0:a1], species=b.species[a0:a1],
                      atom_off=np.array([0, a1 - a0], np.int64), cells=b.cells[1:2], pbc=b.pbc[1:2],
                      orders=[-1, 0, 1, 3], sigmas=[0.3, 0.8])
    else:
        rng = np.random.default_rng(4)
        tri = np.array([[7.0, 0.0, 0.0], [2.5, 6.5, 0.0], [1.0, 1.5, 8.0]])
        pos = rng.uniform(0, 1, (24, 3)) @ tri
        base = synth.workload("random64_box")
        w = base.replace(positions=pos, species=rng.integers(0, 2, 24).astype(np.int32),
                         atom_off=np.array([0, 24], np.int64), cells=tri[None], pbc=np.array([[1, 0, 1]], np.uint8),
                         orders=[0, 1, 2])
    g = synth.upstream_gradient(w.n_atoms, w.n_features, seed=12).astype(np.float64)
    W, Wa = oracle_mod.virial(w, g, want_abs=True)
    h = 1e-5
    n0 = oracle_mod.neighbors(w)[0]
    for a, b in [(0, 0), (1, 1), (2, 2), (0, 1), (2, 0), (1, 2)]:
        E = np.zeros((3, 3))
        E[a, b] = h
        for sgn in (1, -1):
            M = np.eye(3) + sgn * E
            w2 = w.replace(positions=w.positions @ M.T, cells=w.cells @ M.T)
            assert np.array_equal(oracle_mod.neighbors(w2)[0], n0)
        fd = (_strained_loss(oracle_mod, w, g, E) - _strained_loss(oracle_mod, w, g, -E)) / (2 * h)
        assert abs(fd - W[0, a, b]) <= 1e-8 * Wa[0].max(), (kind, a, b, fd, W[0, a, b])


def test_virial_is_symmetric(oracle_mod):
    # rotation invariance of the features: dL/d(theta) = 0 for every
    # infinitesimal rotation, i.e. W - W^T = 0, structure by structure
    w = synth.batched10k(n_struct=6)
    g = synth.upstream_gradient(w.n_atoms, w.n_features, seed=13).astype(np.float64)
    W, Wa = oracle_mod.virial(w, g, want_abs=True)
    for s in range(w.n_struct):
        assert np.abs(W[s] - W[s].T).max() <= 1e-12 * max(Wa[s].max(), 1e-300)


# ------------------------------------------------------------ tolerance scales
# Every parity floor is a fraction of a cancellation-free scale that the
# oracle computes beside its result: F_abs (features: the same reduction
# applied to sums of |per-pair contribution|) and jac_abs (derivatives: sum
# over pairs and components of 2 w_c A_c |d t_c / d d|, A_c = sum of |t_c|).
# An inflated scale would silently loosen every GPU test, so the scales are
# pinned here: they equal the value where nothing can cancel and bound it
# everywhere.
def _lone_pair_workload(orders, sigmas):
    # one element with three primitives; atom 1 is far beyond the cutoff of
    # every point used below, so a point near atom 0 has exactly one pair
    coef, expo = [0.6, 0.3, 0.2], [0.5, 1.1, 2.0]
    return _cluster([[0.0, 0.0, 0.0], [40.0, 0.0, 0.0]], [0, 0], orders, sigmas, coef, expo, [3], cutoff=6.0)


def test_single_pair_scale_equals_feature_and_closed_form(oracle_mod):
    # With one pair, F_abs = f exactly (|t|^2 = t^2), and by the sum rule
    # sum_c w_c S_c(d)^2 = l! (2l-1)!! |d|^(2l) each feature of order l is
    # f = R_{l,s}(r^2)^2 r^(2l) l! (2l-1)!!, R the Gaussian-product radial
    # factor (mean-value route), for every order 0..6.
    orders, sigmas = [-1, 0, 1, 2, 3, 4, 5, 6], [0.3, 0.7, 1.2]
    w = _lone_pair_workload(orders, sigmas)
    p = np.array([[0.8, -0.5, 0.9]])
    f, fa = oracle_mod.point_features(w, p, [0], want_abs=True)
    f, fa = f[0], fa[0]
    d = -p[0]
    r2 = float(d @ d)
    assert np.all(np.abs(f - fa) <= 1e-15 * fa)
    rho = sum(c * math.exp(-a * r2) for c, a in zip(w.gauss_coef, w.gauss_exp))
    assert abs(f[0] - rho) <= 1e-15 * rho
    col = 1
    for l in orders[1:]:
        dfact = math.prod(range(2 * l - 1, 0, -2)) if l > 0 else 1
        for sig in sigmas:
            beta = 1 / (2 * sig * sig)
            R = 0.0
            for c, a in zip(w.gauss_coef, w.gauss_exp):
                g = a + beta
                R += c * (2 * math.pi * sig * sig) ** -1.5 * (math.pi / g) ** 1.5 * (a / g) ** l * \
                    math.exp(-(a * beta / g) * r2)
            want = R * R * r2 ** l * math.factorial(l) * dfact
            assert abs(f[col] - want) <= 1e-12 * want, (l, sig, f[col], want)
            col += 1


def test_center_atom_adds_nothing_to_higher_orders(oracle_mod):
    # A lone atom (its only neighbor image is itself, at d = 0): a density
    # centred on the probe has zero overlap with every harmonic probe of
    # order l >= 1 (mean-value property: the Gaussian average of a harmonic
    # polynomial without constant term is its value at the centre, 0), so
    # those features are exactly 0; order 0 is R_0(0)^2 and the density its
    # own sum of coefficients.  Also a reference point placed exactly on an
    # atom whose neighbors all lie beyond the cutoff.
    orders, sigmas = [-1, 0, 1, 2, 3, 4, 5, 6], [0.1, 0.5, 1.2]
    w = _lone_pair_workload(orders, sigmas)
    f, fa = oracle_mod.features(w, [0], want_abs=True)
    fp = oracle_mod.point_features(w, np.array([[0.0, 0.0, 0.0]]), [0])
    for row in (f[0], fp[0]):
        assert row[0] == pytest.approx(sum(w.gauss_coef), rel=1e-15)
        for s, sig in enumerate(sigmas):
            beta = 1 / (2 * sig * sig)
            R0 = sum(c * (2 * math.pi * sig * sig) ** -1.5 * (math.pi / (a + beta)) ** 1.5
                     for c, a in zip(w.gauss_coef, w.gauss_exp))
            assert row[1 + s] == pytest.approx(R0 * R0, rel=1e-13)
        assert np.all(row[1 + len(sigmas):] == 0.0)
    assert np.all(fa[0, 1 + len(sigmas):] == 0.0)


def test_scales_bound_features_and_derivatives(oracle_mod):
    w = synth.workload("random64_box").replace(orders=[-1, 0, 1, 2, 3, 4, 5, 6])
    f, fa = oracle_mod.features(w, want_abs=True)
    assert np.all(f[:, 1:] >= 0.0) and np.all(f <= fa * (1 + 1e-13))
    # density coefficients are all positive: nothing cancels in order -1 and
    # order 0 (every per-pair term is positive), so there the scale is the value
    assert np.all(np.abs(f[:, :1 + len(w.sigmas)] - fa[:, :1 + len(w.sigmas)]) <= 1e-13 * fa[:, :1 + len(w.sigmas)])
    off, jj, jac, jab = oracle_mod.jacobian_rows(w, np.arange(w.n_atoms), want_abs=True)
    assert np.all(np.linalg.norm(jac, axis=-1) <= jab * (1 + 1e-12) + 1e-300)
    # the VJP scale bounds the VJP
    g = synth.upstream_gradient(w.n_atoms, w.n_features, seed=19).astype(np.float64)
    atoms = np.arange(0, w.n_atoms, 7)
    v, vs = oracle_mod.vjp_atoms(w, g, atoms, want_abs=True)
    assert np.all(np.linalg.norm(v, axis=1) <= vs * (1 + 1e-12))
    # mixed-sign density tables: the bounds still hold
    coef = np.array(w.gauss_coef)
    coef[1] *= -0.5
    coef[6] *= -0.3
    wm = w.replace(gauss_coef=coef)
    f, fa = oracle_mod.features(wm, want_abs=True)
    assert np.all(np.abs(f) <= fa * (1 + 1e-13))
    off, jj, jac, jab = oracle_mod.jacobian_rows(wm, np.arange(0, w.n_atoms, 5), want_abs=True)
    assert np.all(np.linalg.norm(jac, axis=-1) <= jab * (1 + 1e-12) + 1e-300)


def test_derivative_scale_equals_row_where_nothing_cancels(oracle_mod):
    # Two atoms: each center sees its own self pair (d = 0: the order -1 and
    # order 0 terms have zero gradient there) and the other atom.  For orders
    # -1 and 0 every term and moment is positive, so the row of the other
    # atom and the center's own row (minus it) have |J| = jac_abs exactly.
    w = _cluster([[0.0, 0.0, 0.0], [1.1, -0.7, 0.4]], [0, 0], [-1, 0], [0.3, 0.8], [0.6, 0.3], [0.5, 1.7], [2],
                 cutoff=6.0)
    off, jj, jac, jab = oracle_mod.jacobian_rows(w, np.arange(2), want_abs=True)
    assert np.array_equal(off, [0, 2, 4])
    assert np.all(np.abs(np.linalg.norm(jac, axis=-1) - jab) <= 1e-13 * jab)
