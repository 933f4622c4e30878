"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle on
the same seeded inputs.  Neighbor sets bit-exact; features within 1e-5 and
derivatives within 1e-4 relative (with the cancellation floors of
tests/parity.py)."""
import numpy as np
import pytest

from paper_2303_12980_gb300 import synth

from parity import (FEAT_TAU, FEAT_TOL, FP32_MIN_NORMAL, GRAD_TAU, GRAD_TOL, JAC_TAU, feature_errors,
                    grad_errors, record)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    import torch as t
    assert t.cuda.is_available(), "GPU tests need CUDA"
    from paper_2303_12980_gb300 import build
    build.build()
    return t


def _dev(torch, w):
    return (torch.from_numpy(w.positions).cuda(), torch.from_numpy(w.species).cuda())


def _featurizer(w):
    from paper_2303_12980_gb300.binding import GMPFeaturizer
    return GMPFeaturizer.from_workload(w)


WORKLOADS = {
    "random64_box": lambda: synth.workload("random64_box"),
    "fcc4096": lambda: synth.workload("fcc4096"),
    "batched300": lambda: synth.batched10k(n_struct=300),
    "slab_small": lambda: synth.fcc_slab262k(reps=(6, 6, 12)),
}
_cache = {}


def wl(name):
    if name not in _cache:
        _cache[name] = WORKLOADS[name]()
    return _cache[name]


def _neighbor_set(off, j, sh, centers=None):
    out = {}
    rng = range(len(off) - 1) if centers is None else centers
    for t, i in enumerate(rng):
        a, b = (off[i], off[i + 1]) if centers is None else (off[t], off[t + 1])
        out[int(i)] = [(int(j[k]), *map(int, sh[k])) for k in range(a, b)]
    return out


@pytest.mark.parametrize("name", ["random64_box", "fcc4096", "batched300", "slab_small"])
def test_neighbors_bit_exact(torch, oracle_mod, name):
    w = wl(name)
    pos, sp = _dev(torch, w)
    F = _featurizer(w)
    off, j, sh = F.neighbors(pos, sp, w.atom_off, w.cells, w.pbc)
    torch.cuda.synchronize()
    off, j, sh = off.cpu().numpy(), j.cpu().numpy(), sh.cpu().numpy()
    ooff, oj, osh, _ = oracle_mod.neighbors(w)
    assert np.array_equal(off, ooff)
    assert np.array_equal(j, oj)
    assert np.array_equal(sh, osh)
    record(f"neighbors/{name}", pairs=int(off[-1]))


@pytest.mark.parametrize("name", ["random64_box", "fcc4096", "batched300", "slab_small"])
def test_features_parity(torch, oracle_mod, name):
    w = wl(name)
    pos, sp = _dev(torch, w)
    F = _featurizer(w)
    f = F.featurize(pos, sp, w.atom_off, w.cells, w.pbc)
    torch.cuda.synchronize()
    f = f.cpu().numpy()
    ref, fabs = oracle_mod.features(w, want_abs=True)
    err = feature_errors(f, ref, fabs)
    raw = np.abs(f - ref) / np.maximum(np.abs(ref), 1e-300)
    record(f"features/{name}", max_rel_err=err.max(), per_column=err,
           unfloored_max=raw[ref > FEAT_TAU * fabs].max())
    assert err.max() <= FEAT_TOL, (err.max(), np.argmax(err))


def test_density_order_parity(torch, oracle_mod):
    w = wl("random64_box").replace(orders=[0, -1, 2], sigmas=[0.2, 0.5, 0.9])
    pos, sp = _dev(torch, w)
    f = _featurizer(w).featurize(pos, sp, w.atom_off, w.cells, w.pbc)
    torch.cuda.synchronize()
    ref, fabs = oracle_mod.features(w, want_abs=True)
    err = feature_errors(f.cpu().numpy(), ref, fabs)
    record("features/density_order", max_rel_err=err.max())
    assert err.max() <= FEAT_TOL


def test_many_sigmas_split_passes(torch, oracle_mod):
    w = wl("random64_box").replace(sigmas=list(np.geomspace(0.08, 1.6, 21)))
    pos, sp = _dev(torch, w)
    f = _featurizer(w).featurize(pos, sp, w.atom_off, w.cells, w.pbc)
    torch.cuda.synchronize()
    ref, fabs = oracle_mod.features(w, want_abs=True)
    err = feature_errors(f.cpu().numpy(), ref, fabs)
    assert err.max() <= FEAT_TOL


@pytest.mark.parametrize("name,n_atoms", [("random64_box", 64), ("fcc4096", 24), ("batched300", 24)])
def test_vjp_parity(torch, oracle_mod, name, n_atoms):
    w = wl(name)
    pos, sp = _dev(torch, w)
    F = _featurizer(w)
    g = synth.upstream_gradient(w.n_atoms, w.n_features, seed=77)
    feat, gp = F.featurize_vjp(pos, sp, w.atom_off, w.cells, w.pbc, torch.from_numpy(g).cuda())
    torch.cuda.synchronize()
    atoms = synth.subset_centers(w.n_atoms, n_atoms, seed=5)
    ref, scale = oracle_mod.vjp_atoms(w, g, atoms, want_abs=True)
    err = grad_errors(gp.cpu().numpy()[atoms], ref, scale)
    record(f"vjp/{name}", max_rel_err=err.max())
    assert err.max() <= GRAD_TOL, err.max()
    # the features returned alongside equal the forward call's
    f2 = F.featurize(pos, sp, w.atom_off, w.cells, w.pbc)
    torch.cuda.synchronize()
    assert torch.equal(feat, f2)


@pytest.mark.parametrize("name,n_centers", [("random64_box", 64), ("fcc4096", 128)])
def test_jacobian_parity(torch, oracle_mod, name, n_centers):
    w = wl(name)
    pos, sp = _dev(torch, w)
    F = _featurizer(w)
    feat, joff, jj, jac = F.featurize_grad(pos, sp, w.atom_off, w.cells, w.pbc)
    torch.cuda.synchronize()
    joff, jj, jac = joff.cpu().numpy(), jj.cpu().numpy(), jac.cpu().numpy()
    centers = synth.subset_centers(w.n_atoms, n_centers, seed=9)
    ooff, oj, ojac, oabs = oracle_mod.jacobian_rows(w, centers, want_abs=True)
    worst = 0.0
    for t, i in enumerate(centers):
        a, b = joff[i], joff[i + 1]
        assert np.array_equal(jj[a:b], oj[ooff[t]:ooff[t + 1]])
        err = grad_errors(jac[a:b], ojac[ooff[t]:ooff[t + 1]], oabs[ooff[t]:ooff[t + 1]], tau=JAC_TAU)
        worst = max(worst, float(err.max()))
    record(f"jacobian/{name}", max_rel_err=worst, nnz=int(joff[-1]))
    assert worst <= GRAD_TOL, worst


def test_jacobian_central_differences(torch, oracle_mod):
    """The GPU Jacobian (featurize_grad) and VJP, and the oracle's analytic
    Jacobian, against central differences of the FP64 oracle features,
    h = 1e-4 A, on fcc4096: (a) a fixed subset of 128 atoms one at a time,
    each moved along its own random direction, every feature of every
    center that sees it; (b) the whole structure along one random
    displacement field, contracted with random feature weights.  Atoms
    with an image pair near the cutoff stay fixed (the features are
    discontinuous there)."""
    w = wl("fcc4096")
    h = 1e-4
    pos, sp = _dev(torch, w)
    F = _featurizer(w)
    feat, joff, jj, jac = F.featurize_grad(pos, sp, w.atom_off, w.cells, w.pbc)
    torch.cuda.synchronize()
    joff, jj, jac = joff.cpu().numpy(), jj.cpu().numpy(), jac.cpu().numpy().astype(np.float64)
    rng = np.random.default_rng(123)
    # The features jump where a pair crosses the hard cutoff, so only atoms
    # with no image pair within 2e-3 A of rc (on either side) are moved; the
    # steps below move any pair distance by less than 1e-3 A.
    noff_all, nj_all, _, nd_all = oracle_mod.neighbors(w.replace(cutoff=w.cutoff + 2e-3))
    near = np.abs(np.linalg.norm(nd_all, axis=1) - w.cutoff) < 2e-3
    center_of = np.repeat(np.arange(w.n_atoms), np.diff(noff_all))
    movable = np.ones(w.n_atoms, bool)
    movable[center_of[near]] = False
    movable[nj_all[near]] = False
    free = np.flatnonzero(movable)
    assert free.size > w.n_atoms // 2
    worst = worst_oracle = 0.0
    # the oracle's analytic rows of every center, once
    ooff, oj, ojac, oabs = oracle_mod.jacobian_rows(w, np.arange(w.n_atoms), want_abs=True)
    for a in free[synth.subset_centers(free.size, 128, seed=41)]:
        u = rng.normal(size=3)
        u /= np.linalg.norm(u)
        noff, nj, _, _ = oracle_mod.neighbors(w, np.array([a]))
        centers = np.unique(np.concatenate([nj[noff[0]:noff[1]], [a]])).astype(np.int64)
        fd = []
        for sgn in (1.0, -1.0):
            x = w.positions.copy()
            x[a] += sgn * h * u
            fd.append(oracle_mod.features(w.replace(positions=x), centers))
        fd = (fd[0] - fd[1]) / (2.0 * h)                       # [nc, F]
        # denominators as in grad_errors: the derivative vector's length
        # (from the oracle's analytic row), floored at JAC_TAU x its
        # cancellation-free scale and at the smallest normal FP32 number
        gpu = np.zeros_like(fd)
        ana = np.zeros_like(fd)
        den = np.zeros_like(fd)
        for t, i in enumerate(centers):
            k = joff[i] + np.searchsorted(jj[joff[i]:joff[i + 1]], a)
            assert jj[k] == a
            gpu[t] = jac[k] @ u
            ko = ooff[i] + np.searchsorted(oj[ooff[i]:ooff[i + 1]], a)
            assert oj[ko] == a
            ana[t] = ojac[ko] @ u
            den[t] = np.maximum(np.maximum(np.linalg.norm(ojac[ko], axis=-1), JAC_TAU * oabs[ko]), FP32_MIN_NORMAL)
        worst = max(worst, float((np.abs(gpu - fd) / den).max()))
        # the oracle's analytic derivative against the same differences
        # (their O(h^2) truncation reaches ~2e-5 of the floored scale here)
        worst_oracle = max(worst_oracle, float((np.abs(ana - fd) / den).max()))
    # (b) one displacement field over all atoms, weights g: d/de sum g . f(x + e delta)
    delta = np.clip(rng.normal(size=w.positions.shape), -2.5, 2.5) * movable[:, None]
    g = synth.upstream_gradient(w.n_atoms, w.n_features, seed=5)
    sums = []
    for sgn in (1.0, -1.0):
        sums.append(float(np.sum(g * oracle_mod.features(w.replace(positions=w.positions + sgn * h * delta)))))
    fd_all = (sums[0] - sums[1]) / (2.0 * h)
    _, gp = F.featurize_vjp(pos, sp, w.atom_off, w.cells, w.pbc, torch.from_numpy(g).cuda())
    torch.cuda.synchronize()
    vjp_dir = float(np.sum(gp.cpu().numpy().astype(np.float64) * delta))
    rows_i = np.repeat(np.arange(w.n_atoms), np.diff(joff))
    jd = np.einsum("rfc,rc->rf", jac, delta[jj])                 # per row: J delta_j
    jac_dir = float(np.sum(g[rows_i] * jd))
    scale_all = float(np.sum(np.abs(g[rows_i] * jd)))
    err_all = max(abs(vjp_dir - fd_all), abs(jac_dir - fd_all)) / max(abs(fd_all), 1e-3 * scale_all)
    record("jacobian/central_differences", per_atom_max_rel_err=worst, oracle_per_atom_max_rel_err=worst_oracle,
           field_rel_err=err_all, atoms=128)
    assert worst <= GRAD_TOL, worst
    assert worst_oracle <= GRAD_TOL, worst_oracle
    assert err_all <= GRAD_TOL, err_all


def test_autograd_function_matches_vjp(torch):
    from paper_2303_12980_gb300.binding import gmp_features
    w = wl("random64_box")
    pos, sp = _dev(torch, w)
    F = _featurizer(w)
    p = pos.clone().requires_grad_(True)
    f = gmp_features(p, F, sp, w.atom_off, w.cells, w.pbc)
    g = torch.from_numpy(synth.upstream_gradient(w.n_atoms, w.n_features, seed=3)).cuda()
    (f * g).sum().backward()
    _, gp = F.featurize_vjp(pos, sp, w.atom_off, w.cells, w.pbc, g)
    torch.cuda.synchronize()
    assert torch.allclose(p.grad.float(), gp, rtol=0, atol=0)


def test_host_buffers_match_device(torch):
    w = wl("random64_box")
    pos, sp = _dev(torch, w)
    F = _featurizer(w)
    fd = F.featurize(pos, sp, w.atom_off, w.cells, w.pbc)
    torch.cuda.synchronize()
    fh = F.featurize(w.positions, w.species, w.atom_off, w.cells, w.pbc)
    assert np.array_equal(fd.cpu().numpy(), np.asarray(fh))
    # the VJP from host buffers (copies overlapped with the kernels on a
    # side stream) equals the device-buffer call
    for name in ("random64_box", "batched300"):
        w = wl(name)
        pos, sp = _dev(torch, w)
        F = _featurizer(w)
        g = synth.upstream_gradient(w.n_atoms, w.n_features, seed=33)
        fdv, gdv = F.featurize_vjp(pos, sp, w.atom_off, w.cells, w.pbc, torch.from_numpy(g).cuda())
        torch.cuda.synchronize()
        for _ in range(2):
            fhv, ghv = F.featurize_vjp(w.positions, w.species, w.atom_off, w.cells, w.pbc, g)
            assert np.array_equal(fdv.cpu().numpy(), np.asarray(fhv)), name
            assert np.array_equal(gdv.cpu().numpy(), np.asarray(ghv)), name


def test_deterministic(torch):
    w = wl("fcc4096")
    pos, sp = _dev(torch, w)
    F = _featurizer(w)
    a = F.featurize(pos, sp, w.atom_off, w.cells, w.pbc)
    b = F.featurize(pos, sp, w.atom_off, w.cells, w.pbc)
    torch.cuda.synchronize()
    assert torch.equal(a, b)


@pytest.mark.parametrize("name", ["fcc4096", "batched300"])
def test_vjp_bitwise_reproducible(torch, name):
    """The VJP has no float atomics: each pair's gradient is added exactly,
    as an integer, into fixed-point bins of its atom, which are combined in
    a fixed order afterwards, so the sum does not depend on the order the
    pairs are processed in.  Repeated calls and other CTA sizes give the
    same gradient bit for bit, for the split forward/backward kernels and
    for the fused kernel (which differs from the split pair: it does not
    refine ill-conditioned moments before the backward sweep)."""
    w = wl(name)
    pos, sp = _dev(torch, w)
    F = _featurizer(w)
    g = torch.from_numpy(synth.upstream_gradient(w.n_atoms, w.n_features, seed=15)).cuda()
    base = F.tuning()
    ref = {}
    for k, (bwd_warps, fused, fused_warps) in enumerate([(4, 0, 4), (12, 0, 8), (6, 1, 4), (0, 1, 8)]):
        vals = list(base)
        for p in range(len(vals) // 6):
            vals[6 * p + 2], vals[6 * p + 3], vals[6 * p + 4] = bwd_warps, fused, fused_warps
        F.set_tuning(vals)
        for _ in range(2):
            f1, g1 = F.featurize_vjp(pos, sp, w.atom_off, w.cells, w.pbc, g)
            torch.cuda.synchronize()
            if fused not in ref:
                ref[fused] = (f1.clone(), g1.clone())
            assert torch.equal(f1, ref[fused][0]), k
            assert torch.equal(g1, ref[fused][1]), k


@pytest.mark.parametrize("name", ["fcc4096", "batched300", "random64_box"])
def test_fused_vjp_parity(torch, oracle_mod, name):
    """The fused forward+backward kernel (an autotuner choice) against the
    oracle: its adjoints come from the FP32 moments, not the refined ones,
    so its gradient is checked on its own, on sampled atoms of a jittered
    crystal (many refined features), a batch and a random box."""
    w = wl(name)
    pos, sp = _dev(torch, w)
    F = _featurizer(w)
    vals = list(F.tuning())
    for p in range(len(vals) // 6):
        vals[6 * p + 3], vals[6 * p + 4] = 1, 4
    F.set_tuning(vals)
    g = synth.upstream_gradient(w.n_atoms, w.n_features, seed=23)
    feat, gp = F.featurize_vjp(pos, sp, w.atom_off, w.cells, w.pbc, torch.from_numpy(g).cuda())
    torch.cuda.synchronize()
    ref, fabs = oracle_mod.features(w, want_abs=True)
    ferr = feature_errors(feat.cpu().numpy(), ref, fabs)
    atoms = synth.subset_centers(w.n_atoms, 64, seed=6)
    gref, gscale = oracle_mod.vjp_atoms(w, g, atoms, want_abs=True)
    gerr = grad_errors(gp.cpu().numpy()[atoms], gref, gscale)
    record(f"vjp_fused/{name}", features_max_rel_err=ferr.max(), vjp_max_rel_err=gerr.max())
    assert ferr.max() <= FEAT_TOL, ferr.max()
    assert gerr.max() <= GRAD_TOL, gerr.max()


def test_graph_replay_matches_eager(torch):
    """Graph mode: replays on the same buffers give the eager results, follow
    in-place position updates, and fall back eagerly when the batch outgrows
    the captured neighbor capacity."""
    w = wl("batched300")
    F_eager = _featurizer(w)
    F_graph = _featurizer(w)
    F_graph.set_graph(True)
    s = torch.cuda.Stream()
    pos, sp = _dev(torch, w)
    g = torch.from_numpy(synth.upstream_gradient(w.n_atoms, w.n_features, seed=4)).cuda()
    feat = torch.empty((w.n_atoms, w.n_features), device="cuda")
    gp = torch.empty((w.n_atoms, 3), device="cuda")
    with torch.cuda.stream(s):
        for step in range(4):
            if step == 2:   # small in-place move: same buffers, graph replay
                pos += 0.01 * torch.randn_like(pos)
            if step == 3:   # compress the clusters (cells unchanged): more neighbors than captured
                pos *= 0.8
            F_graph.featurize_vjp(pos, sp, w.atom_off, w.cells, w.pbc, g, out=(feat, gp))
            fe, ge = F_eager.featurize_vjp(pos, sp, w.atom_off, w.cells, w.pbc, g)
            s.synchronize()
            assert torch.equal(feat, fe), step
            assert torch.equal(gp, ge), step


def _cutoff_by_grid(w, t):
    """Largest r on a 1e-4 A grid where some single-primitive bound exceeds
    the overlap threshold t (direct evaluation; compare gmp_cutoff)."""
    import math
    r = np.arange(1e-4, 80.0, 1e-4)
    best = 0.0
    go = w.gauss_off
    for e in range(w.n_elements):
        for k in range(go[e], go[e + 1]):
            a, c = w.gauss_exp[k], abs(w.gauss_coef[k])
            for l in w.orders:
                if l < 0:
                    val = c * np.exp(-a * r * r)
                    idx = np.nonzero(val > t)[0]
                    best = max(best, r[idx[-1]] if idx.size else 0.0)
                    continue
                lf = math.factorial(l)
                df = math.prod(range(2 * l - 1, 0, -2)) if l > 0 else 1
                for s in w.sigmas:
                    beta = 1 / (2 * s * s)
                    g = a + beta
                    amp = c * (2 * math.pi * s * s) ** -1.5 * (math.pi / g) ** 1.5 * (a / g) ** l * math.sqrt(lf * df)
                    val = amp * r ** l * np.exp(-(a * beta / g) * r * r)
                    idx = np.nonzero(val > t)[0]
                    best = max(best, r[idx[-1]] if idx.size else 0.0)
    return best


def test_cutoff_from_overlap_threshold(torch, oracle_mod):
    from paper_2303_12980_gb300.binding import GMPFeaturizer
    w = wl("random64_box").replace(orders=[-1, 0, 1, 2])
    for t in (1e-8, 1e-12):
        F = GMPFeaturizer(w.orders, w.sigmas, 0.0, w.n_gauss, w.gauss_coef, w.gauss_exp, overlap_threshold=t)
        ref = _cutoff_by_grid(w, t)
        assert abs(F.cutoff - ref) <= 2e-4, (t, F.cutoff, ref)
    wc = w.replace(cutoff=F.cutoff)
    pos, sp = _dev(torch, wc)
    f = F.featurize(pos, sp, wc.atom_off, wc.cells, wc.pbc)
    torch.cuda.synchronize()
    fref, fabs = oracle_mod.features(wc, want_abs=True)
    assert feature_errors(f.cpu().numpy(), fref, fabs).max() <= FEAT_TOL


def _points_for(w, n_per, seed):
    """Reference points per structure: on atoms, uniform in (and around) the
    cell or the cluster's box, and a few far away."""
    rng = np.random.default_rng(seed)
    pts, off = [], [0]
    for s in range(w.n_struct):
        a0, a1 = int(w.atom_off[s]), int(w.atom_off[s + 1])
        k = n_per if s % 7 != 3 else 0          # some structures own no points
        if k:
            if w.pbc[s].any():
                lo, hi = np.zeros(3), np.ones(3)
                P = rng.uniform(-0.6, 1.6, (k, 3)) @ w.cells[s]
            else:
                X = w.positions[a0:a1] if a1 > a0 else np.zeros((1, 3))
                lo, hi = X.min(0) - 3.0, X.max(0) + 3.0
                P = rng.uniform(lo, hi, (k, 3))
            if a1 > a0:
                P[0] = w.positions[rng.integers(a0, a1)]
            P[-1] = P[-1] + 1e3 * (s % 2)            # far outside the structure
            pts.append(P)
        off.append(off[-1] + k)
    return np.concatenate(pts), np.array(off, np.int64)


@pytest.mark.parametrize("name,n_per", [("random64_box", 40), ("batched300", 5), ("slab_small", 64)])
def test_point_features_parity(torch, oracle_mod, name, n_per):
    w = wl(name)
    pts, poff = _points_for(w, n_per, seed=17)
    pos, sp = _dev(torch, w)
    F = _featurizer(w)
    f = F.featurize_points(pos, sp, w.atom_off, w.cells, w.pbc, torch.from_numpy(pts).cuda(), poff)
    torch.cuda.synchronize()
    pstruct = np.repeat(np.arange(w.n_struct), np.diff(poff))
    ref, fabs = oracle_mod.point_features(w, pts, pstruct, want_abs=True)
    err = feature_errors(f.cpu().numpy(), ref, fabs)
    record(f"points/{name}", max_rel_err=err.max(), points=len(pts))
    assert err.max() <= FEAT_TOL, (err.max(), np.argmax(err))
    # a point on an atom reproduces that atom's features bit for bit (same
    # neighbor enumeration, same kernels)
    fa = F.featurize(pos, sp, w.atom_off, w.cells, w.pbc).cpu().numpy()
    fp = f.cpu().numpy()
    for s in range(w.n_struct):
        if poff[s + 1] > poff[s] and w.atom_off[s + 1] > w.atom_off[s]:
            a = np.nonzero((w.positions == pts[poff[s]]).all(1))[0][0]
            assert np.array_equal(fp[poff[s]], fa[a]), (s, a)
    # host buffers give the same result
    fh = F.featurize_points(w.positions, w.species, w.atom_off, w.cells, w.pbc, pts, poff)
    assert np.array_equal(np.asarray(fh), fp)


def test_mixed_sign_density_tables(torch, oracle_mod):
    """Density coefficients of both signs (radial factors may be negative):
    features, refinement flags and the VJP against the oracle."""
    w = wl("random64_box")
    coef = np.array(w.gauss_coef, np.float64)
    coef[1] *= -0.5
    coef[6] *= -0.3
    w = w.replace(gauss_coef=coef, orders=[-1, 0, 1, 2])
    pos, sp = _dev(torch, w)
    F = _featurizer(w)
    g = synth.upstream_gradient(w.n_atoms, w.n_features, seed=8)
    feat, gp = F.featurize_vjp(pos, sp, w.atom_off, w.cells, w.pbc, torch.from_numpy(g).cuda())
    torch.cuda.synchronize()
    ref, fabs = oracle_mod.features(w, want_abs=True)
    ferr = feature_errors(feat.cpu().numpy(), ref, fabs)
    atoms = synth.subset_centers(w.n_atoms, 16, seed=3)
    gref, gscale = oracle_mod.vjp_atoms(w, g, atoms, want_abs=True)
    gerr = grad_errors(gp.cpu().numpy()[atoms], gref, gscale)
    record("mixed_sign/random64_box", features_max_rel_err=ferr.max(), vjp_max_rel_err=gerr.max())
    assert ferr.max() <= FEAT_TOL, ferr.max()
    assert gerr.max() <= GRAD_TOL, gerr.max()


@pytest.mark.parametrize("name", ["random64_box", "batched300", "fcc4096"])
def test_virial_parity(torch, oracle_mod, name):
    """Per-structure strain derivative against the oracle; the gradient and
    features of the same call equal gmp_featurize_vjp's."""
    w = wl(name)
    pos, sp = _dev(torch, w)
    F = _featurizer(w)
    g = synth.upstream_gradient(w.n_atoms, w.n_features, seed=21)
    gd = torch.from_numpy(g).cuda()
    feat, gp, vir = F.featurize_vjp_virial(pos, sp, w.atom_off, w.cells, w.pbc, gd)
    f2, gp2 = F.featurize_vjp(pos, sp, w.atom_off, w.cells, w.pbc, gd)
    torch.cuda.synchronize()
    assert torch.equal(feat, f2)
    assert torch.equal(gp, gp2)
    W, Wa = oracle_mod.virial(w, g.astype(np.float64), want_abs=True)
    V = vir.cpu().numpy()
    err = np.abs(V - W) / np.maximum(np.maximum(np.abs(W), GRAD_TAU * Wa), 2.0 ** -126)
    record(f"virial/{name}", max_rel_err=err.max(), structures=w.n_struct)
    assert err.max() <= GRAD_TOL, err.max()
    # host buffers, and a second call, give the same result bit for bit
    _, _, vh = F.featurize_vjp_virial(w.positions, w.species, w.atom_off, w.cells, w.pbc, g)
    assert np.array_equal(np.asarray(vh), V)
    _, gp3, vir3 = F.featurize_vjp_virial(pos, sp, w.atom_off, w.cells, w.pbc, gd)
    torch.cuda.synchronize()
    assert torch.equal(gp3, gp) and torch.equal(vir3, vir)


def test_repeated_calls_single_pass_neighbors(torch):
    """A repeated batch builds its neighbor records in one pass with the last
    call's capacities; a batch that outgrows them falls back to counting.
    Every call equals a fresh handle's first (two-pass) call bit for bit."""
    w = wl("fcc4096")
    F = _featurizer(w)
    pos, sp = _dev(torch, w)
    g = torch.from_numpy(synth.upstream_gradient(w.n_atoms, w.n_features, seed=6)).cuda()
    # the cell stays fixed (same batch description); positions: same, same,
    # slightly compressed, much compressed (more pairs than the last call's
    # capacity), back to the start
    moves = [1.0, 1.0, 0.98, 0.8, 1.0]
    for k, scale in enumerate(moves):
        p = (pos * scale).contiguous()
        f1, g1 = F.featurize_vjp(p, sp, w.atom_off, w.cells, w.pbc, g)
        f0, g0 = _featurizer(w).featurize_vjp(p, sp, w.atom_off, w.cells, w.pbc, g)
        torch.cuda.synchronize()
        assert torch.equal(f1, f0), k
        assert torch.equal(g1, g0), k


def test_small_batch_binning_matches_multi_kernel_binning(torch):
    """A batch of at most 1024 atoms is binned by one single-CTA kernel, a
    larger one by the multi-kernel path.  Both put each bin's atoms in index
    order, so a 512-atom crystal's features come out bit-identical alone and
    as each structure of a batch of three jittered copies (1536 atoms)."""
    w = wl("fcc4096")  # its probe set and element table
    F = _featurizer(w)
    rng = np.random.default_rng(23)
    pos0, cell = synth.fcc_supercell(rng, 3.6, (4, 4, 8), 0.1)
    n = pos0.shape[0]
    sp = rng.integers(0, 3, n).astype(np.int32)
    P = [pos0] + [pos0 + rng.normal(0.0, 0.05, pos0.shape) for _ in range(2)]
    off1 = np.array([0, n], np.int64)
    pbc1 = np.ones((1, 3), np.uint8)
    sp_d = torch.from_numpy(sp).cuda()
    f_big = F.featurize(torch.from_numpy(np.concatenate(P)).cuda(), torch.from_numpy(np.concatenate([sp] * 3)).cuda(),
                        np.arange(4, dtype=np.int64) * n, np.stack([cell] * 3), np.ones((3, 3), np.uint8))
    for k, p in enumerate(P):
        f_one = F.featurize(torch.from_numpy(p).cuda(), sp_d, off1, cell[None], pbc1)
        torch.cuda.synchronize()
        assert torch.equal(f_one, f_big[k * n:(k + 1) * n]), k


def test_jacobian_center_chunks(torch):
    """gmp_featurize_grad_centers: the Jacobian taken in center chunks (one
    of them empty; one with host buffers) equals the whole-batch call row
    for row, bit for bit."""
    w = wl("fcc4096")
    F = _featurizer(w)
    pos, sp = _dev(torch, w)
    feat, joff, jj, jac = F.featurize_grad(pos, sp, w.atom_off, w.cells, w.pbc)
    torch.cuda.synchronize()
    for b, e in [(0, 1000), (1000, 1000), (1000, 2731), (2731, 4096)]:
        f2, jo2, jj2, jac2 = F.featurize_grad(pos, sp, w.atom_off, w.cells, w.pbc, centers=(b, e))
        torch.cuda.synchronize()
        r0, r1 = int(joff[b]), int(joff[e])
        assert torch.equal(f2, feat[b:e]), (b, e)
        assert torch.equal(jo2, joff[b:e + 1] - r0), (b, e)
        assert torch.equal(jj2, jj[r0:r1]) and torch.equal(jac2, jac[r0:r1]), (b, e)
    fh, joh, jjh, jach = F.featurize_grad(w.positions, w.species, w.atom_off, w.cells, w.pbc, centers=(1000, 2731))
    r0, r1 = int(joff[1000]), int(joff[2731])
    assert torch.equal(fh, feat[1000:2731].cpu()) and torch.equal(joh, (joff[1000:2732] - r0).cpu())
    assert torch.equal(jjh, jj[r0:r1].cpu()) and torch.equal(jach, jac[r0:r1].cpu())
    with pytest.raises(ValueError):
        F.featurize_grad(pos, sp, w.atom_off, w.cells, w.pbc, centers=(10, 5))


def test_jacobian_capacity_contract(torch):
    """gmp_featurize_grad through the C ABI with a row buffer that is too
    short: status GMP_ERR_CAPACITY, *nnz_out = the rows needed, and no
    output buffer touched; the binding's call then returns exactly that
    many rows."""
    import ctypes as C
    w = wl("random64_box")
    F = _featurizer(w)
    pos, sp = _dev(torch, w)
    off, cell, pbc = F._struct(w.atom_off, w.cells, w.pbc)
    N, nf = w.n_atoms, F.num_features
    feat = torch.full((N, nf), -7.0, device="cuda")
    joff = torch.full((N + 1,), -5, dtype=torch.int64, device="cuda")
    jj = torch.full((8,), -3, dtype=torch.int32, device="cuda")
    jac = torch.full((8, nf, 3), -9.0, device="cuda")
    nnz = C.c_int64(-1)
    st = F._L.gmp_featurize_grad(F._h, 1, off.ctypes.data, pos.data_ptr(), cell.ctypes.data, pbc.ctypes.data,
                                 sp.data_ptr(), feat.data_ptr(), joff.data_ptr(), jj.data_ptr(), jac.data_ptr(), 8,
                                 C.byref(nnz), torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    assert st == 4 and nnz.value > 8, (st, nnz.value)
    assert (feat == -7.0).all() and (joff == -5).all() and (jj == -3).all() and (jac == -9.0).all()
    f2, joff2, jj2, jac2 = F.featurize_grad(pos, sp, w.atom_off, w.cells, w.pbc)
    torch.cuda.synchronize()
    assert int(joff2[-1]) == nnz.value == jj2.shape[0] == jac2.shape[0]


def test_repeated_jacobian_calls_single_pass_neighbors(torch):
    """Repeated featurize_grad calls build their atom-sorted neighbor records
    in one pass (blocks per center in allocation order) and reuse the last
    call's row capacity; each call equals a fresh handle's first call bit for
    bit, and the CSR neighbor lists of gmp_neighbors are unaffected."""
    w = wl("fcc4096")
    F = _featurizer(w)
    pos, sp = _dev(torch, w)
    for k, scale in enumerate([1.0, 1.0, 0.98, 0.8, 1.0]):
        p = (pos * scale).contiguous()
        a = F.featurize_grad(p, sp, w.atom_off, w.cells, w.pbc)
        b = _featurizer(w).featurize_grad(p, sp, w.atom_off, w.cells, w.pbc)
        torch.cuda.synchronize()
        for x, y in zip(a, b):
            assert x.shape == y.shape and torch.equal(x, y), k
        n1 = F.neighbors(p, sp, w.atom_off, w.cells, w.pbc)
        n0 = _featurizer(w).neighbors(p, sp, w.atom_off, w.cells, w.pbc)
        torch.cuda.synchronize()
        for x, y in zip(n1, n0):
            assert torch.equal(x, y), k


@pytest.mark.parametrize("orders,n_sig", [([0, 1, 2, 3], 21), ([-1], 1), ([0], 3), ([-1, 5], 2), ([6, 1, -1], 17)])
def test_vjp_probe_sets(torch, oracle_mod, orders, n_sig):
    """Probe sets beyond the workloads': more than 16 sigmas (several kernel
    passes sharing the moment buffer), density only, one order, unordered
    orders with the density in the middle of the column list."""
    w = wl("random64_box").replace(orders=orders, sigmas=list(np.geomspace(0.1, 1.4, n_sig)))
    pos, sp = _dev(torch, w)
    F = _featurizer(w)
    g = synth.upstream_gradient(w.n_atoms, w.n_features, seed=41)
    feat, gp = F.featurize_vjp(pos, sp, w.atom_off, w.cells, w.pbc, torch.from_numpy(g).cuda())
    torch.cuda.synchronize()
    ref, fabs = oracle_mod.features(w, want_abs=True)
    assert feature_errors(feat.cpu().numpy(), ref, fabs).max() <= FEAT_TOL
    atoms = synth.subset_centers(w.n_atoms, 16, seed=2)
    gref, gscale = oracle_mod.vjp_atoms(w, g, atoms, want_abs=True)
    assert grad_errors(gp.cpu().numpy()[atoms], gref, gscale).max() <= GRAD_TOL
    # the Jacobian rows and the strain derivative of the same probe set
    # (one forward, refinement and derivative kernel per 16-sigma pass)
    feat2, joff, jj, jac = F.featurize_grad(pos, sp, w.atom_off, w.cells, w.pbc)
    _, _, vir = F.featurize_vjp_virial(pos, sp, w.atom_off, w.cells, w.pbc, torch.from_numpy(g).cuda())
    torch.cuda.synchronize()
    assert feature_errors(feat2.cpu().numpy(), ref, fabs).max() <= FEAT_TOL
    joff, jj, jac = joff.cpu().numpy(), jj.cpu().numpy(), jac.cpu().numpy()
    centers = synth.subset_centers(w.n_atoms, 16, seed=3)
    ooff, oj, ojac, oabs = oracle_mod.jacobian_rows(w, centers, want_abs=True)
    for t, i in enumerate(centers):
        a, b = joff[i], joff[i + 1]
        assert np.array_equal(jj[a:b], oj[ooff[t]:ooff[t + 1]])
        err = grad_errors(jac[a:b], ojac[ooff[t]:ooff[t + 1]], oabs[ooff[t]:ooff[t + 1]], tau=JAC_TAU)
        assert err.max() <= GRAD_TOL, err.max()
    W, Wa = oracle_mod.virial(w, g.astype(np.float64), want_abs=True)
    verr = np.abs(vir.cpu().numpy() - W) / np.maximum(np.maximum(np.abs(W), GRAD_TAU * Wa), 2.0 ** -126)
    assert verr.max() <= GRAD_TOL, verr.max()


def test_jacobian_batched_clusters_and_cells(torch, oracle_mod):
    """Every Jacobian row of the first 4096 atoms of a batch mixing clusters
    and periodic cells."""
    w = wl("batched300")
    pos, sp = _dev(torch, w)
    F = _featurizer(w)
    feat, joff, jj, jac = F.featurize_grad(pos, sp, w.atom_off, w.cells, w.pbc)
    torch.cuda.synchronize()
    joff, jj, jac = joff.cpu().numpy(), jj.cpu().numpy(), jac.cpu().numpy()
    centers = np.arange(min(w.n_atoms, 4096))
    ooff, oj, ojac, oabs = oracle_mod.jacobian_rows(w, centers, want_abs=True)
    worst = 0.0
    for t, i in enumerate(centers):
        a, b = joff[i], joff[i + 1]
        assert np.array_equal(jj[a:b], oj[ooff[t]:ooff[t + 1]])
        worst = max(worst, float(grad_errors(jac[a:b], ojac[ooff[t]:ooff[t + 1]], oabs[ooff[t]:ooff[t + 1]],
                                             tau=JAC_TAU).max()))
    record("jacobian/batched300", max_rel_err=worst)
    assert worst <= GRAD_TOL, worst
