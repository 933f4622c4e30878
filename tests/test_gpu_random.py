"""Seeded random batches against the FP64 oracle: small structures with
triclinic cells (shear up to 0.3 of a cell length), every mix of periodic
and open axes, 4-48 atoms of three elements, random order subsets of -1..6
and 1-24 sigmas (two 16-sigma passes above 16), cutoff 5.5 A.  Neighbor
sets bit-exact, features of every center and the position gradients of
sampled atoms within the parity tolerances; on some of them also the
dense Jacobian rows, the strain derivatives and features at random
reference points."""
import numpy as np
import pytest

from paper_2303_12980_gb300 import synth

from parity import FEAT_TOL, GRAD_TAU, GRAD_TOL, JAC_TAU, feature_errors, grad_errors

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    import torch as t
    assert t.cuda.is_available(), "GPU tests need CUDA"
    from paper_2303_12980_gb300 import build
    build.build()
    return t


def _structure(rng):
    n = int(rng.integers(4, 49))
    pbc = rng.integers(0, 2, 3).astype(np.uint8)
    L = rng.uniform(5.0, 11.0, 3)
    cell = np.diag(L)
    cell[1, 0], cell[2, 0], cell[2, 1] = rng.uniform(-0.3, 0.3, 3) * L[[1, 2, 2]]
    pos = []
    tries = 0
    while len(pos) < n and tries < 20000:
        tries += 1
        x = rng.uniform(0.0, 1.0, 3) @ cell
        shifts = [np.array([a, b, c]) @ cell for a in (-1, 0, 1) for b in (-1, 0, 1) for c in (-1, 0, 1)
                  if all(pbc[k] or (a, b, c)[k] == 0 for k in range(3))]
        if all(np.linalg.norm(x - p + sh) >= 0.9 for p in pos for sh in shifts):
            pos.append(x)
    pos = np.array(pos) + rng.uniform(-20.0, 20.0, 3)  # away from the origin
    return pos, rng.integers(0, 3, len(pos)).astype(np.int32), cell, pbc


def _batch(seed, orders, n_sig):
    rng = np.random.default_rng(seed)
    parts = [_structure(rng) for _ in range(12)]
    n_gauss, coef, expo = synth.gaussian_table(rng, [2, 5, 7], 3)
    w = synth.Workload(
        name="random_batch", positions=np.ascontiguousarray(np.concatenate([p for p, _, _, _ in parts])),
        cells=np.stack([c for _, _, c, _ in parts]), pbc=np.stack([b for _, _, _, b in parts]),
        atom_off=np.concatenate([[0], np.cumsum([len(p) for p, _, _, _ in parts])]).astype(np.int64),
        species=np.concatenate([s for _, s, _, _ in parts]), n_gauss=n_gauss, gauss_coef=coef,
        gauss_exp=expo, orders=orders, sigmas=[float(s) for s in np.geomspace(0.1, 1.2, n_sig)], cutoff=5.5)
    return w, rng


@pytest.mark.parametrize("seed,orders,n_sig", [(31, [0, 1, 2, 3, 4], 8), (32, [-1, 2, 6], 5),
                                               (33, [-1, 0, 1, 2, 3, 4, 5, 6], 18)])
def test_random_jacobian_virial_points(torch, oracle_mod, seed, orders, n_sig):
    w, rng = _batch(seed, orders, n_sig)
    from paper_2303_12980_gb300.binding import GMPFeaturizer
    F = GMPFeaturizer.from_workload(w)
    pos = torch.from_numpy(w.positions).cuda()
    sp = torch.from_numpy(w.species).cuda()
    # dense Jacobian rows of every center
    feat, joff, jj, jac = F.featurize_grad(pos, sp, w.atom_off, w.cells, w.pbc)
    torch.cuda.synchronize()
    joff, jj, jac = joff.cpu().numpy(), jj.cpu().numpy(), jac.cpu().numpy()
    centers = np.arange(w.n_atoms)
    ooff, oj, ojac, oabs = oracle_mod.jacobian_rows(w, centers, want_abs=True)
    assert np.array_equal(joff, ooff) and np.array_equal(jj, oj)
    err = grad_errors(jac, ojac, oabs, tau=JAC_TAU)
    assert err.max() <= GRAD_TOL, err.max()
    # strain derivative per structure
    g = synth.upstream_gradient(w.n_atoms, w.n_features, seed=seed)
    _, _, vir = F.featurize_vjp_virial(pos, sp, w.atom_off, w.cells, w.pbc, torch.from_numpy(g).cuda())
    torch.cuda.synchronize()
    W, Wa = oracle_mod.virial(w, g.astype(np.float64), want_abs=True)
    verr = np.abs(vir.cpu().numpy() - W) / np.maximum(np.maximum(np.abs(W), GRAD_TAU * Wa), 2.0 ** -126)
    assert verr.max() <= GRAD_TOL, verr.max()
    # reference points: 4 per structure, anywhere in (or near) the structure
    pts, poff = [], [0]
    for s in range(w.n_struct):
        a0, a1 = w.atom_off[s], w.atom_off[s + 1]
        c = w.positions[a0:a1].mean(0)
        pts.append(c + rng.uniform(-4.0, 4.0, (4, 3)))
        poff.append(poff[-1] + 4)
    pts = np.concatenate(pts)
    poff = np.array(poff, np.int64)
    fp = F.featurize_points(pos, sp, w.atom_off, w.cells, w.pbc, torch.from_numpy(pts).cuda(), poff)
    torch.cuda.synchronize()
    ref, fabs = oracle_mod.point_features(w, pts, np.repeat(np.arange(w.n_struct), 4), want_abs=True)
    perr = feature_errors(fp.cpu().numpy(), ref, fabs)
    assert perr.max() <= FEAT_TOL, perr.max()


@pytest.mark.parametrize("seed,orders,n_sig", [(21, [0, 1, 2, 3, 4, 5, 6], 6),
                                               (22, [-1, 0, 2, 5], 24),
                                               (23, [1, 3, 4, 6], 11),
                                               (24, [-1], 1),
                                               (25, [6], 17),
                                               (26, [4, 0, -1, 2], 3),
                                               (27, [0, 1, 2, 3, 4], 8),
                                               (28, [-1, 0, 1, 2, 3, 4, 5, 6], 16)])
def test_random_batches_against_oracle(torch, oracle_mod, seed, orders, n_sig):
    w, rng = _batch(seed, orders, n_sig)
    from paper_2303_12980_gb300.binding import GMPFeaturizer
    F = GMPFeaturizer.from_workload(w)
    pos = torch.from_numpy(w.positions).cuda()
    sp = torch.from_numpy(w.species).cuda()
    noff, nj, nsh = F.neighbors(pos, sp, w.atom_off, w.cells, w.pbc)
    ooff, oj, osh, _ = oracle_mod.neighbors(w)
    assert np.array_equal(noff.cpu().numpy(), ooff)
    assert np.array_equal(nj.cpu().numpy(), oj)
    assert np.array_equal(nsh.cpu().numpy(), osh)
    g = synth.upstream_gradient(w.n_atoms, w.n_features, seed=seed)
    feat, gp = F.featurize_vjp(pos, sp, w.atom_off, w.cells, w.pbc, torch.from_numpy(g).cuda())
    f_only = F.featurize(pos, sp, w.atom_off, w.cells, w.pbc)
    torch.cuda.synchronize()
    ref, fabs = oracle_mod.features(w, want_abs=True)
    for f in (feat, f_only):
        err = feature_errors(f.cpu().numpy(), ref, fabs)
        assert err.max() <= FEAT_TOL, err.max()
    atoms = rng.choice(w.n_atoms, 24, replace=False)
    gref, gscale = oracle_mod.vjp_atoms(w, g, atoms, want_abs=True)
    gerr = grad_errors(gp.cpu().numpy()[atoms], gref, gscale)
    assert gerr.max() <= GRAD_TOL, gerr.max()


def _random_tables(rng, n_el):
    """Per-element Gaussian tables of 1-8 primitives, exponents 0.1-20 A^-2,
    coefficients 0.05-2 with about one in five negative."""
    n_gauss = rng.integers(1, 9, n_el).astype(np.int32)
    k = int(n_gauss.sum())
    expo = np.exp(rng.uniform(np.log(0.1), np.log(20.0), k))
    coef = rng.uniform(0.05, 2.0, k) * np.where(rng.uniform(size=k) < 0.2, -1.0, 1.0)
    return n_gauss, coef, expo


@pytest.mark.parametrize("seed", [41, 42, 43, 44, 45, 46, 47])
def test_random_tables_chunks_and_graph_replay(torch, oracle_mod, seed):
    """Random probe sets on random batches: 1-5 elements with 1-8 Gaussians
    of either sign, a random order subset, 1-20 sigmas in random order, a
    cutoff of 3.5-7 A.  Neighbor sets bit-exact; features and the VJP of
    sampled atoms against the oracle; the Jacobian call's features too, its
    rows taken in three center chunks bit-identical to the whole-batch call
    and matching the oracle on sampled centers; the strain derivatives and
    features at random points near each structure against the oracle;
    CUDA-graph replays on a side stream give the eager results bit for
    bit."""
    rng = np.random.default_rng(seed)
    n_el = int(rng.integers(1, 6))
    parts = [_structure(rng) for _ in range(10)]
    n_gauss, coef, expo = _random_tables(rng, n_el)
    orders = sorted(rng.choice(np.arange(-1, 7), int(rng.integers(1, 9)), replace=False).tolist())
    rng.shuffle(orders)
    sig = rng.permutation(np.geomspace(0.08, 1.4, int(rng.integers(1, 21)))).tolist()
    w = synth.Workload(
        name="random_tables", positions=np.ascontiguousarray(np.concatenate([p for p, _, _, _ in parts])),
        cells=np.stack([c for _, _, c, _ in parts]), pbc=np.stack([b for _, _, _, b in parts]),
        atom_off=np.concatenate([[0], np.cumsum([len(p) for p, _, _, _ in parts])]).astype(np.int64),
        species=np.concatenate([s % n_el for _, s, _, _ in parts]).astype(np.int32), n_gauss=n_gauss,
        gauss_coef=coef, gauss_exp=expo, orders=[int(o) for o in orders], sigmas=sig,
        cutoff=float(rng.uniform(3.5, 7.0)))
    from paper_2303_12980_gb300.binding import GMPFeaturizer
    F = GMPFeaturizer.from_workload(w)
    pos = torch.from_numpy(w.positions).cuda()
    sp = torch.from_numpy(w.species).cuda()
    noff, nj, nsh = F.neighbors(pos, sp, w.atom_off, w.cells, w.pbc)
    ooff, oj, osh, _ = oracle_mod.neighbors(w)
    assert np.array_equal(noff.cpu().numpy(), ooff)
    assert np.array_equal(nj.cpu().numpy(), oj)
    assert np.array_equal(nsh.cpu().numpy(), osh)
    g = torch.from_numpy(synth.upstream_gradient(w.n_atoms, w.n_features, seed=seed)).cuda()
    feat, gp = F.featurize_vjp(pos, sp, w.atom_off, w.cells, w.pbc, g)
    torch.cuda.synchronize()
    ref, fabs = oracle_mod.features(w, want_abs=True)
    err = feature_errors(feat.cpu().numpy(), ref, fabs)
    assert err.max() <= FEAT_TOL, err.max()
    atoms = rng.choice(w.n_atoms, 16, replace=False)
    gref, gscale = oracle_mod.vjp_atoms(w, g.cpu().numpy(), atoms, want_abs=True)
    gerr = grad_errors(gp.cpu().numpy()[atoms], gref, gscale)
    assert gerr.max() <= GRAD_TOL, gerr.max()
    # the Jacobian whole and in three chunks
    fw, jo, jj, jac = (t.cpu().numpy() for t in F.featurize_grad(pos, sp, w.atom_off, w.cells, w.pbc))
    # (its records are sorted by neighbor atom, not grouped by species: the
    # features agree to rounding, not bit for bit)
    err = feature_errors(fw, ref, fabs)
    assert err.max() <= FEAT_TOL, err.max()
    cuts = np.sort(rng.choice(np.arange(1, w.n_atoms), 2, replace=False))
    for b, e in zip([0, cuts[0], cuts[1]], [cuts[0], cuts[1], w.n_atoms]):
        fc, jc, jjc, jacc = (t.cpu().numpy() for t in
                             F.featurize_grad(pos, sp, w.atom_off, w.cells, w.pbc, centers=(int(b), int(e))))
        assert np.array_equal(fc, fw[b:e])
        assert np.array_equal(jc, jo[b:e + 1] - jo[b])
        assert np.array_equal(jjc, jj[jo[b]:jo[e]]) and np.array_equal(jacc, jac[jo[b]:jo[e]])
    centers = np.sort(rng.choice(w.n_atoms, 24, replace=False))
    co, cj, cjac, cabs = oracle_mod.jacobian_rows(w, centers, want_abs=True)
    for t, i in enumerate(centers):
        a, b = jo[i], jo[i + 1]
        assert np.array_equal(jj[a:b], cj[co[t]:co[t + 1]])
        jerr = grad_errors(jac[a:b], cjac[co[t]:co[t + 1]], cabs[co[t]:co[t + 1]], tau=JAC_TAU)
        assert jerr.max() <= GRAD_TOL, (i, jerr.max())
    # strain derivative of each structure, and features at random points
    # near each structure (some far from every atom)
    _, _, vir = F.featurize_vjp_virial(pos, sp, w.atom_off, w.cells, w.pbc, g)
    pts = np.concatenate([w.positions[w.atom_off[t]:w.atom_off[t + 1]].mean(0) + rng.uniform(-6.0, 6.0, (3, 3))
                          for t in range(w.n_struct)])
    poff = np.arange(0, 3 * w.n_struct + 1, 3, dtype=np.int64)
    fp = F.featurize_points(pos, sp, w.atom_off, w.cells, w.pbc, torch.from_numpy(pts).cuda(), poff)
    torch.cuda.synchronize()
    W, Wa = oracle_mod.virial(w, g.cpu().numpy().astype(np.float64), want_abs=True)
    verr = np.abs(vir.cpu().numpy() - W) / np.maximum(np.maximum(np.abs(W), GRAD_TAU * Wa), 2.0 ** -126)
    assert verr.max() <= GRAD_TOL, verr.max()
    pref, pabs = oracle_mod.point_features(w, pts, np.repeat(np.arange(w.n_struct), 3), want_abs=True)
    perr = feature_errors(fp.cpu().numpy(), pref, pabs)
    assert perr.max() <= FEAT_TOL, perr.max()
    # graph replays on a side stream, positions moved in place between calls
    Fg = GMPFeaturizer.from_workload(w)
    Fg.set_graph(True)
    s = torch.cuda.Stream()
    fo = torch.empty_like(feat)
    go = torch.empty_like(gp)
    with torch.cuda.stream(s):
        for step in range(3):
            if step:
                pos += 0.01 * torch.randn_like(pos)
            Fg.featurize_vjp(pos, sp, w.atom_off, w.cells, w.pbc, g, out=(fo, go))
            fe, ge = F.featurize_vjp(pos, sp, w.atom_off, w.cells, w.pbc, g)
            s.synchronize()
            assert torch.equal(fo, fe), step
            assert torch.equal(go, ge), step


def _dense_structure(rng, nmax, jitter=0.0):
    """2..nmax atoms at 0.04-0.09 atoms/A^3 in a skewed cell plus Gaussian
    jitter of std `jitter` (closer than 0.7 A dropped), random periodic
    axes, moved by up to 30 A."""
    n = int(rng.integers(2, nmax))
    pbc = rng.integers(0, 2, 3).astype(np.uint8)
    L = (n / rng.uniform(0.04, 0.09)) ** (1 / 3) * np.exp(rng.uniform(-0.3, 0.3, 3))
    cell = np.diag(L)
    cell[1, 0], cell[2, 0], cell[2, 1] = rng.uniform(-0.25, 0.25, 3) * L[[1, 2, 2]]
    pos = rng.uniform(0, 1, (n, 3)) @ cell + rng.normal(0.0, jitter, (n, 3))
    keep = [0]
    for a in range(1, n):
        if all(np.linalg.norm(pos[a] - pos[b]) > 0.7 for b in keep):
            keep.append(a)
    return pos[keep] + rng.uniform(-30, 30, 3), rng.integers(0, 4, len(keep)).astype(np.int32), cell, pbc


@pytest.mark.parametrize("seed,many_sigmas", [(101, False), (106, False), (114, False), (119, False),
                                              (124, False), (201, True), (209, True), (213, True)])
def test_random_dense_structures(torch, oracle_mod, seed, many_sigmas):
    """1-4 structures of up to 300 atoms at liquid-like densities (or, with
    many sigmas, 1-3 of up to 120 atoms and 25-60 sigmas: two to four
    16-sigma passes), 1-4 elements, random order subsets in random column
    order, 1-24 sigmas from 0.05-0.2 to 0.5-2 A, cutoff 4-9 A: features, VJP,
    strain derivatives, features at random points and Jacobian rows of
    sampled centers against the oracle.  Seeds 106 and 119 have Jacobian
    rows of far pairs that the center's large adjoints lift above 2^-126
    while their exponentials lie below 2^-158 (the per-lane exponent offset
    of the Jacobian kernel); seed 213 has subnormal features at a point far
    from every atom (the invariant's products are ordered (w m) m)."""
    rng = np.random.default_rng(seed)
    n_el = int(rng.integers(1, 5))
    nmax, nst, ns = (120, 4, (25, 61)) if many_sigmas else (300, 5, (1, 25))
    parts = [_dense_structure(rng, int(rng.integers(3, nmax))) for _ in range(int(rng.integers(1, nst)))]
    n_gauss, coef, expo = synth.gaussian_table(rng, list(rng.integers(1, 9, n_el)), int(rng.integers(1, 7)))
    orders = rng.choice(np.arange(-1, 7), int(rng.integers(1, 9)), replace=False).tolist()
    sig = np.geomspace(rng.uniform(0.05, 0.2), rng.uniform(0.5, 2.0), int(rng.integers(*ns))).tolist()
    w = synth.Workload(
        name="dense", positions=np.ascontiguousarray(np.concatenate([p for p, _, _, _ in parts])),
        cells=np.stack([c for _, _, c, _ in parts]), pbc=np.stack([b for _, _, _, b in parts]),
        atom_off=np.concatenate([[0], np.cumsum([len(p) for p, _, _, _ in parts])]).astype(np.int64),
        species=np.concatenate([s % n_el for _, s, _, _ in parts]).astype(np.int32), n_gauss=n_gauss,
        gauss_coef=coef, gauss_exp=expo, orders=[int(o) for o in orders], sigmas=sig,
        cutoff=float(rng.uniform(4.0, 9.0)))
    from paper_2303_12980_gb300.binding import GMPFeaturizer
    F = GMPFeaturizer.from_workload(w)
    pos = torch.from_numpy(w.positions).cuda()
    sp = torch.from_numpy(w.species).cuda()
    g = torch.from_numpy(synth.upstream_gradient(w.n_atoms, w.n_features, seed=seed)).cuda()
    feat, gp, vir = F.featurize_vjp_virial(pos, sp, w.atom_off, w.cells, w.pbc, g)
    pts = np.concatenate([w.positions[w.atom_off[t]:w.atom_off[t + 1]].mean(0) + rng.uniform(-8, 8, (4, 3))
                          for t in range(w.n_struct)])
    poff = np.arange(0, 4 * w.n_struct + 1, 4, dtype=np.int64)
    fp = F.featurize_points(pos, sp, w.atom_off, w.cells, w.pbc, torch.from_numpy(pts).cuda(), poff)
    _, jo, jj, jac = (t.cpu().numpy() for t in F.featurize_grad(pos, sp, w.atom_off, w.cells, w.pbc))
    torch.cuda.synchronize()
    ref, fabs = oracle_mod.features(w, want_abs=True)
    assert feature_errors(feat.cpu().numpy(), ref, fabs).max() <= FEAT_TOL
    atoms = rng.choice(w.n_atoms, min(32, w.n_atoms), replace=False)
    gref, gscale = oracle_mod.vjp_atoms(w, g.cpu().numpy(), atoms, want_abs=True)
    assert grad_errors(gp.cpu().numpy()[atoms], gref, gscale).max() <= GRAD_TOL
    W, Wa = oracle_mod.virial(w, g.cpu().numpy().astype(np.float64), want_abs=True)
    verr = np.abs(vir.cpu().numpy() - W) / np.maximum(np.maximum(np.abs(W), GRAD_TAU * Wa), 2.0 ** -126)
    assert verr.max() <= GRAD_TOL, verr.max()
    pref, pabs = oracle_mod.point_features(w, pts, np.repeat(np.arange(w.n_struct), 4), want_abs=True)
    assert feature_errors(fp.cpu().numpy(), pref, pabs).max() <= FEAT_TOL
    centers = np.sort(rng.choice(w.n_atoms, min(12, w.n_atoms), replace=False))
    if seed == 119:
        centers = np.arange(w.n_atoms)  # the far rows are spread over the centers
    co, cj, cjac, cabs = oracle_mod.jacobian_rows(w, centers, want_abs=True)
    for t, i in enumerate(centers):
        a, b = jo[i], jo[i + 1]
        assert np.array_equal(jj[a:b], cj[co[t]:co[t + 1]])
        jerr = grad_errors(jac[a:b], cjac[co[t]:co[t + 1]], cabs[co[t]:co[t + 1]], tau=JAC_TAU)
        assert jerr.max() <= GRAD_TOL, (i, jerr.max())
