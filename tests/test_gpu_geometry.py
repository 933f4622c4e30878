"""Geometry stress cases on the GPU against the FP64 oracle: images lying on
the cutoff sphere to the last bit (and within 1e-11 A of it), coordinates
far from the origin, and small or strongly skewed cells whose cutoff spans
several cell widths, and lone pairs whose exponentials fall below the
smallest normal FP32 number.  Neighbor sets bit-exact, features and position
gradients within the parity tolerances."""
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


def _batch(base, parts, **kw):
    """One workload from (positions, species, cell, pbc) structures."""
    pos = np.concatenate([p for p, _, _, _ in parts])
    sp = np.concatenate([s for _, s, _, _ in parts]).astype(np.int32)
    off = np.cumsum([0] + [len(p) for p, _, _, _ in parts]).astype(np.int64)
    cells = np.stack([c for _, _, c, _ in parts]).astype(np.float64)
    pbc = np.array([b for _, _, _, b in parts], np.uint8)
    return base.replace(positions=pos, species=sp, atom_off=off, cells=cells, pbc=pbc, **kw)


def _check(torch, oracle_mod, w, grad_atoms=None):
    from paper_2303_12980_gb300.binding import GMPFeaturizer
    F = GMPFeaturizer.from_workload(w)
    pos = torch.from_numpy(w.positions).cuda()
    sp = torch.from_numpy(w.species).cuda()
    noff, nj, nsh = F.neighbors(pos, sp, w.atom_off, w.cells, w.pbc)
    ooff, oj, osh, _ = oracle_mod.neighbors(w)
    assert np.array_equal(noff.cpu().numpy(), ooff)
    assert np.array_equal(nj.cpu().numpy(), oj)
    assert np.array_equal(nsh.cpu().numpy(), osh)
    g = synth.upstream_gradient(w.n_atoms, w.n_features, seed=77)
    feat, gp = F.featurize_vjp(pos, sp, w.atom_off, w.cells, w.pbc, torch.from_numpy(g).cuda())
    torch.cuda.synchronize()
    ref, fabs = oracle_mod.features(w, want_abs=True)
    ferr = feature_errors(feat.cpu().numpy(), ref, fabs)
    assert ferr.max() <= FEAT_TOL, ferr.max()
    atoms = np.arange(w.n_atoms) if grad_atoms is None else np.asarray(grad_atoms)
    gref, gscale = oracle_mod.vjp_atoms(w, g, atoms, want_abs=True)
    gerr = grad_errors(gp.cpu().numpy()[atoms], gref, gscale)
    assert gerr.max() <= GRAD_TOL, gerr.max()
    return ooff


def _cubic_lattice(a, n):
    g = np.stack(np.meshgrid(*[np.arange(n)] * 3, indexing="ij"), -1).reshape(-1, 3)
    return a * g.astype(np.float64)


@pytest.mark.parametrize("rc", [4.0, 32.0 ** 0.5, 6.0])
def test_cutoff_on_lattice_distances(torch, oracle_mod, rc):
    """Simple cubic lattice, a = 2 A: with rc = 4, sqrt(32) or 6 A whole
    shells of images sit on the cutoff sphere (|d| = rc in exact
    arithmetic); the FP64 expression decides each one, periodic and cluster."""
    base = synth.workload("random64_box")
    x = _cubic_lattice(2.0, 4)
    sp = np.arange(len(x)) % 2
    cell = np.eye(3) * 8.0
    w = _batch(base, [(x, sp, cell, (1, 1, 1)), (x + 0.5, sp, np.zeros((3, 3)), (0, 0, 0))],
               cutoff=rc, orders=[0, 1, 2], sigmas=[0.2, 0.5])
    ooff = _check(torch, oracle_mod, w, grad_atoms=[0, 5, 21, 64, 100])
    assert np.diff(ooff).min() > 0


def test_cutoff_within_1e11_of_lattice_distances(torch, oracle_mod):
    """The same lattice with every coordinate moved by up to 1e-11 A, so
    that the images of the 4 A shell straddle rc = 4 on both sides."""
    base = synth.workload("random64_box")
    rng = np.random.default_rng(11)
    x = _cubic_lattice(2.0, 4)
    x = x + rng.uniform(-1e-11, 1e-11, x.shape)
    sp = np.arange(len(x)) % 2
    w = _batch(base, [(x, sp, np.eye(3) * 8.0, (1, 1, 1)), (x, sp, np.zeros((3, 3)), (0, 0, 0))],
               cutoff=4.0, orders=[0, 1, 2], sigmas=[0.2, 0.5])
    _check(torch, oracle_mod, w, grad_atoms=[0, 9, 64, 99])


def test_far_from_origin(torch, oracle_mod):
    """A cluster translated by ~3e4 A and a periodic box whose atoms sit
    700 lattice vectors away from the cell: the double-float positions keep
    the displacements, the FP64 expression keeps the neighbor sets."""
    base = synth.workload("random64_box")
    x = base.positions[:40]
    sp = base.species[:40]
    cell = base.cells[0]
    shift = np.array([12345.678, -23456.789, 34567.891])
    far = x + 700.0 * (cell[0] + cell[1] - cell[2]) + 0.25
    w = _batch(base, [(x + shift, sp, np.zeros((3, 3)), (0, 0, 0)), (far, sp, cell, (1, 1, 1))],
               orders=[-1, 0, 1, 2, 3])
    _check(torch, oracle_mod, w, grad_atoms=[0, 7, 40, 63])


def test_small_and_skewed_cells(torch, oracle_mod):
    """Two atoms in a 2.5 A cube (cutoff 6: 2.4 cell widths), and a strongly
    skewed triclinic cell with mixed periodicity (reach ~10 cell widths
    along the short reciprocal direction)."""
    base = synth.workload("random64_box")
    cube = np.eye(3) * 2.5
    skew = np.array([[3.0, 0.0, 0.0], [2.95, 0.6, 0.0], [0.3, 0.2, 2.8]])
    p_cube = np.array([[0.1, 0.2, 0.3], [1.4, 1.1, 1.6]])
    p_skew = np.array([[0.0, 0.0, 0.0], [1.7, 0.35, 1.2], [3.9, 0.4, 0.7]])
    w = _batch(base, [(p_cube, np.array([0, 1]), cube, (1, 1, 1)),
                      (p_skew, np.array([1, 0, 1]), skew, (1, 1, 0))],
               orders=[-1, 0, 1, 2], sigmas=[0.1, 0.6])
    ooff = _check(torch, oracle_mod, w)
    assert np.diff(ooff).max() > 150   # many images of few atoms


def test_image_index_limit_reported(torch):
    """Atoms of one periodic structure more than 500 cells apart (an
    unwrapped trajectory that drifted): the packed image index cannot hold
    their pair shifts, so the call fails with a device error naming it, and
    the handle stays usable."""
    from paper_2303_12980_gb300.binding import GMPError, GMPFeaturizer
    w = synth.workload("random64_box")
    pos = w.positions.copy()
    pos[1] += 600.0 * w.cells[0][0]
    F = GMPFeaturizer.from_workload(w)
    sp = torch.from_numpy(w.species).cuda()
    with pytest.raises(GMPError, match="image index"):
        F.featurize(torch.from_numpy(pos).cuda(), sp, w.atom_off, w.cells, w.pbc)
    f = F.featurize(torch.from_numpy(w.positions).cuda(), sp, w.atom_off, w.cells, w.pbc)
    torch.cuda.synchronize()
    assert torch.isfinite(f).all()


def test_near_symmetric_crystals(torch, oracle_mod):
    """One-element FCC crystals, perfect and with 1e-4 / 1e-3 A jitter:
    by symmetry the orders 1, 2, 3 and 5 vanish or nearly vanish at every
    center.  With jitter most of each center's 112 features are
    ill-conditioned in FP32 and take the double-float recomputation; in the
    perfect crystal they vanish below the refinement band and keep their
    FP32 values.  Features and position gradients against the oracle."""
    base = synth.fcc_slab262k(reps=(3, 3, 3))
    rng = np.random.default_rng(3)
    parts = []
    for jitter in (0.0, 1e-4, 1e-3):
        pos, cell = synth.fcc_supercell(rng, 3.9, (4, 4, 4), jitter)
        parts.append((pos, np.zeros(len(pos), np.int32), cell, (1, 1, 1)))
    w = _batch(base, parts)
    from paper_2303_12980_gb300.binding import GMPFeaturizer
    F = GMPFeaturizer.from_workload(w)
    f = F.featurize(torch.from_numpy(w.positions).cuda(), torch.from_numpy(w.species).cuda(),
                    w.atom_off, w.cells, w.pbc)
    torch.cuda.synchronize()
    centers = np.concatenate([np.arange(0, 256, 5), np.arange(256, 768, 3)])
    ref, fabs = oracle_mod.features(w, centers, want_abs=True)
    err = feature_errors(f.cpu().numpy()[centers], ref, fabs)
    assert err.max() <= FEAT_TOL, err.max()
    # the position gradient too: features that vanish by symmetry below the
    # refinement band keep their FP32 moments, whose adjoints are then noise
    # of the size of their rounding
    g = synth.upstream_gradient(w.n_atoms, w.n_features, seed=9)
    _, gp = F.featurize_vjp(torch.from_numpy(w.positions).cuda(), torch.from_numpy(w.species).cuda(),
                            w.atom_off, w.cells, w.pbc, torch.from_numpy(g).cuda())
    torch.cuda.synchronize()
    atoms = np.array([0, 77, 255, 300, 555, 700])
    gref, gscale = oracle_mod.vjp_atoms(w, g, atoms, want_abs=True)
    gerr = grad_errors(gp.cpu().numpy()[atoms], gref, gscale)
    assert gerr.max() <= GRAD_TOL, gerr.max()


def test_many_flags_over_two_sigma_passes(torch, oracle_mod):
    """A jittered (1e-4 A) one-element FCC crystal of 2048 atoms with 24
    sigmas, two 16-sigma passes: most features of every center are
    recomputed in double-float, and a features call refines once after both
    passes, so each order's refinement queue takes an entry per center and
    pass (more than the atoms plus the queue's slack).  Sampled centers
    against the oracle."""
    base = synth.fcc_slab262k(reps=(3, 3, 3))
    rng = np.random.default_rng(8)
    pos, cell = synth.fcc_supercell(rng, 3.9, (8, 8, 8), 1e-4)
    w = _batch(base, [(pos, np.zeros(len(pos), np.int32), cell, (1, 1, 1))],
               sigmas=list(np.geomspace(0.05, 1.5, 24)))
    from paper_2303_12980_gb300.binding import GMPFeaturizer
    F = GMPFeaturizer.from_workload(w)
    f = F.featurize(torch.from_numpy(w.positions).cuda(), torch.from_numpy(w.species).cuda(),
                    w.atom_off, w.cells, w.pbc)
    torch.cuda.synchronize()
    centers = np.arange(0, w.n_atoms, 41)
    ref, fabs = oracle_mod.features(w, centers, want_abs=True)
    err = feature_errors(f.cpu().numpy()[centers], ref, fabs)
    assert err.max() <= FEAT_TOL, err.max()


@pytest.mark.parametrize("sigmas", [[0.1], [0.1, 0.25, 0.6]])
def test_far_pairs_below_fp32_normal_range(torch, oracle_mod, sigmas):
    """Two-atom clusters of one element (a single Gaussian, alpha = 4) at
    4.6, 4.9 and 5.3 A: exp(-alpha r^2) is 2e-37, 2e-42 and 2e-49, the
    probe's exp(-B r^2) at sigma = 0.1 straddles 2^-126 as well.  A row of
    the Jacobian (or, with sigma = 0.1 alone, an atom's whole gradient)
    then consists of those terms only, multiplied by adjoints of order 10,
    and a density at a point 4.69 A from the atom (exp(-alpha r^2) = 6e-39)
    is a single such term: a factor flushed to zero, or kept with the few
    digits of an FP32 subnormal, shows there.  Features, Jacobian rows, the
    VJP of every atom, the strain derivative and features at such points
    against the oracle."""
    u = np.array([0.48, -0.6, 0.64])
    u /= np.linalg.norm(u)
    parts = [(np.array([[1.0, 2.0, 3.0], [1.0, 2.0, 3.0] + r * u]), np.zeros(2, np.int32), np.zeros((3, 3)),
              (0, 0, 0)) for r in (4.6, 4.9, 5.3)]
    base = synth.Workload(name="far_pairs", positions=np.zeros((0, 3)), cells=np.zeros((0, 3, 3)),
                          pbc=np.zeros((0, 3), np.uint8), atom_off=np.zeros(1, np.int64),
                          species=np.zeros(0, np.int32), n_gauss=np.array([1], np.int32),
                          gauss_coef=np.array([5.0]), gauss_exp=np.array([4.0]), orders=[-1, 0, 1, 2, 3, 4],
                          sigmas=sigmas, cutoff=5.5)
    w = _batch(base, parts)
    # the 4.9 A pair exercises the band: its density row lies below 2^-126
    # (a flushed zero is off by ~3% of that floor), its order-0 row at
    # sigma = 0.1 above it (a flushed zero is off by 100%)
    ooff, oj, ojac, oabs = oracle_mod.jacobian_rows(w, None, want_abs=True)
    row = ooff[2] + 1
    assert oj[row] == 3
    assert 1e-41 < np.linalg.norm(ojac[row, 0]) < 2.0 ** -126 < np.linalg.norm(ojac[row, 1])
    _check(torch, oracle_mod, w)
    from paper_2303_12980_gb300.binding import GMPFeaturizer
    F = GMPFeaturizer.from_workload(w)
    pos = torch.from_numpy(w.positions).cuda()
    sp = torch.from_numpy(w.species).cuda()
    _, joff, jj, jac = F.featurize_grad(pos, sp, w.atom_off, w.cells, w.pbc)
    g = synth.upstream_gradient(w.n_atoms, w.n_features, seed=5)
    _, _, vir = F.featurize_vjp_virial(pos, sp, w.atom_off, w.cells, w.pbc, torch.from_numpy(g).cuda())
    # points 4.69 A from one atom of each cluster, beyond the cutoff of the other
    pts = np.stack([w.positions[2 * s] - 4.69 * u for s in range(3)])
    poff = np.arange(4, dtype=np.int64)
    fp = F.featurize_points(pos, sp, w.atom_off, w.cells, w.pbc, torch.from_numpy(pts).cuda(), poff)
    torch.cuda.synchronize()
    assert np.array_equal(joff.cpu().numpy(), ooff) and np.array_equal(jj.cpu().numpy(), oj)
    err = grad_errors(jac.cpu().numpy(), ojac, oabs, tau=JAC_TAU)
    assert err.max() <= GRAD_TOL, err.max()
    W, Wa = oracle_mod.virial(w, g.astype(np.float64), want_abs=True)
    verr = np.abs(vir.cpu().numpy() - W) / np.maximum(np.maximum(np.abs(W), GRAD_TAU * Wa), 2.0 ** -126)
    assert verr.max() <= GRAD_TOL, verr.max()
    ref, fabs = oracle_mod.point_features(w, pts, np.arange(3), want_abs=True)
    assert 2.0 ** -126 < ref[:, 0].min()  # a flushed density would be off by 100%
    perr = feature_errors(fp.cpu().numpy(), ref, fabs)
    assert perr.max() <= FEAT_TOL, perr.max()
