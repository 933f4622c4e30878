"""Full-size workloads on the GPU, checked on sampled outputs the FP64 oracle
can compute one by one: the 262,144-atom FCC alloy slab (orders 0-6, 16
sigmas) and the 10,000-structure batch of periodic boxes and clusters."""
import numpy as np
import pytest

from paper_2303_12980_gb300 import synth

from parity import FEAT_TOL, GRAD_TOL, JAC_TAU, feature_errors, grad_errors, record

pytestmark = pytest.mark.gpu

_cache = {}


def _w(name):
    if name not in _cache:
        _cache[name] = synth.workload(name)
    return _cache[name]


@pytest.fixture(scope="module")
def torch():
    import torch as t
    assert t.cuda.is_available()
    from paper_2303_12980_gb300 import build
    build.build()
    return t


@pytest.mark.parametrize("name,n_centers,n_atoms", [("fcc_slab262k", 192, 6), ("batched10k", 384, 12)])
def test_full_size_sampled(torch, oracle_mod, name, n_centers, n_atoms):
    from paper_2303_12980_gb300.binding import GMPFeaturizer
    w = _w(name)
    F = GMPFeaturizer.from_workload(w)
    pos = torch.from_numpy(w.positions).cuda()
    sp = torch.from_numpy(w.species).cuda()
    F.tune(pos, sp, w.atom_off, w.cells, w.pbc, reps=1)   # the launch shapes bench.py times
    g = synth.upstream_gradient(w.n_atoms, w.n_features, seed=2024)
    feat, gp = F.featurize_vjp(pos, sp, w.atom_off, w.cells, w.pbc, torch.from_numpy(g).cuda())
    torch.cuda.synchronize()
    centers = synth.subset_centers(w.n_atoms, n_centers, seed=31)
    ref, fabs = oracle_mod.features(w, centers, want_abs=True)
    ferr = feature_errors(feat.cpu().numpy()[centers], ref, fabs)
    atoms = synth.subset_centers(w.n_atoms, n_atoms, seed=32)
    gref, gscale = oracle_mod.vjp_atoms(w, g, atoms, want_abs=True)
    gerr = grad_errors(gp.cpu().numpy()[atoms], gref, gscale)
    record(f"fullsize/{name}", features_max_rel_err=ferr.max(), vjp_max_rel_err=gerr.max(),
           centers=n_centers, atoms=n_atoms)
    assert ferr.max() <= FEAT_TOL, ferr.max()
    assert gerr.max() <= GRAD_TOL, gerr.max()
    # neighbor counts of the sampled centers equal the oracle's
    noff, _, _ = F.neighbors(pos, sp, w.atom_off, w.cells, w.pbc)
    cnt = (noff[1:] - noff[:-1]).cpu().numpy()[centers]
    ooff, _, _, _ = oracle_mod.neighbors(w, centers)
    assert np.array_equal(cnt, np.diff(ooff))


def test_full_size_jacobian_chunk(torch, oracle_mod):
    """The slab's dense Jacobian (about 37 M rows, 50 GB in all) taken as one
    chunk of 32,768 centers through gmp_featurize_grad_centers: the rows and
    features of 8 sampled centers of the chunk against the FP64 oracle
    (floors JAC_TAU G_abs and 1e-6 F_abs)."""
    from paper_2303_12980_gb300.binding import GMPFeaturizer
    w = _w("fcc_slab262k")
    F = GMPFeaturizer.from_workload(w)
    pos = torch.from_numpy(w.positions).cuda()
    sp = torch.from_numpy(w.species).cuda()
    b, e = 100000, 100000 + 32768
    feat, joff, jj, jac = F.featurize_grad(pos, sp, w.atom_off, w.cells, w.pbc, centers=(b, e))
    torch.cuda.synchronize()
    assert feat.shape == (e - b, w.n_features) and joff.shape == (e - b + 1,)
    joff, jj = joff.cpu().numpy(), jj.cpu().numpy()
    local = synth.subset_centers(e - b, 8, seed=33)
    ref, fabs = oracle_mod.features(w, local + b, want_abs=True)
    assert feature_errors(feat.cpu().numpy()[local], ref, fabs).max() <= FEAT_TOL
    ooff, oj, ojac, oabs = oracle_mod.jacobian_rows(w, local + b, want_abs=True)
    worst = 0.0
    for t, c in enumerate(local):
        r0, r1 = joff[c], joff[c + 1]
        assert np.array_equal(jj[r0:r1], oj[ooff[t]:ooff[t + 1]])
        err = grad_errors(jac[r0:r1].cpu().numpy(), ojac[ooff[t]:ooff[t + 1]], oabs[ooff[t]:ooff[t + 1]],
                          tau=JAC_TAU)
        worst = max(worst, float(err.max()))
    record("fullsize/jacobian_chunk", max_rel_err=worst, rows=int(joff[-1]))
    assert worst <= GRAD_TOL, worst


def test_edge_cases(torch, oracle_mod):
    """Empty structure in a batch, a single isolated atom, a structure with
    a triclinic cell and mixed periodicity, positions far outside the cell."""
    from paper_2303_12980_gb300.binding import GMPFeaturizer
    base = synth.workload("random64_box")
    rng = np.random.default_rng(5)
    tri = np.array([[7.0, 0.0, 0.0], [2.5, 6.5, 0.0], [1.0, 1.5, 8.0]])
    p_tri = rng.uniform(0, 1, (20, 3)) @ tri + rng.integers(-3, 4, (20, 3)) @ tri  # outside the cell
    p_one = np.array([[0.3, -0.2, 0.1]])
    pos = np.concatenate([base.positions[:10], p_one, p_tri])
    species = np.concatenate([base.species[:10], [1], rng.integers(0, 2, 20)]).astype(np.int32)
    atom_off = np.array([0, 10, 10, 11, 31], np.int64)          # structure 1 is empty
    cells = np.stack([base.cells[0], np.zeros((3, 3)), np.zeros((3, 3)), tri])
    pbc = np.array([[1, 1, 1], [0, 0, 0], [0, 0, 0], [1, 0, 1]], np.uint8)
    w = base.replace(positions=pos, species=species, atom_off=atom_off, cells=cells, pbc=pbc,
                     orders=[-1, 0, 1, 2, 3])
    F = GMPFeaturizer.from_workload(w)
    f = F.featurize(torch.from_numpy(pos).cuda(), torch.from_numpy(species).cuda(), atom_off, cells, pbc)
    torch.cuda.synchronize()
    ref, fabs = oracle_mod.features(w, want_abs=True)
    err = feature_errors(f.cpu().numpy(), ref, fabs)
    assert err.max() <= FEAT_TOL, err.max()
    noff, nj, nsh = F.neighbors(torch.from_numpy(pos).cuda(), torch.from_numpy(species).cuda(),
                                atom_off, cells, pbc)
    ooff, oj, osh, _ = oracle_mod.neighbors(w)
    assert np.array_equal(noff.cpu().numpy(), ooff)
    assert np.array_equal(nj.cpu().numpy(), oj)
    assert np.array_equal(nsh.cpu().numpy(), osh)


def test_invalid_inputs_are_reported(torch):
    from paper_2303_12980_gb300.binding import GMPError, GMPFeaturizer
    w = synth.workload("random64_box")
    F = GMPFeaturizer.from_workload(w)
    pos = torch.from_numpy(w.positions).cuda()
    bad_sp = torch.from_numpy(w.species).cuda().clone()
    bad_sp[3] = 7  # only 2 elements
    with pytest.raises(GMPError, match="species"):
        F.featurize(pos, bad_sp, w.atom_off, w.cells, w.pbc)
    with pytest.raises(GMPError, match="singular"):
        F.featurize(pos, torch.from_numpy(w.species).cuda(), w.atom_off, np.zeros((1, 3, 3)), w.pbc)
    nan_pos = pos.clone()
    nan_pos[5, 1] = float("nan")
    with pytest.raises(GMPError, match="non-finite"):
        F.featurize(nan_pos, torch.from_numpy(w.species).cuda(), w.atom_off, w.cells, w.pbc)
    # the handle stays usable after reported errors
    f = F.featurize(pos, torch.from_numpy(w.species).cuda(), w.atom_off, w.cells, w.pbc)
    torch.cuda.synchronize()
    assert torch.isfinite(f).all()


def test_coincident_atoms(torch, oracle_mod):
    """Distinct atoms at the same position (r = 0 pairs other than the self
    term, where only order 1 has a gradient) in a cluster and in a cell."""
    base = synth.workload("random64_box").replace(orders=[-1, 0, 1, 2, 3])
    p = base.positions[:12].copy()
    p[5] = p[2]
    p[9] = p[2]
    p[11] = p[7]
    w = base.replace(positions=np.concatenate([p, p + 0.0]), species=np.concatenate([base.species[:12]] * 2),
                     atom_off=np.array([0, 12, 24], np.int64), cells=np.stack([base.cells[0], np.zeros((3, 3))]),
                     pbc=np.array([[1, 1, 1], [0, 0, 0]], np.uint8))
    from paper_2303_12980_gb300.binding import GMPFeaturizer
    F = GMPFeaturizer.from_workload(w)
    g = synth.upstream_gradient(w.n_atoms, w.n_features, seed=17)
    feat, gp = F.featurize_vjp(torch.from_numpy(w.positions).cuda(), torch.from_numpy(w.species).cuda(),
                               w.atom_off, w.cells, w.pbc, torch.from_numpy(g).cuda())
    torch.cuda.synchronize()
    ref, fabs = oracle_mod.features(w, want_abs=True)
    assert feature_errors(feat.cpu().numpy(), ref, fabs).max() <= FEAT_TOL
    atoms = np.arange(w.n_atoms)
    gref, gscale = oracle_mod.vjp_atoms(w, g, atoms, want_abs=True)
    assert grad_errors(gp.cpu().numpy(), gref, gscale).max() <= GRAD_TOL


def test_neighbor_image_limit(torch):
    """More neighbor images per center than the fill kernels hold (25,600):
    a capacity error with the count, and the handle stays usable."""
    from paper_2303_12980_gb300.binding import GMPError, GMPFeaturizer
    w = synth.workload("random64_box")
    big = w.replace(cutoff=52.0, orders=[0], sigmas=[0.5])   # ~64 x 590 cells of 10 A: ~37,000 images
    F = GMPFeaturizer.from_workload(big)
    pos = torch.from_numpy(w.positions).cuda()
    sp = torch.from_numpy(w.species).cuda()
    with pytest.raises(GMPError, match="neighbor images"):
        F.featurize(pos, sp, w.atom_off, w.cells, w.pbc)
    ok = GMPFeaturizer.from_workload(w).featurize(pos, sp, w.atom_off, w.cells, w.pbc)
    torch.cuda.synchronize()
    assert torch.isfinite(ok).all()


def test_huge_search_box(torch):
    """A search box of more than 2^20 cells (one atom in a 1 A periodic cube,
    cutoff 52 A: 105^3 image cells) takes the enumeration's integer-division
    path; its ~590,000 images per center end in the capacity error, and the
    handle's next call succeeds."""
    from paper_2303_12980_gb300.binding import GMPError, GMPFeaturizer
    w = synth.workload("random64_box")
    tiny = w.replace(positions=np.array([[0.3, 0.4, 0.5]]), species=np.array([0], np.int32),
                     atom_off=np.array([0, 1], np.int64), cells=np.eye(3)[None].copy(),
                     pbc=np.ones((1, 3), np.uint8), cutoff=52.0, orders=[0], sigmas=[0.5])
    F = GMPFeaturizer.from_workload(tiny)
    with pytest.raises(GMPError, match="neighbor images"):
        F.featurize(torch.from_numpy(tiny.positions).cuda(), torch.from_numpy(tiny.species).cuda(),
                    tiny.atom_off, tiny.cells, tiny.pbc)
    pos = torch.from_numpy(w.positions).cuda()
    sp = torch.from_numpy(w.species).cuda()
    ok = GMPFeaturizer.from_workload(w.replace(orders=[0], sigmas=[0.5])).featurize(pos, sp, w.atom_off,
                                                                                   w.cells, w.pbc)
    torch.cuda.synchronize()
    assert torch.isfinite(ok).all()


def test_throughput_probes(torch):
    """The FP32 FMA probes land near the nominal rate (SMs x 128 lanes x 2
    FLOP x clock, at most the maximum clock) and the ex2 probe reports a
    positive rate."""
    from paper_2303_12980_gb300.binding import probe_peaks
    p = probe_peaks(0)
    sm = torch.cuda.get_device_properties(0).multi_processor_count
    nominal = sm * 128 * 2 * 2.07e9 / 1e12
    assert 0.3 * nominal < p["fp32_fma_tflops"] < 1.05 * nominal, p
    assert 0.3 * nominal < p["fp32_fma2_tflops"] < 2.1 * nominal, p
    assert p["ex2_tops"] > 0.0, p


def test_contraction_probe(torch):
    """The moment-contraction probe: the forward kernel's packed-FP32 scheme
    and the TF32x3 tensor-core version sum 144 pairs to within their
    rounding of the cancellation-free scale, and both report a rate."""
    from paper_2303_12980_gb300.binding import probe_contraction
    r = probe_contraction(0)
    assert r["fp32"]["max_rel_err"] < 2e-6, r
    for k in ("tf32x3_16w", "tf32x3_8w", "tf32x3_presplit_16w"):
        assert r[k]["max_rel_err"] < 1e-5, r
    for v in r.values():
        assert v["gpairs_per_s"] > 0.0 and v["registers"] > 0, r


def test_sync_timeout_and_completion(torch):
    """gmp_sync with a timeout shorter than the queued work returns
    GMP_ERR_TIMEOUT (the work keeps running), and with a long one returns
    once the stream is done; the features are then complete."""
    from paper_2303_12980_gb300.binding import GMPError, GMPFeaturizer
    w = synth.workload("random64_box")
    F = GMPFeaturizer.from_workload(w)
    pos = torch.from_numpy(w.positions).cuda()
    sp = torch.from_numpy(w.species).cuda()
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        f = F.featurize(pos, sp, w.atom_off, w.cells, w.pbc, stream=s)
        a = torch.full((4096, 4096), 1e-3, device="cuda")
        for _ in range(40):  # a few hundred ms of FP32 matrix products queued behind the call
            a = a @ a
    with pytest.raises(GMPError, match="TIMEOUT"):
        F.sync(s, timeout_s=1e-4)
    F.sync(s, timeout_s=60.0)
    assert torch.isfinite(f).all()
