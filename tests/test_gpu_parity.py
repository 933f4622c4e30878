"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle on
the same seeded inputs.  Neighbor sets bit-exact; features within 1e-5 and
derivatives within 1e-4 relative (with the cancellation floors of
tests/parity.py)."""
import numpy as np
import pytest

from paper_2303_12980_gb300 import synth

from parity import (FEAT_TAU, FEAT_TOL, GRAD_TAU, GRAD_TOL, feature_errors, grad_errors, record)

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
        err = grad_errors(jac[a:b], ojac[ooff[t]:ooff[t + 1]], oabs[ooff[t]:ooff[t + 1]])
        worst = max(worst, float(err.max()))
    record(f"jacobian/{name}", max_rel_err=worst, nnz=int(joff[-1]))
    assert worst <= GRAD_TOL, worst


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


def test_deterministic(torch):
    w = wl("fcc4096")
    pos, sp = _dev(torch, w)
    F = _featurizer(w)
    a = F.featurize(pos, sp, w.atom_off, w.cells, w.pbc)
    b = F.featurize(pos, sp, w.atom_off, w.cells, w.pbc)
    torch.cuda.synchronize()
    assert torch.equal(a, b)


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
