"""Multi-rank host logic on CPU (gloo, world_size 2): structure sharding and
the timing/throughput reduction used by bench.py under torchrun."""
import os
import socket

import numpy as np
import pytest

from paper_2303_12980_gb300 import dist_util, synth


def test_shard_structures_covers_batch_once():
    w = synth.batched10k(n_struct=200)
    for world in (1, 2, 3, 8):
        seen = []
        sizes = []
        for r in range(world):
            s0, s1 = dist_util.shard_structures(w.atom_off, r, world)
            seen.extend(range(s0, s1))
            sizes.append(int(w.atom_off[s1] - w.atom_off[s0]))
        assert seen == list(range(w.n_struct))
        if world > 1:
            assert max(sizes) - min(sizes) <= 2 * 256  # within two structures


def test_slice_workload_keeps_structures():
    w = synth.batched10k(n_struct=20)
    sub = dist_util.slice_workload(w, 5, 9)
    assert sub.n_struct == 4
    assert sub.atom_off[0] == 0
    assert np.array_equal(sub.positions, w.positions[w.atom_off[5]:w.atom_off[9]])


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms, units = dist_util.reduce_timing(10.0 + 5.0 * rank, 1000.0 * (rank + 1))
        out[rank] = (ms, units)
    finally:
        dist.destroy_process_group()


def test_reduce_timing_gloo_world2():
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_worker, args=(2, _free_port(), out), nprocs=2, join=True, start_method="spawn")
    assert out[0] == out[1] == (15.0, 3000.0)


def _vjp_push(oracle_mod, w, g, centers):
    """d L / d x of L = sum over the listed centers i of sum_f g[i, f] f_i
    (every atom's [N, 3] row), from the oracle's Jacobian rows of those
    centers: the part of the VJP one rank of a center-sharded run holds."""
    out = np.zeros((w.n_atoms, 3))
    if len(centers) == 0:
        return out
    off, jj, jac = oracle_mod.jacobian_rows(w, np.asarray(centers, np.int64))
    for t, i in enumerate(centers):
        rows = slice(off[t], off[t + 1])
        np.add.at(out, jj[rows], np.einsum("f,rfc->rc", g[i], jac[rows]))
    return out


def _vjp_worker(rank, world, port, out):
    import torch
    import torch.distributed as dist
    from oracle import oracle as O
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # one periodic structure, centers sharded: partials all-reduced
        w = synth.workload("random64_box")
        g = synth.upstream_gradient(w.n_atoms, w.n_features, seed=3).astype(np.float64)
        c0, c1 = dist_util.shard_centers(w.n_atoms, rank, world)
        part = torch.from_numpy(_vjp_push(O, w, g, range(c0, c1)))
        dist_util.allreduce_sum_(part)
        out[("centers", rank)] = part.numpy()
        # many structures, structures sharded: each rank's atoms are complete
        b = synth.batched10k(n_struct=8)
        gb = synth.upstream_gradient(b.n_atoms, b.n_features, seed=4).astype(np.float64)
        s0, s1 = dist_util.shard_structures(b.atom_off, rank, world)
        sub = dist_util.slice_workload(b, s0, s1)
        a0, a1 = int(b.atom_off[s0]), int(b.atom_off[s1])
        out[("structures", rank)] = (a0, a1, _vjp_push(O, sub, gb[a0:a1], range(sub.n_atoms)))
    finally:
        dist.destroy_process_group()


def test_sharded_vjp_matches_whole_batch_gloo_world2(oracle_mod):
    """A center-sharded VJP of one structure (partials of all atoms, one
    all-reduce) and a structure-sharded VJP of a batch (no exchange) equal
    the whole-batch VJP, on two gloo ranks with the FP64 oracle."""
    pytest.importorskip("torch")
    import torch.multiprocessing as mp
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_vjp_worker, args=(2, _free_port(), out), nprocs=2, join=True, start_method="spawn")
    w = synth.workload("random64_box")
    g = synth.upstream_gradient(w.n_atoms, w.n_features, seed=3).astype(np.float64)
    whole = _vjp_push(oracle_mod, w, g, range(w.n_atoms))
    scale = np.abs(whole).max()
    for r in range(2):
        assert np.allclose(out[("centers", r)], whole, rtol=0, atol=1e-12 * scale)
    # the pull form (centers that see each atom) agrees with the push form
    assert np.allclose(oracle_mod.vjp_atoms(w, g, np.arange(w.n_atoms)), whole, rtol=0, atol=1e-12 * scale)
    b = synth.batched10k(n_struct=8)
    gb = synth.upstream_gradient(b.n_atoms, b.n_features, seed=4).astype(np.float64)
    wb = _vjp_push(oracle_mod, b, gb, range(b.n_atoms))
    got = np.zeros_like(wb)
    for r in range(2):
        a0, a1, part = out[("structures", r)]
        got[a0:a1] = part
    assert np.allclose(got, wb, rtol=0, atol=1e-12 * np.abs(wb).max())
