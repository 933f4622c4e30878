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
