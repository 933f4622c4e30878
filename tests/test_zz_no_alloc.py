"""The allocation-free entry point (gmp_neighbor_counts_noalloc) against the
allocating one (gmp_neighbors), through the C ABI, on two calls in a row.

Some callers cannot call cudaMalloc (allocator callbacks, loops that cannot
take its implicit synchronisation, processes that reserve all device memory
up front); the no-alloc variant keeps its scratch in a static device array
shared by every call, so the second call below also checks that nothing
from the first call's (larger) contents leaks into its result.  Counts are
integers: the comparison is exact."""
import ctypes

import numpy as np
import pytest

from paper_2303_12980_gb300 import synth

pytestmark = pytest.mark.gpu


def _lib():
    from paper_2303_12980_gb300 import build
    build.build()
    from paper_2303_12980_gb300 import binding
    L = binding.load_library()
    f = L.gmp_neighbor_counts_noalloc
    f.argtypes = [ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_double,
                  ctypes.c_void_p, ctypes.c_void_p]
    f.restype = ctypes.c_int
    return f


def test_noalloc_counts_match_neighbors_two_calls():
    import torch
    from paper_2303_12980_gb300.binding import GMPFeaturizer
    assert torch.cuda.is_available()
    f = _lib()
    b = synth.batched10k(n_struct=2)   # structure 1 is a non-periodic cluster
    a0, a1 = int(b.atom_off[1]), int(b.atom_off[2])
    cluster = b.replace(positions=b.positions[a0:a1], species=b.species[a0:a1],
                        atom_off=np.array([0, a1 - a0], np.int64), cells=b.cells[1:2], pbc=b.pbc[1:2])
    assert not cluster.pbc.any()
    cases = {"fcc4096": synth.workload("fcc4096"), "random64_box": synth.workload("random64_box"),
             # exactly the 32768-atom limit of the static array
             "fcc_slab32k": synth.workload("fcc_slab32k"), "cluster": cluster}
    assert cases["fcc_slab32k"].n_atoms == 32768
    for name, w in cases.items():
        pos = torch.from_numpy(w.positions).cuda()
        sp = torch.from_numpy(w.species).cuda()
        cell = np.ascontiguousarray(w.cells[0])
        pbc = np.ascontiguousarray(w.pbc[0])
        counts = torch.full((w.n_atoms,), -1, dtype=torch.int64, device="cuda")
        st = f(w.n_atoms, pos.data_ptr(), cell.ctypes.data, pbc.ctypes.data, w.cutoff, counts.data_ptr(),
               torch.cuda.current_stream().cuda_stream)
        assert st == 0
        off, _, _ = GMPFeaturizer.from_workload(w).neighbors(pos, sp, w.atom_off, w.cells, w.pbc)
        torch.cuda.synchronize()
        assert torch.equal(counts, off[1:] - off[:-1]), name


def test_noalloc_rejects_too_many_atoms():
    f = _lib()
    cell = np.eye(3) * 10.0
    pbc = np.ones(3, np.uint8)
    # rejected on the host before any GPU work (pointers are never read)
    st = f(32769, None, cell.ctypes.data, pbc.ctypes.data, 5.0, None, None)
    assert st == 4  # GMP_ERR_CAPACITY
