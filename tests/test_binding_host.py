"""Host logic of the Python binding, against a fake library (no GPU)."""
import numpy as np

from paper_2303_12980_gb300 import binding as B


class _FakeLib:
    """gmp_featurize_grad / gmp_neighbors that need `need[0]` output rows:
    they report the count through nnz_out and return GMP_ERR_CAPACITY when
    the caller's capacity is short, as the library does."""

    def __init__(self, need):
        self.need = need
        self.caps = []

    def _call(self, cap, nnz):
        self.caps.append(cap)
        nnz._obj.value = self.need[0]
        return B.GMP_OK if cap >= self.need[0] else B.GMP_ERR_CAPACITY

    def gmp_featurize_grad(self, h, S, off, pos, cell, pbc, sp, feat, joff, jj, jac, cap, nnz, stream):
        return self._call(cap, nnz)

    def gmp_neighbors(self, h, S, off, pos, cell, pbc, sp, noff, nj, ns, cap, nnz, stream):
        return self._call(cap, nnz)


def _fake_featurizer(need):
    F = object.__new__(B.GMPFeaturizer)
    F._L = _FakeLib(need)
    F._h = None
    F.num_features = 2
    F._rows = {"grad": 0, "neighbors": 0}
    return F


def _args():
    return (np.zeros((4, 3)), np.zeros(4, np.int32), [0, 4], np.eye(3)[None], np.ones((1, 3), np.uint8))


def test_grad_reuses_the_last_row_count():
    """featurize_grad allocates the last call's row count and calls the
    library a second time only when a call needs more rows."""
    need = [100]
    F = _fake_featurizer(need)
    _, _, jj, jac = F.featurize_grad(*_args())
    assert F._L.caps == [1, 100] and jj.shape == (100,) and jac.shape == (100, 2, 3)
    F._L.caps.clear()
    F.featurize_grad(*_args())
    assert F._L.caps == [100]                      # same size: one library call
    need[0] = 80
    F._L.caps.clear()
    _, _, jj, jac = F.featurize_grad(*_args())
    assert F._L.caps == [100] and jj.shape == (80,) and jac.shape == (80, 2, 3)
    need[0] = 120
    F._L.caps.clear()
    _, _, jj, _ = F.featurize_grad(*_args())
    assert F._L.caps == [80, 120] and jj.shape == (120,)


def test_neighbors_reuses_the_last_pair_count():
    need = [50]
    F = _fake_featurizer(need)
    _, nj, ns = F.neighbors(*_args())
    assert F._L.caps == [1, 50] and nj.shape == (50,) and ns.shape == (50, 3)
    F._L.caps.clear()
    need[0] = 70
    _, nj, _ = F.neighbors(*_args())
    assert F._L.caps == [50, 70] and nj.shape == (70,)
