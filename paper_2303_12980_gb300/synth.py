"""Seeded synthetic workloads shaped like the GMP featurization workloads.

This module holds inputs only: atomic structures (positions, cells,
periodicity, species), per-element Gaussian density tables and probe
choices.  It contains none of the feature arithmetic, so both the CUDA path
and the CPU oracle can be fed from it.

The paper (GMP-Featurizer, arXiv 2303.12980) featurizes molecules,
nano-particles and periodic crystals given lattice vectors, positions and
atom types (Statement of Needs; Overview), with per-element Gaussian
densities read from pseudopotential files and probes given as lists of MCSH
orders and Gaussian sigmas (Examples).  No pseudopotential file or dataset
ships here, so every table and structure below is synthetic and seeded
(numpy PCG64, seed = 1000 + workload id).

Density tables: element e has K Gaussians c_k exp(-alpha_k r^2) with alpha_k
log-uniform in [0.1, 20] A^-2 and c_k uniform in [0.1, 1], then all c_k of
the element scaled so that sum_k c_k (pi/alpha_k)^(3/2) equals its valence
charge Z_e (the integral of the density).
"""
from __future__ import annotations

from dataclasses import dataclass, field
import math

import numpy as np

__all__ = [
    "Workload", "gaussian_table", "fcc_supercell", "random_periodic_box",
    "random_cluster", "workload", "WORKLOADS", "subset_centers",
]


@dataclass
class Workload:
    """One batch of structures plus the probe definition.

    positions: [N,3] float64 raw Cartesian positions (Angstrom), structures
        concatenated; atom_off[s]:atom_off[s+1] are the atoms of structure s.
    cells: [S,3,3] float64, rows are lattice vectors (ignored on axes that
        are not periodic; may be zero for clusters).
    pbc: [S,3] uint8.
    species: [N] int32 element ids.
    n_gauss: [E] int32, gauss_coef / gauss_exp: flattened per-element lists.
    orders, sigmas, cutoff: the probe set (feature order is order-major).
    """

    name: str
    positions: np.ndarray
    cells: np.ndarray
    pbc: np.ndarray
    atom_off: np.ndarray
    species: np.ndarray
    n_gauss: np.ndarray
    gauss_coef: np.ndarray
    gauss_exp: np.ndarray
    orders: list
    sigmas: list
    cutoff: float
    meta: dict = field(default_factory=dict)

    @property
    def n_atoms(self) -> int:
        return int(self.positions.shape[0])

    @property
    def n_struct(self) -> int:
        return int(self.cells.shape[0])

    @property
    def n_elements(self) -> int:
        return int(self.n_gauss.shape[0])

    @property
    def n_features(self) -> int:
        return sum(1 if l < 0 else len(self.sigmas) for l in self.orders)

    @property
    def gauss_off(self) -> np.ndarray:
        return np.concatenate([[0], np.cumsum(self.n_gauss)]).astype(np.int32)

    def replace(self, **kw) -> "Workload":
        d = dict(self.__dict__)
        d.update(kw)
        return Workload(**d)


def gaussian_table(rng: np.random.Generator, charges, n_gauss: int):
    """Per-element Gaussian densities normalised to the given charges."""
    coef, expo = [], []
    for z in charges:
        a = np.exp(rng.uniform(math.log(0.1), math.log(20.0), n_gauss))
        c = rng.uniform(0.1, 1.0, n_gauss)
        c *= float(z) / float(np.sum(c * (math.pi / a) ** 1.5))
        coef.append(c)
        expo.append(a)
    return (np.full(len(charges), n_gauss, np.int32),
            np.concatenate(coef).astype(np.float64),
            np.concatenate(expo).astype(np.float64))


def _assign_species(rng, n, fractions):
    counts = [int(round(n * f)) for f in fractions]
    counts[-1] = n - sum(counts[:-1])
    sp = np.concatenate([np.full(c, e, np.int32) for e, c in enumerate(counts)])
    return rng.permutation(sp).astype(np.int32)


def fcc_supercell(rng, a: float, reps, jitter: float, vacuum_z: float = 0.0):
    """FCC conventional cells repeated reps=(nx,ny,nz), Gaussian jitter of
    std `jitter` per coordinate, optional vacuum added to the cell along z."""
    nx, ny, nz = reps
    basis = np.array([[0, 0, 0], [0, .5, .5], [.5, 0, .5], [.5, .5, 0]], np.float64)
    g = np.stack(np.meshgrid(np.arange(nx), np.arange(ny), np.arange(nz), indexing="ij"), -1)
    frac = (g.reshape(-1, 1, 3) + basis[None]).reshape(-1, 3)
    pos = frac * a
    pos = pos + rng.normal(0.0, jitter, pos.shape)
    cell = np.diag([nx * a, ny * a, nz * a + vacuum_z]).astype(np.float64)
    return pos.astype(np.float64), cell


def _violators(pos, L, min_sep, periodic):
    """Indices j of every pair i < j closer than min_sep (minimum image
    when periodic); resampling those j's removes the violation."""
    d = pos[:, None, :] - pos[None, :, :]
    if periodic:
        d -= L * np.round(d / L)
    r2 = np.einsum("ijk,ijk->ij", d, d)
    close = np.triu(r2 < min_sep * min_sep, k=1)
    return np.unique(np.nonzero(close)[1])


def random_periodic_box(rng, n: int, L: float, min_sep: float):
    """n points uniform in a periodic cube of edge L with minimum-image
    separation >= min_sep (rejection: resample offenders until none)."""
    pos = rng.uniform(0.0, L, (n, 3))
    for _ in range(10000):
        bad = _violators(pos, L, min_sep, True)
        if bad.size == 0:
            return pos
        pos[bad] = rng.uniform(0.0, L, (bad.size, 3))
    raise RuntimeError("rejection sampling did not converge")


def random_cluster(rng, n: int, density: float, min_sep: float):
    """n points uniform in a sphere sized to `density`, separation >= min_sep."""
    R = (3.0 * n / (4.0 * math.pi * density)) ** (1.0 / 3.0)

    def draw(k):
        v = rng.normal(size=(k, 3))
        v /= np.linalg.norm(v, axis=1, keepdims=True)
        return v * R * rng.uniform(0.0, 1.0, (k, 1)) ** (1.0 / 3.0)

    pos = draw(n)
    for _ in range(10000):
        bad = _violators(pos, 0.0, min_sep, False)
        if bad.size == 0:
            return pos, R
        pos[bad] = draw(bad.size)
    raise RuntimeError("rejection sampling did not converge")


def _single(name, pos, cell, pbc, species, table, orders, sigmas, cutoff, meta=None):
    n_gauss, coef, expo = table
    return Workload(
        name=name,
        positions=np.ascontiguousarray(pos, np.float64),
        cells=np.ascontiguousarray(cell.reshape(1, 3, 3), np.float64),
        pbc=np.array([pbc], np.uint8),
        atom_off=np.array([0, pos.shape[0]], np.int64),
        species=np.ascontiguousarray(species, np.int32),
        n_gauss=n_gauss, gauss_coef=coef, gauss_exp=expo,
        orders=list(orders), sigmas=[float(s) for s in sigmas], cutoff=float(cutoff),
        meta=dict(meta or {}),
    )


def random64_box(seed: int = 1000) -> Workload:
    """64 atoms in a periodic 10 A cube, 1.0 A minimum separation, two
    elements 50/50 with 4 Gaussians (charges 4 and 6); orders 0-2, sigmas
    {0.1, 0.3, 0.6, 1.0} A, cutoff 6 A."""
    rng = np.random.default_rng(seed)
    table = gaussian_table(rng, [4, 6], 4)
    pos = random_periodic_box(rng, 64, 10.0, 1.0)
    species = _assign_species(rng, 64, [0.5, 0.5])
    return _single("random64_box", pos, np.eye(3) * 10.0, [1, 1, 1], species, table,
                   [0, 1, 2], [0.1, 0.3, 0.6, 1.0], 6.0)


def fcc4096(seed: int = 1001) -> Workload:
    """FCC a = 3.6 A, 8x8x16 conventional cells (4096 atoms), jitter 0.1 A,
    three elements at 0.5/0.3/0.2 with 5 Gaussians (charges 4, 6, 8);
    orders 0-4, 8 sigmas log-spaced 0.05-1.2 A, cutoff 8 A."""
    rng = np.random.default_rng(seed)
    table = gaussian_table(rng, [4, 6, 8], 5)
    pos, cell = fcc_supercell(rng, 3.6, (8, 8, 16), 0.1)
    species = _assign_species(rng, pos.shape[0], [0.5, 0.3, 0.2])
    return _single("fcc4096", pos, cell, [1, 1, 1], species, table,
                   [0, 1, 2, 3, 4], np.geomspace(0.05, 1.2, 8), 8.0)


def batched10k(seed: int = 1002, n_struct: int = 10000) -> Workload:
    """n_struct structures with atom counts log-uniform in [8, 256]; even
    indices periodic cubes at 0.08 atoms/A^3, odd indices clusters (uniform
    in a sphere at the same density); 1.0 A minimum separation; each uses
    1-5 elements drawn from a 10-element table (5 Gaussians, integer charges
    1-8); orders 0-4, 8 sigmas log-spaced 0.05-1.2 A, cutoff 7 A."""
    rng = np.random.default_rng(seed)
    charges = rng.integers(1, 9, 10)
    table = gaussian_table(rng, charges, 5)
    sizes = np.floor(np.exp(rng.uniform(math.log(8), math.log(257), n_struct))).astype(np.int64)
    sizes = np.clip(sizes, 8, 256)
    pos_l, cells, pbc, sp_l = [], [], [], []
    for s in range(n_struct):
        n = int(sizes[s])
        if s % 2 == 0:
            L = (n / 0.08) ** (1.0 / 3.0)
            p = random_periodic_box(rng, n, L, 1.0)
            cells.append(np.eye(3) * L)
            pbc.append([1, 1, 1])
        else:
            p, R = random_cluster(rng, n, 0.08, 1.0)
            cells.append(np.zeros((3, 3)))
            pbc.append([0, 0, 0])
        k = int(rng.integers(1, 6))
        els = rng.choice(10, k, replace=False)
        sp_l.append(els[rng.integers(0, k, n)].astype(np.int32))
        pos_l.append(p)
    n_gauss, coef, expo = table
    return Workload(
        name="batched10k",
        positions=np.ascontiguousarray(np.concatenate(pos_l), np.float64),
        cells=np.ascontiguousarray(np.stack(cells), np.float64),
        pbc=np.array(pbc, np.uint8),
        atom_off=np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64),
        species=np.concatenate(sp_l).astype(np.int32),
        n_gauss=n_gauss, gauss_coef=coef, gauss_exp=expo,
        orders=[0, 1, 2, 3, 4], sigmas=[float(s) for s in np.geomspace(0.05, 1.2, 8)],
        cutoff=7.0,
    )


def fcc_slab262k(seed: int = 1004, reps=(32, 32, 64)) -> Workload:
    """FCC alloy slab a = 3.9 A, 32x32x64 conventional cells (262,144 atoms)
    with a 32-layer (62.4 A) vacuum gap along z, jitter 0.15 A, six elements
    at equal fractions with 6 Gaussians (charges 3-8); orders 0-6, 16 sigmas
    log-spaced 0.05-1.5 A, cutoff 8 A."""
    rng = np.random.default_rng(seed)
    table = gaussian_table(rng, [3, 4, 5, 6, 7, 8], 6)
    a = 3.9
    pos, cell = fcc_supercell(rng, a, reps, 0.15, vacuum_z=32 * a / 2)
    species = _assign_species(rng, pos.shape[0], [1 / 6] * 6)
    return _single("fcc_slab262k", pos, cell, [1, 1, 1], species, table,
                   [0, 1, 2, 3, 4, 5, 6], np.geomspace(0.05, 1.5, 16), 8.0)


def fcc_perfect262k(seed: int = 1004, reps=(32, 32, 64)) -> Workload:
    """A perfect one-element FCC crystal, a = 3.9 A, 32x32x64 conventional
    cells (262,144 atoms), periodic, no jitter: every site is equivalent and
    the orders that vanish by cubic symmetry vanish at every center.  The
    slab's element table (first element only) and probes."""
    rng = np.random.default_rng(seed)
    table = gaussian_table(rng, [3, 4, 5, 6, 7, 8], 6)
    pos, cell = fcc_supercell(rng, 3.9, reps, 0.0)
    species = np.zeros(pos.shape[0], np.int32)
    return _single("fcc_perfect262k", pos, cell, [1, 1, 1], species, table,
                   [0, 1, 2, 3, 4, 5, 6], np.geomspace(0.05, 1.5, 16), 8.0)


def fcc_perfect32k(seed: int = 1004) -> Workload:
    """The perfect crystal at 1/8 size (16x16x32 conventional cells, 32,768
    atoms), same probes; the small case for profiling its refinement."""
    w = fcc_perfect262k(seed=seed, reps=(16, 16, 32))
    return w.replace(name="fcc_perfect32k")


def fcc_slab32k(seed: int = 1004) -> Workload:
    """The alloy slab at 1/8 size (16x16x32 conventional cells, 32,768
    atoms), same probes; the small case for kernel profiling."""
    w = fcc_slab262k(seed=seed, reps=(16, 16, 32))
    return w.replace(name="fcc_slab32k")


WORKLOADS = {
    "random64_box": random64_box,
    "fcc4096": fcc4096,
    "batched10k": batched10k,
    "fcc_slab262k": fcc_slab262k,
    "fcc_slab32k": fcc_slab32k,
    "fcc_perfect32k": fcc_perfect32k,
    "fcc_perfect262k": fcc_perfect262k,
}


def workload(name: str, **kw) -> Workload:
    return WORKLOADS[name](**kw)


def subset_centers(n_atoms: int, k: int, seed: int) -> np.ndarray:
    """A fixed random subset of k atom indices (sorted)."""
    rng = np.random.default_rng(seed)
    return np.sort(rng.choice(n_atoms, size=min(k, n_atoms), replace=False)).astype(np.int64)


def upstream_gradient(n_atoms: int, n_features: int, seed: int) -> np.ndarray:
    """Seeded dL/df used to exercise vector-Jacobian products, [N, F] float32."""
    rng = np.random.default_rng(seed)
    return rng.standard_normal((n_atoms, n_features)).astype(np.float32)
