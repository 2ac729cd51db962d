"""Seeded synthetic inputs for the CheFSI hot path (cluster geometry and start blocks).

This module is the one piece shared by the CUDA path's harness and by the CPU oracle's
tests. It draws random numbers and places atoms; it holds none of the method's
arithmetic (no stencil, potential, projector or filter formula).

Workload presets follow the synthetic clusters that stand in for the paper's Si-H
nanoclusters (Sec. 4.5 uses h = 0.5 bohr and a vacuum margin; Sec. 4 fixes n_o = 6 and
m = 20): a cubic grid of n^3 nodes with spacing h, atoms placed uniformly with a wall
margin and a minimum pairwise separation, valence charges Z in {1..4}, Kleinman-Bylander
coefficients gamma_l uniform in [-2, 2] Ha (one value for l = 0 and one shared by the
three l = 1 projectors, since gamma depends on J and l only, Sec. 2), and a start block
of orbitals uniform in (-0.5, 0.5).

Node coordinates are x_i = i*h for i = 0..n-1; the atom box is therefore
[margin, (n-1)*h - margin]^3.
"""
from __future__ import annotations

import dataclasses
from typing import Optional

import numpy as np

__all__ = [
    "Workload",
    "Cluster",
    "PRESETS",
    "preset",
    "place_atoms",
    "make_cluster",
    "initial_block",
]


@dataclasses.dataclass(frozen=True)
class Workload:
    """One synthetic CheFSI workload: grid, atoms, states, filter degree, iterations."""

    name: str
    n: int              # nodes per axis (cubic grid n^3)
    h: float            # mesh size in bohr
    natoms: int         # atoms requested (placement may fit fewer, see place_atoms)
    ns: int             # number of states (columns of the orbital block)
    degree: int         # Chebyshev filter degree m
    iters: int          # CheFSI iterations
    lanczos_k: int = 10
    margin: float = 4.0
    minsep: float = 2.0
    sigma: float = 0.8  # projector Gaussian width
    rcut: float = 3.0   # projector truncation radius
    rc_erf: float = 1.0  # width of the erf local potential
    filter_dtype: str = "f64"

    @property
    def nd(self) -> int:
        return self.n ** 3


PRESETS = {
    # small FP64 case: 24^3, h = 0.5, 4 atoms, 12 states, degree 10, 10 iterations
    "cluster24": Workload("cluster24", n=24, h=0.5, natoms=4, ns=12, degree=10, iters=10),
    # medium FP64 cluster: 96^3, h = 0.3, 40 atoms, 128 states, degree 20, 20 iterations
    "cluster96": Workload("cluster96", n=96, h=0.3, natoms=40, ns=128, degree=20, iters=20),
    # large mixed-precision cluster: 160^3, h = 0.25, 400 atoms, 1024 states, degree 24
    "cluster160": Workload("cluster160", n=160, h=0.25, natoms=400, ns=1024, degree=24,
                           iters=20, filter_dtype="f32"),
    # dense-diagonalisation check: 12^3, h = 0.5, 1 atom, 10 states
    "cluster12": Workload("cluster12", n=12, h=0.5, natoms=1, ns=10, degree=10, iters=40,
                          margin=2.5),
}


def preset(name: str) -> Workload:
    return PRESETS[name]


@dataclasses.dataclass
class Cluster:
    """Atoms of one synthetic cluster (all arrays float64, C-contiguous)."""

    n: int
    h: float
    R: np.ndarray       # (natoms, 3) positions in bohr
    Z: np.ndarray       # (natoms,) valence charges
    gamma: np.ndarray   # (natoms, 4) KB coefficients for (s, px, py, pz)
    sigma: float = 0.8
    rcut: float = 3.0
    rc_erf: float = 1.0

    @property
    def natoms(self) -> int:
        return int(self.R.shape[0])

    @property
    def nd(self) -> int:
        return self.n ** 3


def place_atoms(rng: np.random.Generator, n: int, h: float, natoms: int,
                margin: float = 4.0, minsep: float = 2.0,
                tries: int = 10_000) -> np.ndarray:
    """Uniform placement by rejection: each atom gets up to `tries` draws in the margin
    box and is kept when it is at least `minsep` from every atom placed before it.
    Placement stops at the first atom that does not fit, so small boxes hold fewer
    atoms than requested; the caller reads the count from the result's shape."""
    lo = margin
    hi = (n - 1) * h - margin
    if hi < lo:
        return np.zeros((0, 3))
    placed: list[np.ndarray] = []
    for _ in range(natoms):
        ok = False
        for _t in range(tries):
            c = rng.uniform(lo, hi, size=3)
            if all(float(np.sqrt(np.sum((c - q) ** 2))) >= minsep for q in placed):
                placed.append(c)
                ok = True
                break
        if not ok:
            break
    return np.ascontiguousarray(np.array(placed, dtype=np.float64).reshape(-1, 3))


def make_cluster(w: Workload, seed: int, natoms: Optional[int] = None) -> Cluster:
    """Cluster for workload `w` from `seed` (positions, Z in {1..4}, gamma_l in [-2, 2])."""
    ss = np.random.SeedSequence(seed)
    g_atoms = np.random.Generator(np.random.PCG64(ss.spawn(1)[0]))
    R = place_atoms(g_atoms, w.n, w.h, w.natoms if natoms is None else natoms,
                    w.margin, w.minsep)
    na = R.shape[0]
    Z = g_atoms.integers(1, 5, size=na).astype(np.float64)
    gl = g_atoms.uniform(-2.0, 2.0, size=(na, 2))
    gamma = np.empty((na, 4))
    gamma[:, 0] = gl[:, 0]
    gamma[:, 1:] = gl[:, 1:2]
    return Cluster(n=w.n, h=w.h, R=R, Z=np.ascontiguousarray(Z),
                   gamma=np.ascontiguousarray(gamma), sigma=w.sigma, rcut=w.rcut,
                   rc_erf=w.rc_erf)


def initial_block(seed: int, nd: int, ns: int, ld: Optional[int] = None,
                  dtype=np.float64) -> np.ndarray:
    """Start block of `ns` orbitals, uniform in (-0.5, 0.5), drawn by PCG64.

    Returned with shape (ns, ld): row c is column c of the column-major Nd x Ns block,
    so the buffer is exactly the column-major layout with leading dimension ld.
    Entries in rows beyond nd (padding up to ld) are zero."""
    ld = nd if ld is None else ld
    ss = np.random.SeedSequence(seed)
    g = np.random.Generator(np.random.PCG64(ss.spawn(2)[1]))
    X = np.zeros((ns, ld), dtype=np.float64)
    X[:, :nd] = g.uniform(-0.5, 0.5, size=(ns, nd))
    return np.ascontiguousarray(X.astype(dtype))
