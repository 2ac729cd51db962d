"""FP64 CPU oracle for the CheFSI hot path of SPARC (arXiv:1603.04334), Python side.

TEST INFRASTRUCTURE. Only the test suite, the package smoke check and the benchmark's
CPU-baseline leg may import this module. It shares no code with the CUDA library and
never loads it.

The grid operators (stencil, potential, projectors, H, filter, Lanczos) are plain C
loops in sparc_oracle.c; this module loads them with ctypes and adds the dense
Ns x Ns steps with numpy / scipy LAPACK calls used as single library steps:

* projection, Eq. (SubspaceGeneralizedEigenproblem) and the two relations after it,
  Sec. 3.4: M_s = Y^T Y, H_s = Y^T (H Y);
* the generalized eigenproblem H_s y = lambda M_s y, reduced through the Cholesky
  factor M_s = L L^T to the standard problem L^-1 H_s L^-T q = lambda q (the
  reduction LAPACK's dsygv performs; the paper solves it with LAPACK, Sec. 4);
* the subspace rotation Psi = Psi_f Y, Eq. (OrbitalTransformation), with
  Y = L^-T Q;
* residual norms ||H x_n - lambda_n x_n||_2 of the rotated, Euclidean-orthonormal
  columns;
* the CheFSI loop of Sec. 3.4 with the bounds rule stated in chefsi_bounds_*.

Readings where the paper is silent (all shared with the CUDA path's contract):
  - eigenvector signs: each column of Q is flipped so that its entry of largest
    magnitude is positive (the lowest index wins ties);
  - filter bounds on a fixed Hamiltonian: first iteration a0 = theta_min and
    a = a0 + 0.25 (b - a0) from Lanczos; later iterations a = largest Ritz value and
    a0 = smallest Ritz value of the previous iteration (the rule of the CheFSI method
    the paper cites); b = max(1.01 theta_max, theta_max + |beta_k s_k|) throughout.
"""
from __future__ import annotations

import ctypes as C
import dataclasses
import os
from fractions import Fraction
from typing import Optional

import numpy as np
import scipy.linalg as sla

from . import build as _build

_lib = None


class _Ham(C.Structure):
    _fields_ = [
        ("n0", C.c_int), ("n1", C.c_int), ("n2", C.c_int),
        ("h", C.c_double), ("no", C.c_int), ("kscale", C.c_double),
        ("V", C.POINTER(C.c_double)),
        ("natoms", C.c_int),
        ("atom_ptr", C.POINTER(C.c_long)),
        ("idx", C.POINTER(C.c_long)),
        ("chi", C.POINTER(C.c_double)),
        ("gamma", C.POINTER(C.c_double)),
    ]


def lib():
    """Load (building first if needed) the C part of the oracle."""
    global _lib
    if _lib is None:
        path = _build.build()
        L = C.CDLL(path)
        dp = C.POINTER(C.c_double)
        lp = C.POINTER(C.c_long)
        L.orc_lap_weights.argtypes = [C.c_int, C.c_double, dp]
        L.orc_laplacian.argtypes = [C.c_int, C.c_int, C.c_int, C.c_double, C.c_int, dp, dp]
        L.orc_veff.argtypes = [C.c_int, C.c_int, C.c_int, C.c_double, C.c_int, dp, dp,
                               C.c_double, dp]
        L.orc_projector_count.argtypes = [C.c_int, C.c_int, C.c_int, C.c_double, C.c_int,
                                          dp, C.c_double, lp]
        L.orc_projector_count.restype = C.c_long
        L.orc_projector_fill.argtypes = [C.c_int, C.c_int, C.c_int, C.c_double, C.c_int,
                                         dp, C.c_double, C.c_double, lp, dp]
        L.orc_apply_H.argtypes = [C.POINTER(_Ham), dp, dp, C.c_int, C.c_long]
        L.orc_apply_H_at.argtypes = [C.POINTER(_Ham), dp, C.c_long, C.c_long, lp,
                                     C.POINTER(C.c_int), dp]
        L.orc_cheb_filter.argtypes = [C.POINTER(_Ham), dp, C.c_int, C.c_long, C.c_int,
                                      C.c_double, C.c_double, C.c_double]
        L.orc_cheb_filter.restype = C.c_int
        L.orc_lanczos_start.argtypes = [C.c_long, C.c_uint64, dp]
        L.orc_lanczos.argtypes = [C.POINTER(_Ham), C.c_int, C.c_uint64, dp, dp]
        L.orc_lanczos.restype = C.c_int
        L.orc_threads.argtypes = [C.c_int]
        L.orc_threads.restype = C.c_int
        _lib = L
    return _lib


def threads(n: int = 0) -> int:
    """Sets the OpenMP thread count of the C loops (n > 0) and returns the count in effect.
    Results do not depend on it."""
    return int(lib().orc_threads(int(n)))


def _dp(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _lp(a: np.ndarray):
    assert a.dtype == np.int64 and a.flags.c_contiguous
    return a.ctypes.data_as(C.POINTER(C.c_long))


# ----------------------------------------------------------------------------------
# Finite-difference weights
# ----------------------------------------------------------------------------------
def lap_weights(no: int = 6, h: float = 1.0) -> np.ndarray:
    """Eq. (weightsLap), Sec. 3.1, in double precision (from the C loops)."""
    w = np.zeros(no + 1)
    lib().orc_lap_weights(no, h, _dp(w))
    return w


def lap_weights_exact(no: int = 6) -> list:
    """Eq. (weightsLap), Sec. 3.1, as exact rationals times 1/h^2 (h = 1)."""
    w0 = -sum(Fraction(1, q * q) for q in range(1, no + 1))
    out = [w0]
    for p in range(1, no + 1):
        ratio = Fraction(1)
        for q in range(1, p + 1):
            ratio *= Fraction(no - q + 1, no + q)
        out.append(Fraction(2 * (-1) ** (p + 1), p * p) * ratio)
    return out


def laplacian(f: np.ndarray, n, h: float, no: int = 6) -> np.ndarray:
    """Eq. (FD:Laplacian) with zero-Dirichlet boundaries, Sec. 3.1. f is a flat
    x-fastest grid function of n = (n0, n1, n2) nodes."""
    n0, n1, n2 = (n, n, n) if np.isscalar(n) else n
    f = np.ascontiguousarray(f, dtype=np.float64).reshape(-1)
    out = np.zeros_like(f)
    lib().orc_laplacian(n0, n1, n2, h, no, _dp(f), _dp(out))
    return out


# ----------------------------------------------------------------------------------
# Potential and projectors
# ----------------------------------------------------------------------------------
def _n3(n):
    return (int(n), int(n), int(n)) if np.isscalar(n) else tuple(int(v) for v in n)


def veff(n, h: float, R: np.ndarray, Z: np.ndarray, rc: float = 1.0) -> np.ndarray:
    """Synthetic local potential sum_J -Z_J erf(r/rc)/r on the grid (flat, x fastest).
    n: nodes per axis (int for a cubic grid, or (n0, n1, n2))."""
    n0, n1, n2 = _n3(n)
    R = np.ascontiguousarray(R, dtype=np.float64).reshape(-1, 3)
    Z = np.ascontiguousarray(Z, dtype=np.float64)
    V = np.zeros(n0 * n1 * n2)
    lib().orc_veff(n0, n1, n2, h, R.shape[0], _dp(R), _dp(Z), rc, _dp(V))
    return V


@dataclasses.dataclass
class Projectors:
    """Support lists of the KB projectors, Eq. (non-localPS:FD), Sec. 3.1."""

    atom_ptr: np.ndarray   # (natoms+1,) int64
    idx: np.ndarray        # (nsup,) int64 linear node index
    chi: np.ndarray        # (nsup, 4) float64: s, px, py, pz


def projectors(n, h: float, R: np.ndarray, sigma: float = 0.8,
               rcut: float = 3.0) -> Projectors:
    n0, n1, n2 = _n3(n)
    R = np.ascontiguousarray(R, dtype=np.float64).reshape(-1, 3)
    na = R.shape[0]
    counts = np.zeros(max(na, 1), dtype=np.int64)
    total = lib().orc_projector_count(n0, n1, n2, h, na, _dp(R), rcut, _lp(counts))
    idx = np.zeros(max(total, 1), dtype=np.int64)
    chi = np.zeros((max(total, 1), 4))
    lib().orc_projector_fill(n0, n1, n2, h, na, _dp(R), sigma, rcut, _lp(idx), _dp(chi))
    ptr = np.zeros(na + 1, dtype=np.int64)
    ptr[1:] = np.cumsum(counts[:na])
    return Projectors(ptr, idx[:total].copy(), chi[:total].copy())


# ----------------------------------------------------------------------------------
# Hamiltonian
# ----------------------------------------------------------------------------------
class Hamiltonian:
    """H = -1/2 kscale L_h + diag(V) + V_nl on an n0 x n1 x n2 grid (Sec. 3.1).

    n: int (cubic grid) or (n0, n1, n2). kscale = 0 keeps only the diagonal part (plus
    V_nl if atoms are given)."""

    def __init__(self, n, h: float, V: np.ndarray, R: Optional[np.ndarray] = None,
                 gamma: Optional[np.ndarray] = None, sigma: float = 0.8,
                 rcut: float = 3.0, no: int = 6, kscale: float = 1.0):
        self.n3 = _n3(n)
        self.n, self.h, self.no, self.kscale = n, h, no, kscale
        self.nd = self.n3[0] * self.n3[1] * self.n3[2]
        self.V = np.ascontiguousarray(V, dtype=np.float64).reshape(-1)
        assert self.V.shape[0] == self.nd
        if R is None or len(R) == 0:
            self.proj = Projectors(np.zeros(1, np.int64), np.zeros(1, np.int64),
                                   np.zeros((1, 4)))
            self.natoms = 0
            self.gamma = np.zeros((1, 4))
        else:
            self.proj = projectors(n, h, R, sigma, rcut)
            self.natoms = int(np.asarray(R).reshape(-1, 3).shape[0])
            self.gamma = np.ascontiguousarray(gamma, dtype=np.float64).reshape(-1, 4)
        self._s = _Ham(*self.n3, h, no, kscale, _dp(self.V), self.natoms,
                       _lp(self.proj.atom_ptr), _lp(self.proj.idx), _dp(self.proj.chi),
                       _dp(self.gamma))

    @classmethod
    def from_cluster(cls, cl, kscale: float = 1.0, V: Optional[np.ndarray] = None):
        """Hamiltonian of a synth.Cluster (V_eff built by the oracle unless given)."""
        if V is None:
            V = veff(cl.n, cl.h, cl.R, cl.Z, cl.rc_erf)
        return cls(cl.n, cl.h, V, cl.R, cl.gamma, cl.sigma, cl.rcut, 6, kscale)

    # -- applications ------------------------------------------------------------
    def apply(self, X: np.ndarray) -> np.ndarray:
        """H X for X of shape (ncols, ld) (column-major Nd x ncols block)."""
        X = np.ascontiguousarray(X, dtype=np.float64)
        if X.ndim == 1:
            X = X.reshape(1, -1)
        ncols, ld = X.shape
        out = np.zeros_like(X)
        lib().orc_apply_H(C.byref(self._s), _dp(X), _dp(out), ncols, ld)
        return out

    def apply_at(self, X: np.ndarray, pts: np.ndarray, cols: np.ndarray) -> np.ndarray:
        """(H X)[p, c] for sampled pairs, each from the definition on its own."""
        X = np.ascontiguousarray(X, dtype=np.float64)
        pts = np.ascontiguousarray(pts, dtype=np.int64)
        cols = np.ascontiguousarray(cols, dtype=np.int32)
        out = np.zeros(pts.shape[0])
        lib().orc_apply_H_at(C.byref(self._s), _dp(X), X.shape[1], pts.shape[0], _lp(pts),
                             cols.ctypes.data_as(C.POINTER(C.c_int)), _dp(out))
        return out

    def dense(self) -> np.ndarray:
        """The Nd x Nd matrix H, column by column from H e_p (small grids only)."""
        nd = self.nd
        Hm = np.zeros((nd, nd))
        blk = 256
        for c0 in range(0, nd, blk):
            c1 = min(nd, c0 + blk)
            E = np.zeros((c1 - c0, nd))
            E[np.arange(c1 - c0), np.arange(c0, c1)] = 1.0
            Hm[:, c0:c1] = self.apply(E).T
        return Hm

    # -- Chebyshev filter ---------------------------------------------------------
    def cheb_filter(self, X: np.ndarray, degree: int, a: float, b: float,
                    a0: float) -> np.ndarray:
        """Algorithm ChebychevFilter, Sec. 3.4 (scaled recurrence; returns a new block)."""
        Y = np.array(X, dtype=np.float64, order="C", copy=True)
        if Y.ndim == 1:
            Y = Y.reshape(1, -1)
        rc = lib().orc_cheb_filter(C.byref(self._s), _dp(Y), Y.shape[0], Y.shape[1],
                                   degree, a, b, a0)
        if rc != 0:
            raise ValueError(f"orc_cheb_filter failed ({rc}): need degree >= 1, a0 < a < b")
        return Y

    # -- Lanczos bounds -----------------------------------------------------------
    def lanczos(self, k: int = 10, seed: int = 0):
        """alpha, beta of k plain Lanczos steps (Sec. 4: 'a few iterations of the Lanczos
        method' for the extremal eigenvalues)."""
        al = np.zeros(k)
        be = np.zeros(k)
        done = lib().orc_lanczos(C.byref(self._s), k, seed & (2 ** 64 - 1), _dp(al), _dp(be))
        if done < 0:
            raise MemoryError("orc_lanczos")
        return al[:done], be[:done]

    def lanczos_bounds(self, k: int = 10, seed: int = 0):
        """(lo, hi, theta_max) from the k x k tridiagonal T_k of k Lanczos steps.

        lo = theta_min (lower end for the filter's scaling). hi is the upper bound of
        the spectrum: max(1.01 theta_max, theta_max + |beta_k s_k|), s_k the last
        component of theta_max's unit eigenvector of T_k. The Ritz-residual term is
        kept because 1.01 theta_max alone can fall below lambda_max after 10 steps,
        and an eigencomponent above the filter interval is amplified, not damped."""
        al, be = self.lanczos(k, seed)
        T = np.diag(al) + np.diag(be[:-1], 1) + np.diag(be[:-1], -1)
        th, S = np.linalg.eigh(T)
        hi = max(1.01 * th[-1], th[-1] + abs(be[-1] * S[-1, -1]))
        return float(th[0]), float(hi), float(th[-1])


def lanczos_start(nd: int, seed: int) -> np.ndarray:
    v = np.zeros(nd)
    lib().orc_lanczos_start(nd, seed & (2 ** 64 - 1), _dp(v))
    return v


# ----------------------------------------------------------------------------------
# Rayleigh-Ritz and the CheFSI loop
# ----------------------------------------------------------------------------------
class NotSPD(ArithmeticError):
    pass


def fix_signs(Q: np.ndarray) -> np.ndarray:
    """Flip each column so its largest-magnitude entry is positive (lowest index on ties)."""
    Q = Q.copy()
    for j in range(Q.shape[1]):
        i = int(np.argmax(np.abs(Q[:, j])))
        if Q[i, j] < 0:
            Q[:, j] = -Q[:, j]
    return Q


def orth_rr(Yf: np.ndarray, HYf: np.ndarray):
    """Projection + generalized eigenproblem + rotation, Sec. 3.4.

    Yf, HYf: (ncols, ld) blocks (rows are columns of the Nd x Ns matrices).
    Returns (X, HX, ritz ascending, residual norms, coefficient matrix Y = L^-T Q)."""
    Y = np.asarray(Yf, dtype=np.float64)
    HY = np.asarray(HYf, dtype=np.float64)
    M = Y @ Y.T                      # M_s = Psi_f^T Psi_f
    Hs = Y @ HY.T                    # H_s = Psi_f^T H Psi_f
    M = 0.5 * (M + M.T)
    Hs = 0.5 * (Hs + Hs.T)
    try:
        L = sla.cholesky(M, lower=True)
    except np.linalg.LinAlgError as e:
        raise NotSPD(str(e)) from e
    # numerically positive definite: every pivot L_jj^2 above 4 n eps M_jj (the squared
    # sine of the angle between column j and the span of the columns before it)
    n = M.shape[0]
    if np.any(np.diag(L) ** 2 <= 4.0 * n * np.finfo(float).eps * np.diag(M)):
        raise NotSPD("Cholesky pivot below 4 n eps of its diagonal entry")
    W = sla.solve_triangular(L, Hs, lower=True)          # L^-1 H_s
    A = sla.solve_triangular(L, W.T, lower=True).T       # L^-1 H_s L^-T
    A = 0.5 * (A + A.T)
    lam, Q = sla.eigh(A)
    Q = fix_signs(Q)
    Cf = sla.solve_triangular(L.T, Q, lower=False)       # L^-T Q
    X = Cf.T @ Y                                         # (Psi_f Y)^T
    HX = Cf.T @ HY
    resid = np.sqrt(np.sum((HX - lam[:, None] * X) ** 2, axis=1))
    return X, HX, lam, resid, Cf


def chefsi_first_bounds(lo: float, hi: float):
    """[a, b, a0] for the first CheFSI iteration from the Lanczos bounds."""
    return [lo + 0.25 * (hi - lo), hi, lo]


def chefsi_next_bounds(bounds, ritz):
    """[a, b, a0] for the next iteration: a = largest, a0 = smallest Ritz value."""
    return [float(np.max(ritz)), bounds[1], float(np.min(ritz))]


def chefsi_step(H: Hamiltonian, X: np.ndarray, degree: int, bounds):
    """One CheFSI iteration (Sec. 3.4): filter, project, solve, rotate."""
    a, b, a0 = bounds
    Yf = H.cheb_filter(X, degree, a, b, a0)
    HYf = H.apply(Yf)
    Xn, HXn, ritz, resid, _ = orth_rr(Yf, HYf)
    return Xn, ritz, resid, chefsi_next_bounds(bounds, ritz)


def chefsi_solve(H: Hamiltonian, X0: np.ndarray, degree: int, iters: int,
                 k_lanczos: int = 10, seed: int = 0, tol: Optional[float] = None):
    """The first-SCF-step regime of Sec. 3.4: repeated CheFSI from a random block on a
    fixed H. Stops after `iters` iterations, or earlier once max residual <= tol."""
    lo, hi, _ = H.lanczos_bounds(k_lanczos, seed)
    bounds = chefsi_first_bounds(lo, hi)
    X = np.array(X0, dtype=np.float64, copy=True)
    hist = []
    ritz = resid = None
    for it in range(iters):
        X, ritz, resid, bounds = chefsi_step(H, X, degree, bounds)
        hist.append((ritz.copy(), resid.copy()))
        if tol is not None and float(np.max(resid)) <= tol:
            break
    return X, ritz, resid, hist, (lo, hi)
