"""FP64 CPU oracle for the steps that follow the subspace rotation (Sec. 3.4, Sec. 3.6).

TEST INFRASTRUCTURE. Only the test suite, the package smoke check and the benchmark's
CPU-baseline leg may import this module. It shares no code with the CUDA library and
never loads it.

* Fermi level, Eq. (FermiEnergyConstraintFormulation): the root lambda_f of
  2 sum_n g_n = N_e with g_n = 1 / (1 + exp((lambda_n - lambda_f) / (k_B T))), found with
  Brent's method as Sec. 4 states (written here from Brent's published algorithm:
  inverse quadratic interpolation or a secant step where it is safe, bisection
  otherwise).
* Electron density, the equation after Eq. (OrbitalTransformation):
  rho = (2 / h^3) sum_n g_n psi_n^2, psi_n the Euclidean-normalised columns of Psi.
* Finite-difference gradient, Eq. (gradient:approximate), zero-Dirichlet (Sec. 3.1).
* Non-local force, Eq. (NonlocForce:Discrete) with Y and W of Eq. (NonLocForce:U:W),
  in the steps of Algorithm non-localForceCalculation: over each atom's projector
  support, Y_Jnlm = h^3 sum psi chi and W_Jnlm = h^3 sum (grad_h psi) chi, then
  f_J = -4 sum_n g_n sum_lm gamma_Jl Y_Jnlm W_Jnlm.

Reading of the force's normalisation. The density formula holds for Euclidean-normalised
columns x_n (h^3 sum rho = 2 sum g_n). The force formula is minus the derivative of the
non-local energy E_nl = 2 sum_n g_n x_n^T V_nl x_n with respect to R_J only for
psi_n = x_n / h^(3/2) (h^3 sum psi^2 = 1, the continuum normalisation): with x_n in
Y and W it carries an extra factor h^3. The oracle therefore forms Y and W from x_n and
returns f_J = -(4 / h^3) sum_n g_n sum_lm gamma_Jl Y_Jnlm W_Jnlm, which is the paper's
formula for psi_n = x_n / h^(3/2). tests/test_oracle_pins.py checks it against central
differences of E_nl in the atom positions.
"""
from __future__ import annotations

from fractions import Fraction
from math import factorial

import numpy as np

from .oracle import Hamiltonian, _n3

_EPS = np.finfo(np.float64).eps


# ----------------------------------------------------------------------------------
# Occupations and the Fermi level
# ----------------------------------------------------------------------------------
def occupations(lam: np.ndarray, lam_f: float, kT: float) -> np.ndarray:
    """g_n of Eq. (FermiEnergyConstraintFormulation). exp overflow gives g = 0."""
    t = (np.asarray(lam, dtype=np.float64) - lam_f) / kT
    with np.errstate(over="ignore"):
        return 1.0 / (1.0 + np.exp(t))


def electron_excess(lam: np.ndarray, lam_f: float, nelec: float, kT: float) -> float:
    """2 sum_n g_n - N_e, increasing in lam_f."""
    return float(2.0 * np.sum(occupations(lam, lam_f, kT)) - nelec)


def brent_root(f, a: float, b: float, xtol: float = 0.0, maxit: int = 500) -> float:
    """A zero of f in [a, b] (f(a) f(b) <= 0) by Brent's method. Each step keeps b as the
    best estimate and c on the other side of the root; it tries inverse quadratic
    interpolation through (a, b, c) (a secant step when only two points differ), and
    falls back to bisection when the interpolated point leaves the safe part of [b, c]
    or the steps stop shrinking. Ends when half the bracket is below
    2 eps |b| + xtol / 2."""
    fa, fb = f(a), f(b)
    if fa == 0.0:
        return a
    if fb == 0.0:
        return b
    if np.sign(fa) == np.sign(fb):
        raise ValueError("root not bracketed")
    c, fc = a, fa
    step = prev = b - a
    for _ in range(maxit):
        if np.sign(fb) == np.sign(fc):
            c, fc = a, fa
            step = prev = b - a
        if abs(fc) < abs(fb):
            a, fa = b, fb
            b, fb = c, fc
            c, fc = a, fa
        tol = 2.0 * _EPS * abs(b) + 0.5 * xtol
        half = 0.5 * (c - b)
        if abs(half) <= tol or fb == 0.0:
            return b
        bisect = True
        if abs(prev) >= tol and abs(fa) > abs(fb):
            s = fb / fa
            if a == c:
                num, den = 2.0 * half * s, 1.0 - s
            else:
                qa, rb = fa / fc, fb / fc
                num = s * (2.0 * half * qa * (qa - rb) - (b - a) * (rb - 1.0))
                den = (qa - 1.0) * (rb - 1.0) * (s - 1.0)
            if num > 0.0:
                den = -den
            else:
                num = -num
            if 2.0 * num < min(3.0 * half * den - abs(tol * den), abs(prev * den)):
                prev, step = step, num / den
                bisect = False
        if bisect:
            step = prev = half
        a, fa = b, fb
        b = b + (step if abs(step) > tol else (tol if half > 0 else -tol))
        fb = f(b)
    raise ArithmeticError("Brent's method did not converge")


def fermi_level(lam: np.ndarray, nelec: float, kT: float) -> float:
    """lambda_f with 2 sum_n g_n = N_e (0 < N_e < 2 Ns, kT > 0)."""
    lam = np.asarray(lam, dtype=np.float64)
    ns = lam.shape[0]
    if not (kT > 0.0) or not (0.0 < nelec < 2.0 * ns):
        raise ValueError("need kT > 0 and 0 < N_e < 2 Ns")
    f = lambda mu: electron_excess(lam, mu, nelec, kT)  # noqa: E731
    lo, hi = float(lam.min()) - 1.0, float(lam.max()) + 1.0
    width = hi - lo
    while f(lo) > 0.0:
        lo -= width
        width *= 2.0
    width = hi - lo
    while f(hi) < 0.0:
        hi += width
        width *= 2.0
    return brent_root(f, lo, hi)


# ----------------------------------------------------------------------------------
# Density
# ----------------------------------------------------------------------------------
def density(X: np.ndarray, g: np.ndarray, h: float) -> np.ndarray:
    """rho = (2 / h^3) sum_n g_n x_n^2 for X of shape (ncols, ld): Nd values (the first
    Nd rows of each column are used; pass nd through X[:, :nd] for padded blocks)."""
    X = np.asarray(X, dtype=np.float64)
    g = np.asarray(g, dtype=np.float64)
    rho = np.zeros(X.shape[1])
    for n in range(X.shape[0]):
        rho += g[n] * X[n] * X[n]
    return (2.0 / h ** 3) * rho


# ----------------------------------------------------------------------------------
# Finite-difference gradient
# ----------------------------------------------------------------------------------
def grad_weights_exact(no: int = 6) -> list:
    """The weights of Eq. (gradient:approximate) as exact rationals times 1/h (h = 1):
    w~_p = (-1)^(p+1) / p * (n_o!)^2 / ((n_o - p)! (n_o + p)!)."""
    out = []
    for p in range(1, no + 1):
        out.append(Fraction((-1) ** (p + 1), p) *
                   Fraction(factorial(no) ** 2, factorial(no - p) * factorial(no + p)))
    return out


def grad_weights(no: int = 6, h: float = 1.0) -> np.ndarray:
    """w~_1 .. w~_no of Eq. (gradient:approximate) in double precision (index 0 unused)."""
    w = np.zeros(no + 1)
    for p, v in enumerate(grad_weights_exact(no), start=1):
        w[p] = float(v) / h
    return w


def gradient(f: np.ndarray, n, h: float, no: int = 6) -> np.ndarray:
    """Eq. (gradient:approximate) with f = 0 outside the grid: returns (3, Nd), the x, y
    and z components, for a flat x-fastest grid function f."""
    n0, n1, n2 = _n3(n)
    F = np.asarray(f, dtype=np.float64).reshape(n2, n1, n0)
    w = grad_weights(no, h)
    out = np.zeros((3, n2, n1, n0))
    for axis, comp in ((2, 0), (1, 1), (0, 2)):
        m = F.shape[axis]
        for p in range(1, no + 1):
            if p >= m:
                continue
            plus = np.zeros_like(F)   # f(i + p)
            minus = np.zeros_like(F)  # f(i - p)
            sl_dst = [slice(None)] * 3
            sl_src = [slice(None)] * 3
            sl_dst[axis], sl_src[axis] = slice(0, m - p), slice(p, m)
            plus[tuple(sl_dst)] = F[tuple(sl_src)]
            sl_dst[axis], sl_src[axis] = slice(p, m), slice(0, m - p)
            minus[tuple(sl_dst)] = F[tuple(sl_src)]
            out[comp] += w[p] * (plus - minus)
    return out.reshape(3, -1)


def gradient_at(f: np.ndarray, n, h: float, pts: np.ndarray, no: int = 6) -> np.ndarray:
    """Eq. (gradient:approximate) at the nodes pts only (same result as gradient()[:, pts]
    up to the order of the sums): returns (3, len(pts))."""
    n0, n1, n2 = _n3(n)
    f = np.asarray(f, dtype=np.float64).reshape(-1)
    pts = np.asarray(pts, dtype=np.int64)
    i, j, k = pts % n0, (pts // n0) % n1, pts // (n0 * n1)
    w = grad_weights(no, h)
    out = np.zeros((3, pts.shape[0]))
    for comp, (c, m, stride) in enumerate(((i, n0, 1), (j, n1, n0), (k, n2, n0 * n1))):
        for p in range(1, no + 1):
            up = np.where(c + p < m, f[np.minimum(pts + p * stride, f.shape[0] - 1)], 0.0)
            dn = np.where(c - p >= 0, f[np.maximum(pts - p * stride, 0)], 0.0)
            out[comp] += w[p] * (up - dn)
    return out


# ----------------------------------------------------------------------------------
# Non-local force
# ----------------------------------------------------------------------------------
def nonlocal_energy(H: Hamiltonian, X: np.ndarray, g: np.ndarray) -> float:
    """E_nl = 2 sum_n g_n x_n^T V_nl x_n with V_nl of Eq. (non-localPS:FD)."""
    X = np.asarray(X, dtype=np.float64)
    P = H.proj
    e = 0.0
    for J in range(H.natoms):
        a, b = int(P.atom_ptr[J]), int(P.atom_ptr[J + 1])
        chi = P.chi[a:b]                      # (nsup, 4)
        xs = X[:, P.idx[a:b]]                 # (ncols, nsup)
        c = xs @ chi                          # chi^T x_n, (ncols, 4)
        e += 2.0 * H.h ** 3 * float(np.sum(g[:, None] * H.gamma[J][None, :] * c * c))
    return e


def nonlocal_projections(H: Hamiltonian, X: np.ndarray):
    """Y (natoms, ncols, 4) and W (natoms, ncols, 3, 4) of Eq. (NonLocForce:U:W) from the
    Euclidean columns x_n, over each atom's support (Algorithm non-localForceCalculation)."""
    X = np.asarray(X, dtype=np.float64)
    P = H.proj
    h3 = H.h ** 3
    ncols = X.shape[0]
    Y = np.zeros((H.natoms, ncols, 4))
    W = np.zeros((H.natoms, ncols, 3, 4))
    for J in range(H.natoms):
        a, b = int(P.atom_ptr[J]), int(P.atom_ptr[J + 1])
        pts = P.idx[a:b]
        chi = P.chi[a:b]
        for n in range(ncols):
            x = X[n, :H.nd]
            Y[J, n] = h3 * (x[pts] @ chi)
            gr = gradient_at(x, H.n3, H.h, pts, H.no)   # (3, nsup)
            W[J, n] = h3 * (gr @ chi)
    return Y, W


def nonlocal_force(H: Hamiltonian, X: np.ndarray, g: np.ndarray) -> np.ndarray:
    """f_J (natoms, 3) = -(4 / h^3) sum_n g_n sum_lm gamma_Jl Y_Jnlm W_Jnlm (the paper's
    Eq. (NonlocForce:Discrete) for psi_n = x_n / h^(3/2); see the module docstring)."""
    g = np.asarray(g, dtype=np.float64)
    Y, W = nonlocal_projections(H, X)
    f = np.zeros((H.natoms, 3))
    for J in range(H.natoms):
        # sum over n and lm of g_n gamma_Jl Y_Jnlm W_Jnlm,d
        f[J] = -(4.0 / H.h ** 3) * np.einsum("n,l,nl,ndl->d", g, H.gamma[J], Y[J], W[J])
    return f
