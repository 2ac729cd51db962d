"""FP64 CPU oracle for the electrostatic potential (Sec. 3.3, Sec. 4).

TEST INFRASTRUCTURE. Only the test suite, the package smoke check and the benchmark's
CPU-baseline leg may import this module. It shares no code with the CUDA library and
never loads it.

Steps, in the paper's order:
* pseudocharges, Eq. (PseudochargeDiscrete) and Algorithm PseudochargeCalculation:
  b = sum_J b_J, b_J = -(1/4 pi) L_h V_J, with V_J evaluated at the grid nodes and at the
  n_o nodes beyond each face (the FD Laplacian of Eq. FD:Laplacian reaches them);
* multipole moments Q_lm = h^3 sum |x|^l Y_lm(x/|x|) (rho + b), the equation after
  Eq. (phi:BC:discrete), real spherical harmonics up to l_max = 6 (Sec. 4);
* boundary values phi(x) = sum_lm 4 pi / ((2l+1) |x|^(l+1)) Y_lm Q_lm, Eq. (phi:BC:discrete),
  at the nodes outside the grid that the stencil of a grid node reaches;
* the charge correction d of Eq. (Phi:correction) from those values;
* the linear system -(1/4 pi) L_h phi = rho + b - d of Eq. (FD:PoissonDiscrete), zero
  Dirichlet, by conjugate gradients with a Jacobi preconditioner (Sec. 4).

Readings (where the paper is silent or at odds with itself):
* sign of the pseudocharge: Eq. (PseudochargeDefinition) states int b_J = Z_J while
  V_J is the attractive local pseudopotential; with b_J = -(1/4 pi) lap V_J and V_J ~
  -Z_J / r, int b_J = -Z_J. The definition b_J = -(1/4 pi) lap V_J is kept, so b_J carries
  the nuclear charge in the sign convention of rho + b (electrons positive);
* V_J is the configurations' synthetic local potential -Z_J erf(r/r_c)/r; its pseudocharge
  decays as a Gaussian, so it is kept on the whole grid (no truncation radius r_b);
* |x| is measured from the centre of the box, ((n_d - 1) h / 2 per axis);
* the block-Jacobi preconditioner of Sec. 4 acts on the processors' blocks of the
  domain; on one device it is read as the point-Jacobi (diagonal) preconditioner;
* CG starts from phi = 0 and stops at ||r|| <= tol ||rhs||.
"""
from __future__ import annotations

import numpy as np
from scipy.special import erf, sph_harm_y

from .oracle import _n3, lap_weights, laplacian

FOUR_PI = 4.0 * np.pi


def box_centre(n, h: float) -> np.ndarray:
    n0, n1, n2 = _n3(n)
    return np.array([(n0 - 1) * h / 2, (n1 - 1) * h / 2, (n2 - 1) * h / 2])


def local_potential(pts: np.ndarray, R: np.ndarray, Z: np.ndarray, rc: float) -> np.ndarray:
    """sum_J -Z_J erf(r/rc)/r at the points pts (m, 3); the r -> 0 limit is -2 Z/(sqrt(pi) rc)."""
    V = np.zeros(pts.shape[0])
    for J in range(R.shape[0]):
        r = np.sqrt(np.sum((pts - R[J]) ** 2, axis=1))
        small = r < 1e-12
        rs = np.where(small, 1.0, r)
        V += np.where(small, -2.0 * Z[J] / (np.sqrt(np.pi) * rc), -Z[J] * erf(rs / rc) / rs)
    return V


def pseudocharge(n, h: float, R: np.ndarray, Z: np.ndarray, rc: float = 1.0,
                 no: int = 6) -> np.ndarray:
    """b = -(1/4 pi) L_h (sum_J V_J) at the grid nodes, the stencil reaching V_J at the
    n_o layers beyond each face (Algorithm PseudochargeCalculation)."""
    n0, n1, n2 = _n3(n)
    R = np.asarray(R, dtype=np.float64).reshape(-1, 3)
    Z = np.asarray(Z, dtype=np.float64)
    e0, e1, e2 = n0 + 2 * no, n1 + 2 * no, n2 + 2 * no
    k, j, i = np.meshgrid(np.arange(e2) - no, np.arange(e1) - no, np.arange(e0) - no,
                          indexing="ij")
    pts = np.stack([i.reshape(-1) * h, j.reshape(-1) * h, k.reshape(-1) * h], axis=1)
    Ve = local_potential(pts, R, Z, rc).reshape(e2, e1, e0)
    w = lap_weights(no, h)
    core = (slice(no, no + n2), slice(no, no + n1), slice(no, no + n0))
    # Eq. (FD:Laplacian): the p = 0 term counts the node six times
    L = 6.0 * w[0] * Ve[core]
    for p in range(1, no + 1):
        L = L + w[p] * (Ve[no + p:no + p + n2, no:no + n1, no:no + n0] +
                        Ve[no - p:no - p + n2, no:no + n1, no:no + n0] +
                        Ve[no:no + n2, no + p:no + p + n1, no:no + n0] +
                        Ve[no:no + n2, no - p:no - p + n1, no:no + n0] +
                        Ve[no:no + n2, no:no + n1, no + p:no + p + n0] +
                        Ve[no:no + n2, no:no + n1, no - p:no - p + n0])
    return (-L / FOUR_PI).reshape(-1)


def real_harmonics(lmax: int, v: np.ndarray) -> list:
    """Real orthonormal spherical harmonics Y_lm(v/|v|) for l <= lmax, m = -l..l, from
    scipy's complex ones: m > 0: sqrt(2) (-1)^m Re Y_l^m, m < 0: sqrt(2) (-1)^m Im Y_l^|m|.
    v: (npts, 3), nonzero rows. Returns [l][m + l] arrays."""
    r = np.sqrt(np.sum(v * v, axis=1))
    theta = np.arccos(np.clip(v[:, 2] / r, -1.0, 1.0))
    phi = np.arctan2(v[:, 1], v[:, 0])
    out = []
    for l in range(lmax + 1):
        row = []
        for m in range(-l, l + 1):
            y = sph_harm_y(l, abs(m), theta, phi)
            if m == 0:
                row.append(np.real(y))
            elif m > 0:
                row.append(np.sqrt(2.0) * (-1) ** m * np.real(y))
            else:
                row.append(np.sqrt(2.0) * (-1) ** m * np.imag(y))
        out.append(row)
    return out


def node_coords(n, h: float) -> np.ndarray:
    n0, n1, n2 = _n3(n)
    k, j, i = np.meshgrid(np.arange(n2), np.arange(n1), np.arange(n0), indexing="ij")
    return np.stack([i.reshape(-1) * h, j.reshape(-1) * h, k.reshape(-1) * h], axis=1)


def multipole_moments(f: np.ndarray, n, h: float, lmax: int = 6) -> list:
    """Q_lm = h^3 sum |x|^l Y_lm(x/|x|) f over the grid, x from the box centre (a node at
    the centre contributes to Q_00 only)."""
    x = node_coords(n, h) - box_centre(n, h)
    r = np.sqrt(np.sum(x * x, axis=1))
    f = np.asarray(f, dtype=np.float64).reshape(-1)
    nz = r > 0
    Y = real_harmonics(lmax, x[nz])
    Q = []
    for l in range(lmax + 1):
        row = []
        for m in range(2 * l + 1):
            q = h ** 3 * np.sum(r[nz] ** l * Y[l][m] * f[nz])
            if l == 0:
                q += h ** 3 * np.sum(f[~nz]) / np.sqrt(FOUR_PI)
            row.append(q)
        Q.append(row)
    return Q


def multipole_potential(Q: list, pts: np.ndarray, centre: np.ndarray) -> np.ndarray:
    """Eq. (phi:BC:discrete) at the points pts (m, 3), all away from the centre."""
    lmax = len(Q) - 1
    x = pts - centre
    r = np.sqrt(np.sum(x * x, axis=1))
    Y = real_harmonics(lmax, x)
    phi = np.zeros(pts.shape[0])
    for l in range(lmax + 1):
        for m in range(2 * l + 1):
            phi += FOUR_PI / ((2 * l + 1) * r ** (l + 1)) * Y[l][m] * Q[l][m]
    return phi


def charge_correction(n, h: float, Q: list, no: int = 6) -> np.ndarray:
    """d of Eq. (Phi:correction): d = -(1/4 pi) sum_p w_p sum over the six neighbours at
    distance p that lie outside the grid of phi there (phi from Eq. phi:BC:discrete)."""
    n0, n1, n2 = _n3(n)
    dims = (n0, n1, n2)
    w = lap_weights(no, h)
    c = box_centre(n, h)
    d = np.zeros(n0 * n1 * n2)
    X = node_coords(n, h)
    idx = np.arange(n0 * n1 * n2)
    ijk = np.stack([idx % n0, (idx // n0) % n1, idx // (n0 * n1)], axis=1)
    for axis in range(3):
        for sgn in (1, -1):
            for p in range(1, no + 1):
                tgt = ijk[:, axis] + sgn * p
                out = (tgt < 0) | (tgt >= dims[axis])
                if not np.any(out):
                    continue
                pts = X[out].copy()
                pts[:, axis] += sgn * p * h
                d[out] += w[p] * multipole_potential(Q, pts, c)
    return -d / FOUR_PI


def poisson_apply(phi: np.ndarray, n, h: float, no: int = 6) -> np.ndarray:
    """-(1/4 pi) L_h phi, zero Dirichlet (Eq. FD:PoissonDiscrete's operator)."""
    return -laplacian(phi, n, h, no) / FOUR_PI


def poisson_rhs(rho: np.ndarray, n, h: float, R, Z, rc: float = 1.0, no: int = 6,
                lmax: int = 6):
    """rho + b - d and the pieces: (rhs, b, d, Q)."""
    b = pseudocharge(n, h, R, Z, rc, no)
    Q = multipole_moments(np.asarray(rho, dtype=np.float64) + b, n, h, lmax)
    d = charge_correction(n, h, Q, no)
    return np.asarray(rho, dtype=np.float64) + b - d, b, d, Q


def cg_solve(apply, f: np.ndarray, diag: float, tol: float = 1e-10, maxit: int = 2000):
    """Preconditioned CG for A x = f (A SPD) with z = r / diag, from x = 0; stops at
    ||r||_2 <= tol ||f||_2. Returns (x, iterations, ||r|| / ||f||)."""
    x = np.zeros_like(f)
    r = f.copy()
    nf = np.linalg.norm(f)
    if nf == 0.0:
        return x, 0, 0.0
    z = r / diag
    p = z.copy()
    rz = r @ z
    for it in range(1, maxit + 1):
        Ap = apply(p)
        alpha = rz / (p @ Ap)
        x += alpha * p
        r -= alpha * Ap
        rel = np.linalg.norm(r) / nf
        if rel <= tol:
            return x, it, rel
        z = r / diag
        rz_new = r @ z
        p = z + (rz_new / rz) * p
        rz = rz_new
    return x, maxit, np.linalg.norm(r) / nf


def poisson_solve(rho: np.ndarray, n, h: float, R, Z, rc: float = 1.0, tol: float = 1e-10,
                  maxit: int = 4000, no: int = 6):
    """phi on the grid from Eq. (FD:PoissonDiscrete): (phi, iterations, relative residual)."""
    f, _, _, _ = poisson_rhs(rho, n, h, R, Z, rc, no)
    diag = -6.0 * lap_weights(no, h)[0] / FOUR_PI
    return cg_solve(lambda v: poisson_apply(v, n, h, no), f, diag, tol, maxit)
