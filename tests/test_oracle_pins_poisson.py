"""Pins of the oracle's electrostatic potential (no GPU).

* Real spherical harmonics: orthonormal under a product Gauss-Legendre x trapezoid
  quadrature of the sphere; Y_00 and the l = 1 functions in closed form.
* Multipole expansion (Eq. phi:BC:discrete): for point charges it converges to the exact
  Coulomb sum at the rate (a/r)^(l_max+1).
* Pseudocharge (Eq. PseudochargeDiscrete): h^3 sum b_J = -Z_J for an atom whose potential
  is Coulombic at the box faces (the charge constraint of Eq. PseudochargeDefinition with
  the sign of the attractive V_J).
* Poisson problem (Eq. FD:PoissonDiscrete + Eq. Phi:correction): for one Gaussian charge
  at the box centre the boundary values are exact up to the charge's erfc tail, and the
  discrete solution equals V_J at every node; an off-centre pair agrees to the l_max = 6
  truncation; CG against a direct sparse solve.
"""
import numpy as np
import pytest
import scipy.sparse as sps
import scipy.sparse.linalg as spla

from oracle import poisson as P
from oracle import lap_weights


def _sphere_quadrature(nt=24, nph=48):
    x, wx = np.polynomial.legendre.leggauss(nt)
    ph = np.arange(nph) * 2 * np.pi / nph
    T, PH = np.meshgrid(np.arccos(x), ph, indexing="ij")
    W = np.outer(wx, np.full(nph, 2 * np.pi / nph))
    v = np.stack([np.sin(T) * np.cos(PH), np.sin(T) * np.sin(PH), np.cos(T)], -1).reshape(-1, 3)
    return v, W.reshape(-1)


def test_real_harmonics_orthonormal_and_closed_forms():
    v, w = _sphere_quadrature()
    Y = P.real_harmonics(6, v)
    flat = [Y[l][m] for l in range(7) for m in range(2 * l + 1)]
    G = np.array([[np.sum(w * a * b) for b in flat] for a in flat])
    assert np.max(np.abs(G - np.eye(len(flat)))) <= 1e-12
    assert np.allclose(Y[0][0], 1 / np.sqrt(4 * np.pi), atol=1e-15)
    c1 = np.sqrt(3 / (4 * np.pi))
    # the three l = 1 functions are +-c1 times y, z, x (m = -1, 0, 1)
    for m, comp in ((0, 1), (1, 2), (2, 0)):
        assert np.allclose(np.abs(Y[1][m]), c1 * np.abs(v[:, comp]), atol=1e-13)


def test_multipole_expansion_of_point_charges():
    rng = np.random.default_rng(2)
    c = np.zeros(3)
    src = rng.uniform(-1, 1, (5, 3))
    q = rng.uniform(-1, 1, 5)
    # moments of the point charges directly
    Y = P.real_harmonics(6, src)
    r = np.linalg.norm(src, axis=1)
    Q = [[np.sum(q * r ** l * Y[l][m]) for m in range(2 * l + 1)] for l in range(7)]
    errs = []
    for R0 in (6.0, 12.0):
        d = rng.normal(size=(50, 3))
        pts = R0 * d / np.linalg.norm(d, axis=1, keepdims=True)
        exact = np.array([np.sum(q / np.linalg.norm(p - src, axis=1)) for p in pts])
        got = P.multipole_potential(Q, pts, c)
        errs.append(np.max(np.abs(got - exact)))
    assert errs[0] <= 2e-5
    assert errs[0] / errs[1] >= 2 ** 7 * 0.5       # (a/r)^7 over r -> 2r, r^-1 prefactor


def test_pseudocharge_integrates_to_minus_z():
    n, h = 40, 0.3
    c = P.box_centre(n, h)
    R = np.array([c + [0.5, -0.3, 0.2], c - [0.9, 0.4, -0.6]])
    Z = np.array([3.0, 1.0])
    b = P.pseudocharge(n, h, R, Z, 1.0)
    assert abs(h ** 3 * b.sum() + 4.0) <= 1e-10
    # it is -(1/4 pi) L_h V inside the grid
    V = P.local_potential(P.node_coords(n, h), R, Z, 1.0)
    from oracle import laplacian
    Lv = laplacian(V, n, h).reshape(n, n, n)[6:-6, 6:-6, 6:-6]
    assert np.allclose(b.reshape(n, n, n)[6:-6, 6:-6, 6:-6], -Lv / (4 * np.pi), rtol=0,
                       atol=1e-12)


def test_centred_gaussian_charge_gives_its_potential_exactly():
    n, h = 40, 0.3
    c = P.box_centre(n, h)
    R, Z = c.reshape(1, 3), np.array([3.0])
    phi, it, rel = P.poisson_solve(np.zeros(n ** 3), n, h, R, Z, 1.0, tol=1e-13)
    V = P.local_potential(P.node_coords(n, h), R, Z, 1.0)
    assert rel <= 1e-13
    assert np.max(np.abs(phi - V)) <= 1e-10


def test_off_centre_pair_within_multipole_truncation():
    n, h = 40, 0.3
    c = P.box_centre(n, h)
    R = np.array([c + [1.1, -0.4, 0.3], c - [0.8, 0.9, -0.5]])
    Z = np.array([2.0, 1.0])
    phi, _, _ = P.poisson_solve(np.zeros(n ** 3), n, h, R, Z, 1.0, tol=1e-12)
    V = P.local_potential(P.node_coords(n, h), R, Z, 1.0)
    assert np.max(np.abs(phi - V)) <= 1e-5
    # with zero boundary values instead (d = 0) the error is the full monopole tail
    f = P.pseudocharge(n, h, R, Z, 1.0)
    diag = -6 * lap_weights(6, h)[0] / (4 * np.pi)
    phi0, _, _ = P.cg_solve(lambda v: P.poisson_apply(v, n, h), f, diag, 1e-12)
    assert np.max(np.abs(phi0 - V)) > 0.1


def test_charge_correction_structure():
    n, h = 20, 0.4
    Q = P.multipole_moments(np.zeros(n ** 3), n, h)
    assert np.all(P.charge_correction(n, h, Q) == 0)
    rng = np.random.default_rng(1)
    f = rng.uniform(0, 1, n ** 3)
    d = P.charge_correction(n, h, P.multipole_moments(f, n, h)).reshape(n, n, n)
    assert np.all(d[6:-6, 6:-6, 6:-6] == 0)         # only nodes within n_o of a face
    assert np.all(d[0] != 0) and np.all(d[:, :, -1] != 0)


def test_cg_matches_direct_solve():
    n, h = 11, 0.5
    nd = n ** 3
    rng = np.random.default_rng(4)
    f = rng.standard_normal(nd)
    A = np.zeros((nd, nd))
    for j in range(nd):
        e = np.zeros(nd)
        e[j] = 1.0
        A[:, j] = P.poisson_apply(e, n, h)
    assert np.allclose(A, A.T, atol=1e-12)
    x_ref = spla.spsolve(sps.csr_matrix(A), f)
    diag = -6 * lap_weights(6, h)[0] / (4 * np.pi)
    x, it, rel = P.cg_solve(lambda v: P.poisson_apply(v, n, h), f, diag, 1e-13)
    assert rel <= 1e-13
    assert np.max(np.abs(x - x_ref)) <= 1e-10 * np.max(np.abs(x_ref))
