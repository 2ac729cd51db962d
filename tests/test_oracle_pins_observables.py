"""Pins of the oracle's Fermi level, density, FD gradient and non-local force (no GPU).

* FD gradient weights (Eq. gradient:approximate): the exact rationals match the stored
  table and satisfy the Taylor moment conditions of a centred first-derivative stencil
  of order 2 n_o; the stencil is exact on polynomials of degree <= 12 per axis at
  interior nodes, not on degree 13, and its error falls as h^12; with zero-Dirichlet
  values it is antisymmetric (summation by parts).
* Fermi level (Eq. FermiEnergyConstraintFormulation): closed forms for one level and for
  a symmetric pair, and the root scipy's brentq finds on random spectra.
* Density: h^3 sum rho = 2 sum g_n ||x_n||^2, and with equal occupations it is invariant
  under an orthogonal mixing of the columns.
* Non-local force (Eq. NonlocForce:Discrete): equal to minus the central-difference
  derivative of E_nl = 2 sum g_n x_n^T V_nl x_n in each atom coordinate, projectors
  re-sampled at the displaced positions.
"""
import math
import os
from fractions import Fraction

import numpy as np
import pytest
from scipy.optimize import brentq

import oracle
from oracle import observables as OB

HERE = os.path.dirname(os.path.abspath(__file__))


# ------------------------------------------------------------------------------------
# FD gradient
# ------------------------------------------------------------------------------------
def test_grad_weights_match_golden_table():
    rows = []
    with open(os.path.join(HERE, "golden", "fd_grad_weights_no6.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            p, a, b = (int(v) for v in line.split())
            rows.append((p, Fraction(a, b)))
    w = OB.grad_weights_exact(6)
    assert [p for p, _ in rows] == list(range(1, 7))
    assert [x for _, x in rows] == w


@pytest.mark.parametrize("no", [1, 2, 3, 6])
def test_grad_weights_moment_conditions(no):
    # f'(0) from sum_p w_p (f(p) - f(-p)): odd moments 2 sum_p w_p p^(2k+1) = [k == 0]
    w = OB.grad_weights_exact(no)
    for k in range(no):
        m = 2 * sum(wp * Fraction(p) ** (2 * k + 1) for p, wp in enumerate(w, start=1))
        assert m == (1 if k == 0 else 0), (no, k, m)
    # the next odd moment does not vanish: order exactly 2 n_o
    m = 2 * sum(wp * Fraction(p) ** (2 * no + 1) for p, wp in enumerate(w, start=1))
    assert m != 0
    if no == 1:
        assert w == [Fraction(1, 2)]  # the plain central difference (f(x+h) - f(x-h)) / 2h


def test_gradient_exact_on_polynomials_interior():
    n = (30, 28, 27)
    h = 0.5
    i = np.arange(n[0]) * h - 7.0
    j = np.arange(n[1]) * h - 6.5
    k = np.arange(n[2]) * h - 6.0
    Z, Yg, X = np.meshgrid(k, j, i, indexing="ij")
    inner = (slice(6, n[2] - 6), slice(6, n[1] - 6), slice(6, n[0] - 6))
    for a, b, c in [(12, 0, 0), (0, 12, 1), (3, 1, 12), (7, 5, 2), (1, 1, 1)]:
        f = (X / 7) ** a * (Yg / 7) ** b * (Z / 7) ** c
        g = OB.gradient(f.reshape(-1), n, h).reshape(3, n[2], n[1], n[0])
        ex = [a * (X / 7) ** max(a - 1, 0) / 7 * (Yg / 7) ** b * (Z / 7) ** c,
              b * (X / 7) ** a * (Yg / 7) ** max(b - 1, 0) / 7 * (Z / 7) ** c,
              c * (X / 7) ** a * (Yg / 7) ** b * (Z / 7) ** max(c - 1, 0) / 7]
        for d in range(3):
            err = np.max(np.abs(g[d][inner] - ex[d][inner]))
            assert err <= 1e-10 * max(1.0, np.max(np.abs(ex[d][inner]))), (a, b, c, d, err)
    # degree 13 is not differentiated exactly
    f = (X / 7) ** 13
    g = OB.gradient(f.reshape(-1), n, h).reshape(3, n[2], n[1], n[0])
    err13 = np.max(np.abs(g[0][inner] - (13 * (X / 7) ** 12 / 7)[inner]))
    assert err13 > 1e-10, err13  # (about 1.3e-9 here, above the bound the exact cases meet)


def test_gradient_order_twelve():
    # d/dx sin(x) on refined grids: error ratio 2^12 under h -> h/2
    errs = []
    for h in (0.4, 0.2):
        n = (int(round(12.0 / h)), 13, 13)
        x = np.arange(n[0]) * h
        f = np.broadcast_to(np.sin(x)[None, None, :], (n[2], n[1], n[0])).copy()
        g = OB.gradient(f.reshape(-1), n, h).reshape(3, n[2], n[1], n[0])[0, 6, 6]
        sl = slice(6, n[0] - 6)
        errs.append(np.max(np.abs(g[sl] - np.cos(x[sl]))))
    rate = math.log2(errs[0] / errs[1])
    assert 11.0 < rate < 13.0, (errs, rate)


def test_gradient_summation_by_parts_and_gradient_at():
    rng = np.random.default_rng(3)
    n = (17, 11, 9)
    nd = n[0] * n[1] * n[2]
    f, g = rng.standard_normal(nd), rng.standard_normal(nd)
    Gf, Gg = OB.gradient(f, n, 0.3), OB.gradient(g, n, 0.3)
    for d in range(3):
        lhs, rhs = g @ Gf[d], -(f @ Gg[d])
        assert abs(lhs - rhs) <= 1e-12 * (np.abs(g) @ np.abs(Gf[d])), d
    pts = rng.choice(nd, 200, replace=False)
    assert np.allclose(OB.gradient_at(f, n, 0.3, pts), Gf[:, pts], rtol=0, atol=1e-12)


# ------------------------------------------------------------------------------------
# Fermi level
# ------------------------------------------------------------------------------------
def test_fermi_level_single_level_closed_form():
    lam = np.array([-0.37])
    for ne, kT in [(0.5, 1e-3), (1.0, 1e-3), (1.9, 2e-2)]:
        mu = OB.fermi_level(lam, ne, kT)
        # g = N_e / 2 = 1 / (1 + exp((lam - mu) / kT))
        assert abs(mu - (lam[0] - kT * math.log(2.0 / ne - 1.0))) <= 1e-13


def test_fermi_level_symmetric_pair_is_the_midpoint():
    for d in (1e-4, 0.05, 3.0):
        lam = np.array([0.2 - d, 0.2 + d])
        assert abs(OB.fermi_level(lam, 2.0, 1e-3) - 0.2) <= 1e-13


def test_fermi_level_matches_library_root_on_random_spectra():
    rng = np.random.default_rng(11)
    for trial in range(20):
        ns = int(rng.integers(2, 300))
        lam = np.sort(rng.uniform(-12.0, 3.0, ns))
        ne = float(rng.uniform(0.2, 2 * ns - 0.2))
        kT = float(rng.choice([1e-3, 1e-2, 1e-4]))
        mu = OB.fermi_level(lam, ne, kT)
        f = lambda m: 2.0 * np.sum(1.0 / (1.0 + np.exp(np.minimum((lam - m) / kT, 700.0)))) - ne  # noqa: E731
        ref = brentq(f, lam[0] - 5.0, lam[-1] + 5.0, xtol=1e-15, rtol=4 * np.finfo(float).eps,
                     maxiter=500)
        assert abs(mu - ref) <= 1e-12 * max(1.0, abs(ref)), (trial, mu, ref)
        g = OB.occupations(lam, mu, kT)
        assert abs(2 * g.sum() - ne) <= 1e-9 * ns
        assert np.all(np.diff(g) <= 0)


def test_fermi_level_rejects_impossible_counts():
    for ne in (0.0, -1.0, 8.0, 9.0):
        with pytest.raises(ValueError):
            OB.fermi_level(np.array([0.0, 1.0, 2.0, 3.0]), ne, 1e-3)


# ------------------------------------------------------------------------------------
# Density
# ------------------------------------------------------------------------------------
def test_density_integrates_and_is_rotation_invariant():
    rng = np.random.default_rng(5)
    nd, ns, h = 700, 9, 0.4
    X, _ = np.linalg.qr(rng.standard_normal((nd, ns)))
    X = np.ascontiguousarray(X.T)
    g = rng.uniform(0, 1, ns)
    rho = OB.density(X, g, h)
    assert np.all(rho >= 0)
    assert abs(h ** 3 * rho.sum() - 2 * g.sum()) <= 1e-13 * ns
    # equal occupations: rho = (2 g / h^3) diag(X^T X) does not see an orthogonal mixing
    Q, _ = np.linalg.qr(rng.standard_normal((ns, ns)))
    ge = np.full(ns, 0.7)
    r1, r2 = OB.density(X, ge, h), OB.density(Q.T @ X, ge, h)
    assert np.max(np.abs(r1 - r2)) <= 1e-13 * np.max(r1)
    # one column, g = 1: 2 x^2 / h^3
    assert np.allclose(OB.density(X[:1], [1.0], h), 2 * X[0] ** 2 / h ** 3, rtol=1e-15, atol=0)


# ------------------------------------------------------------------------------------
# Non-local force
# ------------------------------------------------------------------------------------
def _force_case():
    n, h = 48, 0.25
    c = (n - 1) * h / 2
    R = np.array([[c - 0.41, c + 0.23, c - 0.07], [c + 0.52, c - 0.31, c + 0.44]])
    gamma = np.array([[1.3, -0.8, -0.8, -0.8], [-1.7, 0.9, 0.9, 0.9]])
    V = np.zeros(n ** 3)
    rng = np.random.default_rng(7)
    X = rng.uniform(-0.5, 0.5, (3, n ** 3))
    g = np.array([1.0, 0.6, 0.25])
    # chi(r_c) / max chi ~ 1e-8: the truncated support hardly moves the derivative (at
    # r_c = 4.5 the mismatch is 9e-5, at 5.0 it is 4e-6 of the largest component)
    rcut = 5.0
    return n, h, R, gamma, V, X, g, rcut


def test_nonlocal_force_is_minus_energy_derivative():
    n, h, R, gamma, V, X, g, rcut = _force_case()
    H = oracle.Hamiltonian(n, h, V, R, gamma, 0.8, rcut)
    f = OB.nonlocal_force(H, X, g)

    def energy(Rs):
        return OB.nonlocal_energy(oracle.Hamiltonian(n, h, V, Rs, gamma, 0.8, rcut), X, g)

    # Richardson-extrapolated central differences (error O(delta^4))
    d1, d2 = 2e-3, 1e-3
    num = np.zeros_like(f)
    for J in range(R.shape[0]):
        for d in range(3):
            def cd(dl):
                Rp, Rm = R.copy(), R.copy()
                Rp[J, d] += dl
                Rm[J, d] -= dl
                return (energy(Rp) - energy(Rm)) / (2 * dl)
            num[J, d] = -(4 * cd(d2) - cd(d1)) / 3
    scale = np.max(np.abs(num))
    assert scale > 1e-3
    assert np.max(np.abs(f - num)) <= 2e-5 * scale, (f, num)


def test_nonlocal_force_structure():
    # no atoms' gamma -> no force; gamma scales it linearly; g = 0 -> no force
    n, h, R, gamma, V, X, g, rcut = _force_case()
    X = X[:2]
    g = g[:2]
    H = oracle.Hamiltonian(n, h, V, R, gamma, 0.8, 3.0)
    f = OB.nonlocal_force(H, X, g)
    H2 = oracle.Hamiltonian(n, h, V, R, 2.5 * gamma, 0.8, 3.0)
    assert np.allclose(OB.nonlocal_force(H2, X, g), 2.5 * f, rtol=1e-13, atol=0)
    assert np.all(OB.nonlocal_force(H, X, np.zeros(2)) == 0)
    # the force is a sum over columns
    f0 = OB.nonlocal_force(H, X[:1], g[:1])
    f1 = OB.nonlocal_force(H, X[1:], g[1:])
    assert np.allclose(f, f0 + f1, rtol=1e-12, atol=1e-15)
