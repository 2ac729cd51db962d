"""Pins of the CPU oracle against what the paper and the mathematics fix (no GPU).

Each test is chosen so that a plausible slip in the oracle (a dropped term, a wrong sign,
index or stride, a transposed operand, a wrong normalisation) fails at least one of them:

* FD weights (Eq. weightsLap): exact rationals satisfy the moment conditions of a
  centred second-derivative stencil of order 2 n_o; n_o = 1 is the 7-point Laplacian.
* Stencil (Eq. FD:Laplacian): exact on polynomials of degree <= 2 n_o + 1 per axis
  (interior nodes), error order 12 under h -> h/2, Dirichlet spectrum is the Kronecker
  sum of three 1-D spectra on a non-cubic grid.
* H: symmetric; V_nl vanishes away from the supports, has rank 4 per atom, and its
  s/p blocks reproduce closed-form Gaussian moment integrals (midpoint rule, Eq. IntApprox).
* V_eff: Coulomb tail and the r -> 0 limit.
* Filter (Algorithm ChebychevFilter): on a diagonal H and on exact kinetic eigenvectors
  it equals the scalar C_m(L(t)) / C_m(L(a0)) from cos/cosh closed forms.
* Lanczos: published splitmix64 outputs; interlacing; exact extremes for k = Nd.
* Rayleigh-Ritz: exact eigenvalues from an exact invariant subspace; converged CheFSI
  Ritz values equal dense eigenvalues (12^3 grid, Nd = 1728).
"""
import math
import os
from fractions import Fraction

import numpy as np
import pytest
import scipy.linalg as sla
from scipy.special import erf as sp_erf

import oracle
from oracle import oracle as O
from paper_1603_04334_gb300 import synth

HERE = os.path.dirname(os.path.abspath(__file__))


# ------------------------------------------------------------------------------------
# FD weights
# ------------------------------------------------------------------------------------
def _golden_weights():
    rows = []
    with open(os.path.join(HERE, "golden", "fd_weights_no6.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            p, a, b = line.split()
            rows.append(Fraction(int(a), int(b)))
    return rows


@pytest.mark.parametrize("no", [1, 2, 3, 4, 5, 6])
def test_weights_moment_conditions(no):
    # 1-D share of the stencil: 2 w0 f(0) + sum_p w_p (f(p) + f(-p)) must equal f''(0)
    # for f = x^(2k), k = 0..n_o (odd powers cancel by symmetry): 0 for k != 1, 2 for k = 1.
    w = oracle.lap_weights_exact(no)
    for k in range(0, no + 1):
        s = (2 * w[0] if k == 0 else Fraction(0)) + sum(w[p] * 2 * Fraction(p) ** (2 * k)
                                                       for p in range(1, no + 1))
        assert s == (2 if k == 1 else 0), (no, k, s)


def test_weights_7point_and_golden():
    w1 = oracle.lap_weights_exact(1)
    assert 6 * w1[0] == -6 and w1[1] == 1           # standard 7-point Laplacian
    gold = _golden_weights()
    assert oracle.lap_weights_exact(6) == gold
    for h in (0.5, 0.3, 0.25, 0.37):
        wd = oracle.lap_weights(6, h)
        for p in range(7):
            assert wd[p] == pytest.approx(float(gold[p]) / (h * h), rel=4e-16, abs=0)


# ------------------------------------------------------------------------------------
# Stencil
# ------------------------------------------------------------------------------------
def _grid(n, h):
    n0, n1, n2 = n
    k, j, i = np.meshgrid(np.arange(n2), np.arange(n1), np.arange(n0), indexing="ij")
    return (i * h).reshape(-1), (j * h).reshape(-1), (k * h).reshape(-1), i.reshape(-1), \
        j.reshape(-1), k.reshape(-1)


def test_laplacian_exact_on_polynomials():
    # Degree <= 13 per axis is integrated exactly by the order-12 centred stencil.
    n, h, no = (19, 20, 21), 0.37, 6
    x, y, z, i, j, k = _grid(n, h)
    cx, cy, cz = 9 * h, 9.5 * h, 10 * h
    X, Y, Zc = x - cx, y - cy, z - cz
    for (a, b, c) in [(0, 0, 0), (2, 0, 0), (0, 2, 0), (0, 0, 2), (13, 0, 0), (0, 13, 0),
                      (0, 0, 13), (12, 7, 3), (5, 13, 11), (1, 1, 1)]:
        f = X ** a * Y ** b * Zc ** c
        lap = (a * (a - 1) * X ** max(a - 2, 0) * Y ** b * Zc ** c if a >= 2 else 0 * X) \
            + (b * (b - 1) * X ** a * Y ** max(b - 2, 0) * Zc ** c if b >= 2 else 0 * X) \
            + (c * (c - 1) * X ** a * Y ** b * Zc ** max(c - 2, 0) if c >= 2 else 0 * X)
        out = oracle.laplacian(f, n, h, no)
        inner = ((i >= no) & (i < n[0] - no) & (j >= no) & (j < n[1] - no)
                 & (k >= no) & (k < n[2] - no))
        scale = np.max(np.abs(f[inner])) / h ** 2 + 1.0
        err = np.max(np.abs(out[inner] - lap[inner]))
        assert err <= 1e-11 * scale, ((a, b, c), err, scale)


def test_laplacian_order_twelve():
    # Gaussian of width 1 centred in a 16 bohr box (negligible at the walls).
    L, s = 16.0, 1.0
    errs = []
    hs = [0.4, 0.2]
    for h in hs:
        n = int(round(L / h)) + 1
        x, y, z, *_ = _grid((n, n, n), h)
        r2 = (x - L / 2) ** 2 + (y - L / 2) ** 2 + (z - L / 2) ** 2
        f = np.exp(-r2 / (2 * s * s))
        exact = (r2 / s ** 4 - 3 / s ** 2) * f
        errs.append(np.max(np.abs(oracle.laplacian(f, (n, n, n), h, 6) - exact)))
    slope = math.log(errs[0] / errs[1]) / math.log(hs[0] / hs[1])
    assert 11.0 < slope < 13.5, (errs, slope)


def test_dirichlet_spectrum_is_kronecker_sum():
    # On a non-cubic grid, L_h = T_x (+) T_y (+) T_z with each 1-D operator read off the
    # oracle on an (m, 1, 1) grid minus 2/3 of the (1, 1, 1) diagonal. A transposed stride
    # or a boundary slip on one axis breaks the equality.
    h = 0.5

    def dense(n):
        nd = n[0] * n[1] * n[2]
        M = np.zeros((nd, nd))
        for c in range(nd):
            e = np.zeros(nd)
            e[c] = 1.0
            M[:, c] = oracle.laplacian(e, n, h, 6)
        return M

    d1 = dense((1, 1, 1))[0, 0]
    T = {m: dense((m, 1, 1)) - (2.0 / 3.0) * d1 * np.eye(m) for m in (5, 7, 8)}
    for m in T:
        # the (m,1,1) operator read along y or z is the same matrix
        assert np.allclose(dense((1, m, 1)), dense((m, 1, 1)), atol=0, rtol=0)
    Lfull = dense((5, 7, 8))
    assert np.array_equal(Lfull, Lfull.T)
    ev = np.sort(np.linalg.eigvalsh(Lfull))
    t5, t7, t8 = (np.linalg.eigvalsh(T[m]) for m in (5, 7, 8))
    sums = np.sort((t5[:, None, None] + t7[None, :, None] + t8[None, None, :]).reshape(-1))
    assert np.max(np.abs(ev - sums)) < 1e-11 * np.max(np.abs(ev))


# ------------------------------------------------------------------------------------
# Hamiltonian
# ------------------------------------------------------------------------------------
@pytest.fixture(scope="module")
def cluster24():
    w = synth.preset("cluster24")
    cl = synth.make_cluster(w, 0)
    return w, cl, oracle.Hamiltonian.from_cluster(cl)


def test_hamiltonian_symmetric(cluster24):
    w, cl, H = cluster24
    rng = np.random.default_rng(5)
    U = rng.standard_normal((3, w.nd))
    HU = H.apply(U)
    G = U @ HU.T
    assert np.max(np.abs(G - G.T)) <= 1e-13 * np.linalg.norm(U[0]) * np.linalg.norm(HU[0]) * 3


def test_apply_at_matches_apply(cluster24):
    w, cl, H = cluster24
    X = synth.initial_block(3, w.nd, 4)
    HX = H.apply(X)
    rng = np.random.default_rng(1)
    # include support nodes of atom 0 so that the nonlocal branch is exercised
    pts = np.concatenate([rng.integers(0, w.nd, 40), H.proj.idx[:20]])
    cols = rng.integers(0, 4, pts.shape[0]).astype(np.int32)
    got = H.apply_at(X, pts, cols)
    assert np.max(np.abs(got - HX[cols, pts])) <= 1e-13 * np.max(np.abs(HX))


def test_nonlocal_vanishes_off_support_and_has_rank_4_per_atom():
    n, h = 14, 0.5
    w = synth.Workload("t", n=n, h=h, natoms=2, ns=4, degree=4, iters=1, margin=2.0)
    cl = synth.make_cluster(w, 3)
    assert cl.natoms == 2
    V0 = np.zeros(n ** 3)
    Hnl = oracle.Hamiltonian(n, h, V0, cl.R, cl.gamma, kscale=0.0)  # H = V_nl only
    D = Hnl.dense()
    assert np.allclose(D, D.T, rtol=0, atol=1e-15)
    sv = np.linalg.svd(D, compute_uv=False)
    assert np.sum(sv > 1e-10 * sv[0]) == 4 * cl.natoms
    # rows/columns outside every support are zero
    sup = np.zeros(n ** 3, bool)
    sup[Hnl.proj.idx] = True
    assert np.all(D[~sup, :] == 0) and np.all(D[:, ~sup] == 0)
    # a support node's own distance from its atom is within rcut
    x, y, z, *_ = _grid((n, n, n), h)
    for J in range(cl.natoms):
        b, e = Hnl.proj.atom_ptr[J], Hnl.proj.atom_ptr[J + 1]
        idx = Hnl.proj.idx[b:e]
        r = np.sqrt((x[idx] - cl.R[J, 0]) ** 2 + (y[idx] - cl.R[J, 1]) ** 2
                    + (z[idx] - cl.R[J, 2]) ** 2)
        assert np.all(r <= 3.0 + 1e-12)


def test_projector_support_count_lattice_ball():
    # Atom on a node: r^2 = h^2 (i^2+j^2+k^2) <= 9 exactly <=> i^2+j^2+k^2 <= 36 at h = 0.5.
    h, n = 0.5, 24
    R = np.array([[6.0, 6.0, 6.0]])
    P = oracle.projectors(n, h, R, 0.8, 3.0)
    r = np.arange(-6, 7)
    brute = int(np.sum((r[:, None, None] ** 2 + r[None, :, None] ** 2
                        + r[None, None, :] ** 2) <= 36))
    assert P.atom_ptr[1] == brute


@pytest.mark.parametrize("gs,gp", [(1.3, -0.7), (-2.0, 0.4)])
def test_nonlocal_moments_closed_form(gs, gp):
    # One atom on a node of a fine grid. By symmetry the s and p projectors are orthogonal
    # on the grid, so V_nl chi_s = gs * h^3 |chi_s|^2 chi_s and V_nl chi_px = gp h^3 |chi_px|^2
    # chi_px. The midpoint sums (Eq. IntApprox) approach the Gaussian moment integrals
    #   int_{r<=3} Y00^2 e^{-r^2/s^2} = int_0^3 r^2 e^{-r^2/s^2} dr,
    #   int_{r<=3} (3/4pi) x^2 e^{-r^2/s^2} = int_0^3 r^4 e^{-r^2/s^2} dr.
    n, h, sig = 40, 0.25, 0.8
    R = np.array([[5.0, 5.0, 5.0]])
    gamma = np.array([[gs, gp, gp, gp]])
    H = oracle.Hamiltonian(n, h, np.zeros(n ** 3), R, gamma, sigma=sig, rcut=3.0, kscale=0.0)
    P = H.proj
    chi_s = np.zeros(n ** 3)
    chi_px = np.zeros(n ** 3)
    chi_s[P.idx] = P.chi[:, 0]
    chi_px[P.idx] = P.chi[:, 1]
    a = sig * sig
    I2 = (math.sqrt(math.pi) * a ** 1.5 / 4) * math.erf(3 / sig) - (a / 2) * 3 * math.exp(-9 / a)
    I4 = (3 * math.sqrt(math.pi) * a ** 2.5 / 8) * math.erf(3 / sig) \
        - (a / 2) * 27 * math.exp(-9 / a) - (3 * a * a / 4) * 3 * math.exp(-9 / a)
    out_s = H.apply(chi_s)[0]
    out_p = H.apply(chi_px)[0]
    m = chi_s != 0
    ratio_s = out_s[m] / chi_s[m]
    mp = np.abs(chi_px) > 1e-3 * np.max(np.abs(chi_px))
    ratio_p = out_p[mp] / chi_px[mp]
    assert np.ptp(ratio_s) <= 1e-12 * abs(ratio_s[0])
    assert np.ptp(ratio_p) <= 1e-12 * abs(ratio_p[0])
    assert ratio_s[0] == pytest.approx(gs * I2, rel=2e-4)
    assert ratio_p[0] == pytest.approx(gp * I4, rel=2e-4)


def test_veff_limits():
    n, h = 24, 0.5
    R = np.array([[3.0, 3.0, 3.0]])
    Zv = np.array([3.0])
    V = oracle.veff(n, h, R, Zv, 1.0)
    x, y, z, *_ = _grid((n, n, n), h)
    r = np.sqrt((x - 3) ** 2 + (y - 3) ** 2 + (z - 3) ** 2)
    c = np.argmin(r)
    assert r[c] == 0 and V[c] == pytest.approx(-2 * 3.0 / math.sqrt(math.pi), rel=1e-15)
    far = r > 7.0
    assert np.max(np.abs(V[far] + 3.0 / r[far]) * r[far] / 3.0) < 1e-15
    mid = (r > 0) & (r < 7.0)
    ref = -3.0 * sp_erf(r[mid]) / r[mid]
    assert np.max(np.abs(V[mid] - ref)) <= 4e-16 * np.max(np.abs(ref))


# ------------------------------------------------------------------------------------
# Chebyshev filter
# ------------------------------------------------------------------------------------
def _cheb(m, x):
    x = np.asarray(x, dtype=np.float64)
    out = np.empty_like(x)
    inside = np.abs(x) <= 1
    out[inside] = np.cos(m * np.arccos(x[inside]))
    ax = np.abs(x[~inside])
    out[~inside] = np.cosh(m * np.arccosh(ax)) * np.sign(x[~inside]) ** m
    return out


@pytest.mark.parametrize("m", [1, 2, 3, 7, 10, 20])
def test_filter_on_diagonal_H(m):
    n = 10
    nd = n ** 3
    a0, a, b = -4.0, 1.5, 30.0
    rng = np.random.default_rng(m)
    V = rng.uniform(a0 - 0.5, b + 0.2, nd)
    V[0] = a0
    H = oracle.Hamiltonian(n, 0.5, V, kscale=0.0)
    X = rng.uniform(-0.5, 0.5, (3, nd))
    Y = H.cheb_filter(X, m, a, b, a0)
    e, c = (b - a) / 2, (b + a) / 2
    p = _cheb(m, (V - c) / e) / _cheb(m, np.array([(a0 - c) / e]))[0]
    ref = X * p[None, :]
    err = np.abs(Y - ref)
    assert np.all(err <= 1e-13 * np.maximum(np.abs(ref), np.max(np.abs(ref)) * 1e-3))
    assert np.allclose(Y[:, 0], X[:, 0], rtol=1e-14, atol=0)       # p(a0) = 1


def test_filter_on_kinetic_eigenvectors():
    # V = 0, no atoms: eigenvectors of -1/2 L_h are products of 1-D eigenvectors.
    n, h, m = 8, 0.5, 12
    T = np.zeros((n, n))
    d1 = None
    for c in range(n):
        e = np.zeros(n)
        e[c] = 1.0
        T[:, c] = oracle.laplacian(e, (n, 1, 1), h, 6)
    d1 = oracle.laplacian(np.ones(1), (1, 1, 1), h, 6)[0]
    T -= (2.0 / 3.0) * d1 * np.eye(n)
    t, U = np.linalg.eigh(-0.5 * T)
    H = oracle.Hamiltonian(n, h, np.zeros(n ** 3))
    cols, lams = [], []
    for (p, q, r) in [(0, 0, 0), (1, 0, 2), (3, 5, 7), (7, 7, 7), (2, 4, 1)]:
        v = np.einsum("k,j,i->kji", U[:, r], U[:, q], U[:, p]).reshape(-1)
        cols.append(v)
        lams.append(t[p] + t[q] + t[r])
    X = np.array(cols)
    lam = np.array(lams)
    a0, a, b = t[0] * 3 - 0.01, t[2] * 3, t[-1] * 3 + 0.1
    Y = H.cheb_filter(X, m, a, b, a0)
    e, c = (b - a) / 2, (b + a) / 2
    p = _cheb(m, (lam - c) / e) / _cheb(m, np.array([(a0 - c) / e]))[0]
    ref = X * p[:, None]
    assert np.max(np.abs(Y - ref)) <= 1e-12 * np.max(np.abs(ref))


def test_filter_rejects_bad_bounds(cluster24):
    w, cl, H = cluster24
    X = synth.initial_block(0, w.nd, 1)
    with pytest.raises(ValueError):
        H.cheb_filter(X, 3, 1.0, 0.5, -1.0)   # a > b
    with pytest.raises(ValueError):
        H.cheb_filter(X, 0, 1.0, 5.0, -1.0)   # degree 0


@pytest.fixture(scope="module")
def dense12():
    w = synth.preset("cluster12")
    cl = synth.make_cluster(w, 7)
    H = oracle.Hamiltonian.from_cluster(cl)
    D = H.dense()
    ev, EV = np.linalg.eigh(D)
    return w, cl, H, D, ev, EV


# ------------------------------------------------------------------------------------
# Lanczos
# ------------------------------------------------------------------------------------
def test_splitmix64_published_outputs():
    # SplitMix64 seeded with 0 yields 0xe220a8397b1dcdaf, 0x6e789e6aa1b965f4, ...
    # (state advances by the golden gamma before mixing, so seed ^ p with p = 0 and
    # seed = gamma gives the second output). u(z) = (z >> 11) 2^-53, start = u - 0.5.
    v = oracle.lanczos_start(1, 0)
    assert v[0] == (0xE220A8397B1DCDAF >> 11) * 2.0 ** -53 - 0.5
    v = oracle.lanczos_start(1, 0x9E3779B97F4A7C15)
    assert v[0] == (0x6E789E6AA1B965F4 >> 11) * 2.0 ** -53 - 0.5
    v = oracle.lanczos_start(3, 2)
    assert v[2] == (0xE220A8397B1DCDAF >> 11) * 2.0 ** -53 - 0.5  # 2 ^ 2 = 0


def test_lanczos_full_dimension():
    n = 3
    rng = np.random.default_rng(0)
    V = np.sort(rng.uniform(-3, 5, n ** 3))
    H = oracle.Hamiltonian(n, 0.5, V, kscale=0.0)
    al, be = H.lanczos(n ** 3, seed=11)
    T = np.diag(al) + np.diag(be[:-1], 1) + np.diag(be[:-1], -1)
    th = np.linalg.eigvalsh(T)
    assert th[0] == pytest.approx(V[0], abs=1e-10) and th[-1] == pytest.approx(V[-1], abs=1e-10)


def test_lanczos_interlacing_and_upper_bound(dense12):
    # k = 10: Ritz values of T_k lie inside the spectrum, and the upper bound covers
    # lambda_max.
    w, cl, H, D, ev, EV = dense12
    for seed in (0, 1, 2):
        lo, hi, thmax = H.lanczos_bounds(10, seed=seed)
        assert ev[0] - 1e-9 <= lo and thmax <= ev[-1] + 1e-9
        assert hi >= ev[-1]


# ------------------------------------------------------------------------------------
# Rayleigh-Ritz and the CheFSI loop
# ------------------------------------------------------------------------------------
def test_rr_recovers_exact_invariant_subspace(dense12):
    w, cl, H, D, ev, EV = dense12
    rng = np.random.default_rng(2)
    ns = 7
    mix = rng.standard_normal((ns, ns)) + 3 * np.eye(ns)
    Y = (EV[:, :ns] @ mix).T          # rows are columns of Psi_f
    X, HX, lam, res, Cf = oracle.orth_rr(Y, H.apply(Y))
    assert np.max(np.abs(lam - ev[:ns])) < 1e-11
    assert np.max(res) < 1e-10
    assert np.max(np.abs(X @ X.T - np.eye(ns))) < 1e-12


def test_rr_raises_on_rank_deficient_block(dense12):
    w, cl, H, D, ev, EV = dense12
    Y = np.vstack([EV[:, 0], EV[:, 0], EV[:, 1]])
    with pytest.raises(oracle.NotSPD):
        oracle.orth_rr(Y, H.apply(Y))


def test_chefsi_converges_to_dense_eigenvalues(dense12):
    w, cl, H, D, ev, EV = dense12
    X0 = synth.initial_block(4, w.nd, w.ns)
    X, ritz, res, hist, _ = oracle.chefsi_solve(H, X0, 12, 40, tol=1e-9)
    # With the cutoff at the largest Ritz value and no buffer states, the top states
    # converge slowest; the lowest ns - 2 are converged to rounding.
    k = w.ns - 2
    assert np.max(np.abs(ritz[:k] - ev[:k])) < 1e-10
    assert np.max(np.abs(ritz - ev[:w.ns])) < 1e-3
    assert np.max(np.abs(X @ X.T - np.eye(w.ns))) < 1e-12
    assert np.all(ritz >= ev[:w.ns] - 1e-10)     # Ritz values bound eigenvalues from above


def test_chefsi_free_box_shells():
    # V = 0, no atoms: eigenvalues are sums of three 1-D eigenvalues; the first shells
    # (sizes 1, 3, 3, 3, 1) close at 11 states.
    n, h, ns = 12, 0.5, 11
    H = oracle.Hamiltonian(n, h, np.zeros(n ** 3))
    T = np.zeros((n, n))
    for c in range(n):
        e = np.zeros(n)
        e[c] = 1.0
        T[:, c] = oracle.laplacian(e, (n, 1, 1), h, 6)
    d1 = oracle.laplacian(np.ones(1), (1, 1, 1), h, 6)[0]
    t = np.linalg.eigvalsh(-0.5 * (T - (2.0 / 3.0) * d1 * np.eye(n)))
    sums = np.sort((t[:, None, None] + t[None, :, None] + t[None, None, :]).reshape(-1))
    X0 = synth.initial_block(9, n ** 3, ns)
    X, ritz, res, hist, _ = oracle.chefsi_solve(H, X0, 14, 60, tol=1e-10)
    assert np.max(np.abs(ritz[:10] - sums[:10])) < 1e-10


# --------------------------------------------------------------------------------------
# eigenvector sign convention (largest-magnitude entry positive, lowest index on ties)
# --------------------------------------------------------------------------------------
def test_fix_signs_hand_built():
    # column 0: largest |.| is -0.8 -> flipped; column 1: largest is +0.9 -> kept;
    # column 2: exact tie 0.5 / -0.5, the first (+0.5) decides -> kept; column 3: exact tie
    # -0.5 / 0.5, the first (-0.5) decides -> flipped; column 4: all zero -> kept.
    Q = np.array([[0.6, -0.3, 0.5, -0.5, 0.0],
                  [-0.8, 0.9, -0.5, 0.5, 0.0],
                  [0.0, -0.3, 0.1, 0.2, 0.0]])
    want = np.array([[-0.6, -0.3, 0.5, 0.5, 0.0],
                     [0.8, 0.9, -0.5, -0.5, 0.0],
                     [-0.0, -0.3, 0.1, -0.2, 0.0]])
    got = O.fix_signs(Q)
    assert np.array_equal(got, want)
    assert np.array_equal(Q[:, 1], got[:, 1])        # the input is not modified in place
    assert Q[1, 0] == -0.8


def test_rr_keeps_signs_of_an_exact_eigenbasis(dense12):
    # Rows of Y: exact eigenvectors of H, shuffled and with chosen signs. Then M_s = I, the
    # projected matrix is diagonal, Q is a permutation whose +-1 entries the convention turns
    # to +1, and X must be Y's rows sorted by eigenvalue with the signs Y gave them.
    w, cl, H, D, ev, EV = dense12
    ns = 6
    order = np.array([3, 0, 5, 1, 4, 2])
    sgn = np.array([-1.0, 1.0, -1.0, -1.0, 1.0, 1.0])
    Y = sgn[:, None] * EV[:, order].T
    X, HX, lam, res, Cf = oracle.orth_rr(Y, H.apply(Y))
    assert np.max(np.abs(lam - ev[:ns])) < 1e-11
    want = Y[np.argsort(order)]
    assert np.max(np.abs(X - want)) < 1e-10
    # the coefficient matrix is the permutation itself, every nonzero entry +1
    assert np.max(np.abs(Cf - np.eye(ns)[:, np.argsort(order)])) < 1e-10
