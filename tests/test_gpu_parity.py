"""GPU parity: the CUDA path through the C ABI against the FP64 CPU oracle.

Tolerances (stated by the hot path's contract, or derived from it):
* H X (FP64): max|dHX| / max|HX_oracle| <= 1e-12 (normwise).
* Chebyshev filter (FP64): degree * 1e-12 normwise (m applications of H, each within the
  H X bound; the scaled recurrence keeps |Y_j| <= |Y_0| on the filtered components).
* Ritz values (FP64): <= 1e-10 Ha absolute; Lanczos bounds: <= 1e-10 absolute.
* FP32 arithmetic: 2e-6 normwise for H X, 1e-5 for the filter output.
Integer results (support sizes) are compared exactly.
"""
import math

import numpy as np
import pytest

import oracle
from paper_1603_04334_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # collected on CPU-only hosts with -m gpu: skip loudly
    pytestmark = [pytest.mark.gpu, pytest.mark.skip(reason="no CUDA device")]

from paper_1603_04334_gb300 import sparc  # noqa: E402


DEV = "cuda:0"


def to_dev(X, dtype=torch.float64):
    return torch.from_numpy(np.ascontiguousarray(X)).to(DEV, dtype=dtype)


def nrm_err(got, ref):
    return float(np.max(np.abs(got - ref)) / max(np.max(np.abs(ref)), 1e-300))


def make_ctx(cl, V=None, n=None):
    return sparc.Context(n if n is not None else cl.n, cl.h, cl.R, cl.Z, cl.gamma, veff=V,
                         sigma=cl.sigma, rcut=cl.rcut, rc_erf=cl.rc_erf)


@pytest.fixture(scope="module")
def c24():
    w = synth.preset("cluster24")
    cl = synth.make_cluster(w, 0)
    H = oracle.Hamiltonian.from_cluster(cl)
    ctx = make_ctx(cl, V=H.V)
    yield w, cl, H, ctx
    ctx.close()


# --------------------------------------------------------------------------------------
# setup: V_eff and projector tables
# --------------------------------------------------------------------------------------
def test_veff_built_on_device_matches_oracle():
    w = synth.preset("cluster24")
    cl = synth.make_cluster(w, 1)
    ctx = make_ctx(cl, V=None)
    Vg = ctx.get_veff()
    Vo = oracle.veff(cl.n, cl.h, cl.R, cl.Z, cl.rc_erf)
    assert nrm_err(Vg, Vo) <= 1e-14
    ctx.close()


@pytest.mark.parametrize("name,seed", [("cluster24", 0), ("cluster24", 3), ("cluster96", 0)])
def test_projector_support_size_exact(name, seed):
    w = synth.preset(name)
    cl = synth.make_cluster(w, seed)
    P = oracle.projectors(cl.n, cl.h, cl.R, cl.sigma, cl.rcut)
    ctx = make_ctx(cl, V=np.zeros(w.nd))
    info = ctx.info()
    assert info["natoms"] == cl.natoms
    assert info["nsupport"] == int(P.atom_ptr[-1])
    ctx.close()


# --------------------------------------------------------------------------------------
# H X
# --------------------------------------------------------------------------------------
def test_apply_H_f64_cluster24(c24):
    w, cl, H, ctx = c24
    X = synth.initial_block(2, w.nd, w.ns)
    ref = H.apply(X)
    Xd = to_dev(X)
    HXd = torch.empty_like(Xd)
    ctx.apply_H(Xd, HXd)
    torch.cuda.synchronize()
    assert nrm_err(HXd.cpu().numpy(), ref) <= 1e-12
    # deterministic: a second call is bitwise identical
    HX2 = torch.empty_like(Xd)
    ctx.apply_H(Xd, HX2)
    assert torch.equal(HXd, HX2)


@pytest.mark.parametrize("n3,natoms", [((37, 29, 23), 3), ((5, 7, 9), 0), ((13, 13, 13), 1),
                                       ((70, 9, 33), 2)])
def test_apply_H_f64_ragged_grids(n3, natoms):
    # several 32 x 8 tiles with ragged tails in x and y, grids smaller than the radius-6
    # halo, and the no-atom case
    h = 0.45
    rng = np.random.default_rng(sum(n3))
    R = np.array([[rng.uniform(0, (n3[0] - 1) * h), rng.uniform(0, (n3[1] - 1) * h),
                   rng.uniform(0, (n3[2] - 1) * h)] for _ in range(natoms)]).reshape(-1, 3)
    gamma = rng.uniform(-2, 2, (natoms, 4))
    nd = n3[0] * n3[1] * n3[2]
    V = rng.uniform(-3, 1, nd)
    H = oracle.Hamiltonian(n3, h, V, R if natoms else None, gamma if natoms else None)
    ctx = sparc.Context(n3, h, R if natoms else None, None, gamma if natoms else None, veff=V)
    ld = nd + 5                                       # padded leading dimension
    X = rng.uniform(-0.5, 0.5, (3, ld))
    X[:, nd:] = 0.0
    ref = H.apply(X[:, :nd].copy())
    Xd = to_dev(X)
    HXd = torch.full_like(Xd, 7.0)
    ctx.apply_H(Xd, HXd)
    got = HXd.cpu().numpy()
    assert nrm_err(got[:, :nd], ref) <= 1e-12
    assert np.all(got[:, nd:] == 7.0)                 # padding rows untouched
    ctx.close()


@pytest.mark.parametrize("h,ncols", [(0.45, 5), (0.15, 3)])
def test_nonlocal_part_f64_alone(h, ncols):
    # H with the kinetic part off and V = 0 is V_nl alone, so its FP64 projection and
    # scatter are compared with the oracle directly (random columns: their projections
    # cancel strongly, so the sums must be exact), on two overlapping supports and on one
    # support of about 33 500 entries (radius 20 grid spacings at h = 0.15: more than 128
    # per thread of the projection's 256-thread CTA, the pre-shifted warp sum).
    n3 = (48, 48, 48) if h < 0.2 else (23, 19, 21)
    nd = n3[0] * n3[1] * n3[2]
    rng = np.random.default_rng(int(h * 100))
    c = np.array([(n3[0] - 1) * h / 2, (n3[1] - 1) * h / 2, (n3[2] - 1) * h / 2])
    R = np.vstack([c, c + [0.7, -0.4, 0.3]]) if h > 0.2 else c.reshape(1, 3)
    gamma = rng.uniform(-2, 2, (R.shape[0], 4))
    V = np.zeros(nd)
    H = oracle.Hamiltonian(n3, h, V, R, gamma, kscale=0.0)
    ctx = sparc.Context(n3, h, R, None, gamma, veff=V)
    ctx.set_kinetic_scale(0.0)
    if h < 0.2:
        assert ctx.info()["nsupport"] > 32768
    X = rng.uniform(-0.5, 0.5, (ncols, nd))
    # a column far below the others' scale (its coefficients stay within the FP32 range of
    # the pair scatter's coefficients)
    X[-1] *= 1e-20
    ref = H.apply(X)
    Xd = to_dev(X)
    HXd = torch.empty_like(Xd)
    ctx.apply_H(Xd, HXd)
    got = HXd.cpu().numpy()
    assert np.abs(ref).max() > 0.0
    for j in range(ncols):
        assert nrm_err(got[j:j + 1], ref[j:j + 1]) <= 1e-12
    ctx.close()


def test_apply_H_f32(c24):
    w, cl, H, ctx = c24
    X = synth.initial_block(5, w.nd, 4)
    ref = H.apply(X)
    Xd = to_dev(X, torch.float32)
    HXd = torch.empty_like(Xd)
    ctx.apply_H(Xd, HXd)
    got = HXd.double().cpu().numpy()
    ref32 = H.apply(Xd.double().cpu().numpy())       # same rounded input, FP64 oracle
    assert nrm_err(got, ref32) <= 2e-6
    assert nrm_err(got, ref) <= 1e-5


@pytest.mark.parametrize("n3,pad", [((40, 29, 23), 0),   # TMA path: 2 x tiles, ragged y, z
                                    ((40, 29, 23), 4),   # TMA path, padded ld
                                    ((37, 29, 23), 0),   # n0 not a multiple of 4: plain path
                                    ((40, 29, 23), 3)])  # ld not a multiple of 4: plain path
def test_apply_H_and_filter_f32_both_stencil_paths(n3, pad):
    h = 0.45
    rng = np.random.default_rng(n3[0] + pad)
    nd = n3[0] * n3[1] * n3[2]
    R = np.array([[rng.uniform(2, (n3[0] - 1) * h - 2), rng.uniform(2, (n3[1] - 1) * h - 2),
                   rng.uniform(2, (n3[2] - 1) * h - 2)] for _ in range(3)])
    gamma = rng.uniform(-2, 2, (3, 4))
    V = rng.uniform(-3, 1, nd)
    H = oracle.Hamiltonian(n3, h, V, R, gamma)
    ctx = sparc.Context(n3, h, R, None, gamma, veff=V)
    ld = nd + pad
    X = np.zeros((5, ld))
    X[:, :nd] = rng.uniform(-0.5, 0.5, (5, nd))
    Xd = to_dev(X, torch.float32)
    X32 = Xd.double().cpu().numpy()[:, :nd].copy()
    HXd = torch.full_like(Xd, 7.0)
    ctx.apply_H(Xd, HXd)
    got = HXd.double().cpu().numpy()
    assert nrm_err(got[:, :nd], H.apply(X32)) <= 2e-6
    assert np.all(got[:, nd:] == 7.0)
    a0, a, b = -4.0, 5.0, 45.0
    ref = H.cheb_filter(X32, 8, a, b, a0)
    ctx.cheb_filter(Xd, torch.empty_like(Xd), 8, a, b, a0)
    assert nrm_err(Xd.double().cpu().numpy()[:, :nd], ref) <= 1e-5
    ctx.close()


def test_apply_H_f64_smooth_block():
    # Smooth, bound-state-like columns: H x is a small difference of large stencil terms
    # (|H x| ~ |lambda x| while sum|terms| ~ 100 |x| at h = 0.3), the hardest case for the
    # normwise 1e-12 bound.
    w = synth.preset("cluster24")
    n, h = 40, 0.3
    cl = synth.make_cluster(synth.Workload("s", n=n, h=h, natoms=3, ns=4, degree=4, iters=1), 2)
    H = oracle.Hamiltonian.from_cluster(cl)
    ctx = make_ctx(cl, V=H.V)
    k, j, i = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    x, y, z = i.reshape(-1) * h, j.reshape(-1) * h, k.reshape(-1) * h
    c = (n - 1) * h / 2
    r2 = (x - c) ** 2 + (y - c) ** 2 + (z - c) ** 2
    X = np.array([np.exp(-r2 / 8.0), (x - c) * np.exp(-r2 / 6.0), np.exp(-np.sqrt(r2 + 1.0)),
                  (x - c) * (y - c) * np.exp(-r2 / 10.0)])
    ref = H.apply(X)
    Xd = to_dev(X)
    HXd = torch.empty_like(Xd)
    ctx.apply_H(Xd, HXd)
    got = HXd.cpu().numpy()
    for col in range(X.shape[0]):
        assert nrm_err(got[col], ref[col]) <= 1e-12, col
    ctx.close()


def test_apply_H_single_column(c24):
    w, cl, H, ctx = c24
    X = synth.initial_block(8, w.nd, 1)
    Xd = to_dev(X)
    HXd = torch.empty_like(Xd)
    ctx.apply_H(Xd, HXd)
    assert nrm_err(HXd.cpu().numpy(), H.apply(X)) <= 1e-12


# --------------------------------------------------------------------------------------
# Chebyshev filter
# --------------------------------------------------------------------------------------
@pytest.mark.parametrize("degree", [1, 2, 10])
def test_cheb_filter_f64(c24, degree):
    w, cl, H, ctx = c24
    X = synth.initial_block(3, w.nd, w.ns)
    a0, a, b = -3.3, 7.6, 40.1
    ref = H.cheb_filter(X, degree, a, b, a0)
    Xd = to_dev(X)
    Wd = torch.empty_like(Xd)
    ctx.cheb_filter(Xd, Wd, degree, a, b, a0)
    assert nrm_err(Xd.cpu().numpy(), ref) <= degree * 1e-12


def test_f64_column_scales_zero_and_nonfinite(c24):
    # The FP64 stencil puts each column on a fixed-point grid scaled by a power of two from
    # the column's magnitude bound, and the filter hands the bound of Y_{j+1} from step to
    # step: columns of very different sizes, a zero column and a column holding a NaN
    # (which turns that column, and only it, into NaN). The sizes stay where the FP32-pair
    # projection and scatter keep their precision (|y| >= 2^-74: the low part of a pair
    # must stay a normal FP32 number).
    w, cl, H, ctx = c24
    X = synth.initial_block(4, w.nd, 5)
    sc = np.array([1e-15, 1.0, 3e25, 0.0, 1.0])
    X = X * sc[:, None]
    X[4, 1234] = np.nan
    Xd = to_dev(X)
    HXd = torch.empty_like(Xd)
    ctx.apply_H(Xd, HXd)
    got = HXd.cpu().numpy()
    for c in (0, 1, 2):
        ref = H.apply(X[c:c + 1] / sc[c]) * sc[c]
        assert nrm_err(got[c:c + 1], ref) <= 1e-12
    assert np.all(got[3] == 0.0)
    assert np.all(np.isnan(got[4]))
    a0, a, b = -3.3, 7.6, 40.1
    Wd = torch.empty_like(Xd)
    ctx.cheb_filter(Xd, Wd, 10, a, b, a0)
    got = Xd.cpu().numpy()
    for c in (0, 1, 2):
        ref = H.cheb_filter(X[c:c + 1] / sc[c], 10, a, b, a0) * sc[c]
        assert nrm_err(got[c:c + 1], ref) <= 10 * 1e-12
    assert np.all(got[3] == 0.0)
    assert np.all(np.isnan(got[4]))


def test_cheb_filter_f32(c24):
    w, cl, H, ctx = c24
    X = synth.initial_block(3, w.nd, 6)
    a0, a, b = -3.3, 7.6, 40.1
    Xd = to_dev(X, torch.float32)
    ref = H.cheb_filter(Xd.double().cpu().numpy(), 10, a, b, a0)
    Wd = torch.empty_like(Xd)
    ctx.cheb_filter(Xd, Wd, 10, a, b, a0)
    assert nrm_err(Xd.double().cpu().numpy(), ref) <= 1e-5


def _cheb(m, x):
    x = np.asarray(x, dtype=np.float64)
    out = np.empty_like(x)
    ins = np.abs(x) <= 1
    out[ins] = np.cos(m * np.arccos(x[ins]))
    out[~ins] = np.cosh(m * np.arccosh(np.abs(x[~ins]))) * np.sign(x[~ins]) ** m
    return out


def test_cheb_filter_diagonal_closed_form():
    # kscale = 0 and no atoms: H = diag(V); the filter must equal the scalar Chebyshev value.
    n, m = 20, 12
    rng = np.random.default_rng(4)
    a0, a, b = -4.0, 1.5, 30.0
    V = rng.uniform(a0 - 0.3, b + 0.1, n ** 3)
    ctx = sparc.Context(n, 0.5, veff=V)
    ctx.set_kinetic_scale(0.0)
    X = rng.uniform(-0.5, 0.5, (2, n ** 3))
    Xd = to_dev(X)
    ctx.cheb_filter(Xd, torch.empty_like(Xd), m, a, b, a0)
    e, c = (b - a) / 2, (b + a) / 2
    p = _cheb(m, (V - c) / e) / _cheb(m, np.array([(a0 - c) / e]))[0]
    ref = X * p[None, :]
    got = Xd.cpu().numpy()
    # the filter's contract: degree * 1e-12 normwise (the FP64 path computes in FP32-pair
    # arithmetic, about 2^-48 per step, so the element-wise 1e-13 of the CPU oracle's own
    # pin is not the bound here)
    assert nrm_err(got, ref) <= m * 1e-12
    big = np.abs(ref) > 1e-3 * np.max(np.abs(ref))
    assert np.max(np.abs(got - ref)[big] / np.abs(ref)[big]) <= 1e-11
    ctx.close()


def test_cheb_filter_rejects_bad_bounds(c24):
    w, cl, H, ctx = c24
    Xd = to_dev(synth.initial_block(0, w.nd, 2))
    before = Xd.clone()
    with pytest.raises(sparc.SparcError) as ei:
        ctx.cheb_filter(Xd, torch.empty_like(Xd), 5, 1.0, 0.5, -1.0)
    assert ei.value.status == sparc.SPARC_ERR_ARG
    with pytest.raises(sparc.SparcError):
        ctx.cheb_filter(Xd, torch.empty_like(Xd), 0, 1.0, 5.0, -1.0)
    assert torch.equal(Xd, before)


# --------------------------------------------------------------------------------------
# Lanczos bounds
# --------------------------------------------------------------------------------------
@pytest.mark.parametrize("seed", [0, 7])
def test_lanczos_bounds(c24, seed):
    w, cl, H, ctx = c24
    lo, hi = ctx.lanczos_bounds(10, seed)
    olo, ohi, _ = H.lanczos_bounds(10, seed)
    assert abs(lo - olo) <= 1e-10 and abs(hi - ohi) <= 1e-10


def test_lanczos_early_stop_tiny_grid():
    # Nd = 8 < k: the Krylov space is exhausted and beta reaches (numerically) zero.
    n = 2
    V = np.array([-1.0, 0.5, 2.0, 3.0, -0.25, 1.0, 4.0, 0.0])
    H = oracle.Hamiltonian(n, 0.5, V)
    ctx = sparc.Context(n, 0.5, veff=V)
    lo, hi = ctx.lanczos_bounds(12, 3)
    olo, ohi, _ = H.lanczos_bounds(12, 3)
    ev = np.linalg.eigvalsh(H.dense())
    assert abs(lo - olo) <= 1e-9 and abs(hi - ohi) <= 1e-9
    assert lo == pytest.approx(ev[0], abs=1e-8) and hi >= ev[-1] - 1e-12
    ctx.close()


# --------------------------------------------------------------------------------------
# Rayleigh-Ritz and CheFSI
# --------------------------------------------------------------------------------------
def test_orth_rr_f64(c24):
    w, cl, H, ctx = c24
    X0 = synth.initial_block(6, w.nd, w.ns)
    Yf = H.cheb_filter(X0, 10, 7.6, 40.1, -3.3)
    Xo, HXo, lam, res, _ = oracle.orth_rr(Yf, H.apply(Yf))
    Yd = to_dev(Yf)
    ritz, resid = ctx.orth_rr(Yd)
    assert np.max(np.abs(ritz - lam)) <= 1e-10
    assert np.max(np.abs(resid - res)) <= 1e-9
    Xg = Yd.cpu().numpy()
    # vectors compared as they are: both sides sign each eigenvector of the projected
    # problem so that its largest-magnitude entry is positive (lowest index on ties)
    assert np.max(np.abs(Xg - Xo)) <= 1e-9
    assert np.max(np.abs(Xg @ Xg.T - np.eye(w.ns))) <= 1e-12


def test_orth_rr_sign_convention_exact_eigenbasis():
    # Rows: exact eigenvectors of the 12^3 Hamiltonian, shuffled, with chosen signs. The
    # projected problem is diagonal, its eigenvectors a permutation with +-1 entries that the
    # sign convention makes +1, so the rotated block is the input sorted by eigenvalue with
    # the input's signs (the oracle is pinned to the same outcome on the CPU).
    w = synth.preset("cluster12")
    cl = synth.make_cluster(w, 7)
    H = oracle.Hamiltonian.from_cluster(cl)
    ev, EV = np.linalg.eigh(H.dense())
    order = np.array([3, 0, 5, 1, 4, 2])
    sgn = np.array([-1.0, 1.0, -1.0, -1.0, 1.0, 1.0])
    Y = sgn[:, None] * EV[:, order].T
    Xo, _, lam_o, _, _ = oracle.orth_rr(Y, H.apply(Y))
    ctx = make_ctx(cl, V=H.V)
    Yd = to_dev(Y)
    ritz, _ = ctx.orth_rr(Yd)
    Xg = Yd.cpu().numpy()
    assert np.max(np.abs(ritz - ev[:6])) <= 1e-10
    assert np.max(np.abs(Xg - Y[np.argsort(order)])) <= 1e-10
    assert np.max(np.abs(Xg - Xo)) <= 1e-10
    ctx.close()


@pytest.mark.parametrize("ns", [97, 300])
def test_orth_rr_f64_many_columns(c24, ns):
    # enough columns to spread the Cholesky over many CTAs (and an odd count for the
    # Jacobi's padded round-robin)
    w, cl, H, ctx = c24
    X0 = synth.initial_block(9, w.nd, ns)
    Yf = H.cheb_filter(X0, 2, 7.6, 40.1, -3.3)
    Xo, HXo, lam, res, _ = oracle.orth_rr(Yf, H.apply(Yf))
    Yd = to_dev(Yf)
    ritz, resid = ctx.orth_rr(Yd)
    assert np.max(np.abs(ritz - lam)) <= 1e-10
    assert np.max(np.abs(resid - res)) <= 1e-9
    Xg = Yd.cpu().numpy()
    assert np.max(np.abs(Xg @ Xg.T - np.eye(ns))) <= 1e-12


def test_orth_rr_f32_many_columns(c24):
    # the mixed-precision form at 300 columns: tensor-core Gram, mixed-precision eigensolve,
    # register-blocked FP32 rotation; Ritz values within the 1e-5 Ha contract of the FP64
    # oracle on the same (FP32-rounded) block, rotated block orthonormal to FP32 level
    w, cl, H, ctx = c24
    X0 = synth.initial_block(10, w.nd, 300)
    Yf = H.cheb_filter(X0, 2, 7.6, 40.1, -3.3)
    Yd = to_dev(Yf, torch.float32)
    Y64 = Yd.double().cpu().numpy()
    Xo, HXo, lam, res, _ = oracle.orth_rr(Y64, H.apply(Y64))
    ritz, resid = ctx.orth_rr(Yd)
    assert np.max(np.abs(ritz - lam)) <= 1e-5
    assert np.all(np.diff(ritz) >= 0)
    Xg = Yd.double().cpu().numpy()
    assert np.max(np.abs(Xg @ Xg.T - np.eye(300))) <= 1e-5
    assert np.max(np.abs(resid - res)) <= 1e-4


def test_orth_rr_not_spd_leaves_block(c24):
    w, cl, H, ctx = c24
    X = synth.initial_block(6, w.nd, 3)
    X[1] = X[0]                                   # rank-deficient block
    Xd = to_dev(X)
    before = Xd.clone()
    with pytest.raises(sparc.SparcError) as ei:
        ctx.orth_rr(Xd)
    assert ei.value.status == sparc.SPARC_ERR_NOT_SPD
    assert torch.equal(Xd, before)


def test_orth_rr_nonfinite(c24):
    w, cl, H, ctx = c24
    X = synth.initial_block(6, w.nd, 3)
    X[2, 100] = np.nan
    Xd = to_dev(X)
    with pytest.raises(sparc.SparcError) as ei:
        ctx.orth_rr(Xd)
    assert ei.value.status == sparc.SPARC_ERR_NONFINITE


def test_chefsi_loop_matches_oracle_cluster24(c24):
    w, cl, H, ctx = c24
    X0 = synth.initial_block(1, w.nd, w.ns)
    olo, ohi, _ = H.lanczos_bounds(w.lanczos_k, 0)
    b_g = ctx.first_bounds(w.lanczos_k, 0)
    b_o = oracle.chefsi_first_bounds(olo, ohi)
    assert np.max(np.abs(np.array(b_g) - np.array(b_o))) <= 1e-10
    Xd = to_dev(X0)
    Wd = torch.empty_like(Xd)
    Xo = X0.copy()
    for it in range(w.iters):
        ritz, resid, b_g = ctx.chefsi_step(Xd, Wd, w.degree, b_g)
        Xo, ritz_o, res_o, b_o = oracle.chefsi_step(H, Xo, w.degree, b_o)
        assert np.max(np.abs(ritz - ritz_o)) <= 1e-10, (it, ritz - ritz_o)
        assert np.max(np.abs(np.array(b_g) - np.array(b_o))) <= 1e-10
    Xg = Xd.cpu().numpy()
    assert np.max(np.abs(Xg @ Xg.T - np.eye(w.ns))) <= 1e-12
    # converged lower states agree with the oracle's vectors, signs included
    k = w.ns - 2
    assert np.max(np.abs(Xg[:k] - Xo[:k])) <= 1e-8


def test_chefsi_dense_12cubed_eigenvalues():
    w = synth.preset("cluster12")
    cl = synth.make_cluster(w, 7)
    H = oracle.Hamiltonian.from_cluster(cl)
    ev = np.linalg.eigvalsh(H.dense())
    ctx = make_ctx(cl, V=H.V)
    Xd = to_dev(synth.initial_block(4, w.nd, w.ns))
    Wd = torch.empty_like(Xd)
    b = ctx.first_bounds(10, 0)
    for it in range(40):
        ritz, resid, b = ctx.chefsi_step(Xd, Wd, 12, b)
        if np.max(resid) <= 1e-9:
            break
    k = w.ns - 2
    assert np.max(np.abs(ritz[:k] - ev[:k])) <= 1e-10
    ctx.close()


def test_mixed_precision_ritz_within_1e5(c24):
    # FP32 filter + FP64 Rayleigh-Ritz, then one FP64 refinement sweep: Ritz values of the
    # converged states within 1e-5 Ha of the FP64 run.
    w, cl, H, ctx = c24
    X0 = synth.initial_block(1, w.nd, w.ns)
    b64 = ctx.first_bounds(10, 0)
    X64 = to_dev(X0)
    W64 = torch.empty_like(X64)
    for it in range(w.iters):
        r64, _, b64 = ctx.chefsi_step(X64, W64, w.degree, b64)
    b32 = ctx.first_bounds(10, 0)
    X32 = to_dev(X0, torch.float32)
    W32 = torch.empty_like(X32)
    for it in range(w.iters):
        r32, _, b32 = ctx.chefsi_step(X32, W32, w.degree, b32)
    Xr = X32.double()
    rr, res, _ = ctx.chefsi_step(Xr, torch.empty_like(Xr), w.degree, b32)
    k = w.ns - 2
    assert np.max(np.abs(rr[:k] - r64[:k])) <= 1e-5


# --------------------------------------------------------------------------------------
# projection contraction
# --------------------------------------------------------------------------------------
@pytest.mark.parametrize("ncols,dt", [(12, "f64"), (70, "f64"), (33, "f32"), (20, "mix")])
def test_gram_matches_fp64_products(c24, ncols, dt):
    # G = A^T B against the FP64 product of the same (possibly FP32-rounded) inputs;
    # 70 and 33 columns leave ragged 64-column tiles.
    w, cl, H, ctx = c24
    rng = np.random.default_rng(ncols)
    A = rng.uniform(-0.5, 0.5, (ncols, w.nd))
    B = rng.uniform(-0.5, 0.5, (ncols, w.nd))
    ta = torch.float32 if dt in ("f32", "mix") else torch.float64
    tb = torch.float32 if dt == "f32" else torch.float64
    Ad, Bd = to_dev(A, ta), to_dev(B, tb)
    G = ctx.gram(Ad, Bd).cpu().numpy().T          # column-major -> (i, j)
    ref = Ad.double().cpu().numpy() @ Bd.double().cpu().numpy().T
    assert nrm_err(G, ref) <= 1e-13
    G2 = ctx.gram(Ad, Bd).cpu().numpy().T
    assert np.array_equal(G, G2)


# --------------------------------------------------------------------------------------
# tensor-core contraction of the mixed-precision form
# --------------------------------------------------------------------------------------
def _chunk_max(X, chunk=256):
    """|X| maximum over each 256-row chunk of every column, expanded back to rows.
    X: (ncols, nd) rows are columns of the Nd x ncols block."""
    nc, nd = X.shape
    nchunk = (nd + chunk - 1) // chunk
    P = np.zeros((nc, nchunk * chunk))
    P[:, :nd] = np.abs(X)
    m = P.reshape(nc, nchunk, chunk).max(axis=2)
    return np.repeat(m, chunk, axis=1)[:, :nd]


@pytest.mark.parametrize("n3,ncols,dts", [((24, 24, 24), 12, ("f32", "f32")),
                                          ((37, 29, 23), 130, ("f32", "f64")),
                                          ((37, 29, 23), 33, ("f64", "f64")),
                                          ((24, 24, 24), 257, ("f32", "f32"))])
def test_gram_tc_within_chunk_rounding_bound(n3, ncols, dts):
    # G = A^T B against the exact FP64 product of the same data; bound of sparc_gram_tc:
    # |dG_ij| <= 2^-21 sum_k (m_i m_j + m_i |B_kj| + |A_ki| m_j), m = chunk maxima
    w = synth.preset("cluster24")
    cl = synth.make_cluster(w, 0)
    ctx = make_ctx(cl, n=n3)
    nd = int(np.prod(n3))
    rng = np.random.default_rng(11)
    scale = 10.0 ** rng.uniform(-3, 3, size=(ncols, 1))     # columns of very different size
    A = (rng.standard_normal((ncols, nd)) * scale)
    A[:, ::7] *= 1e-4                                         # small entries inside chunks
    B = rng.standard_normal((ncols, nd)) * scale[::-1]
    tA = torch.float32 if dts[0] == "f32" else torch.float64
    tB = torch.float32 if dts[1] == "f32" else torch.float64
    Ad, Bd = to_dev(A, tA), to_dev(B, tB)
    A64, B64 = Ad.double().cpu().numpy(), Bd.double().cpu().numpy()
    Gd = ctx.gram_tc(Ad, Bd)
    G = Gd.cpu().numpy().T                                    # G[i, j] = entry (i, j)
    ref = A64 @ B64.T
    mA, mB = _chunk_max(A64), _chunk_max(B64)
    bound = 2.0 ** -21 * (mA @ mB.T + mA @ np.abs(B64).T + np.abs(A64) @ mB.T)
    err = np.abs(G - ref)
    assert np.all(err <= bound), float(np.max(err / bound))
    # bitwise repeatable
    assert torch.equal(ctx.gram_tc(Ad, Bd), Gd)
    ctx.close()


def test_gram_tc_symmetric_and_nonfinite(c24):
    w, cl, H, ctx = c24
    X = synth.initial_block(4, w.nd, 40)
    Xd = to_dev(X, torch.float32)
    G = ctx.gram_tc(Xd, Xd).cpu().numpy()
    assert np.array_equal(G, G.T)                 # exact digit sums: bitwise symmetric
    X[5, 300] = np.inf
    Gn = ctx.gram_tc(to_dev(X, torch.float32), to_dev(X, torch.float32)).cpu().numpy()
    assert np.all(np.isnan(Gn[5, :])) and np.all(np.isfinite(np.delete(np.delete(Gn, 5, 0), 5, 1)))
