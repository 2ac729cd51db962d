"""GPU parity of the steps after the rotation: occupations and Fermi level, density,
non-local force (through the C ABI, against the FP64 oracle in oracle/observables.py).

Tolerances:
* Fermi level: |d lambda_f| <= 1e-10 Ha and |d g_n| <= 1e-10. Both sides find the same
  root of a monotone function to a few ulps; F' = (2/kT) sum g (1-g) turns the ~ns eps
  error of evaluating F into the root's uncertainty, far below 1e-10 for these spectra.
* Density: max|d rho| <= 1e-14 max rho: a sum of ncols non-negative FP64 terms, each
  within a few ulps on both sides.
* Force: |d f_Jd| <= 1e-12 S_Jd + 1e-15, S_Jd = (4/h^3) sum_n g_n sum_lm |gamma Y W|: the
  oracle and the kernel sum the same FP64 products in different orders, so each result
  is within a small multiple of eps times the sum of the magnitudes it cancels.
"""
import numpy as np
import pytest

import oracle
from oracle import observables as OB
from paper_1603_04334_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # collected on CPU-only hosts with -m gpu: skip loudly
    pytestmark = [pytest.mark.gpu, pytest.mark.skip(reason="no CUDA device")]

from paper_1603_04334_gb300 import sparc  # noqa: E402

DEV = "cuda:0"


def to_dev(X, dtype=torch.float64):
    return torch.from_numpy(np.ascontiguousarray(X)).to(DEV, dtype=dtype)


def make_ctx(cl, V=None, n=None):
    return sparc.Context(n if n is not None else cl.n, cl.h, cl.R, cl.Z, cl.gamma, veff=V,
                         sigma=cl.sigma, rcut=cl.rcut, rc_erf=cl.rc_erf)


@pytest.fixture(scope="module")
def solved24():
    """The 24^3 cluster after three CheFSI iterations: orthonormal X, its Ritz values."""
    w = synth.preset("cluster24")
    cl = synth.make_cluster(w, 0)
    H = oracle.Hamiltonian.from_cluster(cl)
    ctx = make_ctx(cl, V=H.V)
    X = to_dev(synth.initial_block(1, w.nd, w.ns))
    W = torch.empty_like(X)
    bounds = ctx.first_bounds(w.lanczos_k, 0)
    for _ in range(3):
        ritz, _, bounds = ctx.chefsi_step(X, W, w.degree, bounds)
    yield w, cl, H, ctx, X, ritz
    ctx.close()


def _force_tol(H, X, g):
    Y, W = OB.nonlocal_projections(H, X)
    S = np.zeros((H.natoms, 3))
    for J in range(H.natoms):
        S[J] = (4.0 / H.h ** 3) * np.einsum("n,l,nl,ndl->d", np.abs(g), np.abs(H.gamma[J]),
                                             np.abs(Y[J]), np.abs(W[J]))
    return 1e-12 * S + 1e-15


# --------------------------------------------------------------------------------------
# occupations
# --------------------------------------------------------------------------------------
@pytest.mark.parametrize("ns,kT", [(1, 1e-3), (2, 1e-3), (300, 1e-3), (1024, 1e-3),
                                   (5000, 1e-2), (77, 1e-4)])
def test_occupations_match_oracle(c_any, ns, kT):
    rng = np.random.default_rng(ns)
    lam = rng.uniform(-12.0, 3.0, ns)
    for ne in (0.37, float(ns) + 0.113, 2.0 * ns - 0.29):
        mu, g = c_any.occupations(lam, ne, kT)
        mu_o = OB.fermi_level(lam, ne, kT)
        g_o = OB.occupations(lam, mu_o, kT)
        assert abs(mu - mu_o) <= 1e-10, (ns, ne, mu, mu_o)
        assert np.max(np.abs(g - g_o)) <= 1e-10
        assert abs(2.0 * g.sum() - ne) <= 1e-9 * ns


def test_occupations_of_the_ritz_values(solved24):
    w, cl, H, ctx, X, ritz = solved24
    # fractional fillings: the root sits on a partly occupied level (for an integer filling
    # of a wide gap every point of the gap is a root; see test_occupations_in_a_wide_gap)
    for ne in (2.3, 9.5, 2.0 * w.ns - 1.0):
        mu, g = ctx.occupations(ritz, ne, 1e-3)
        mu_o = OB.fermi_level(ritz, ne, 1e-3)
        assert abs(mu - mu_o) <= 1e-10
        assert np.max(np.abs(g - OB.occupations(ritz, mu_o, 1e-3))) <= 1e-10


def test_occupations_in_a_wide_gap(c_any):
    # both levels 3000 kT from the midpoint: g rounds to (1, 0) and every point of the gap
    # is a root in double precision; the occupations are still exact
    mu, g = c_any.occupations(np.array([-2.8, 3.2]), 2.0, 1e-3)
    assert -2.8 + 0.04 < mu < 3.2 - 0.04
    assert g[0] == 1.0 and g[1] == 0.0


def test_occupations_errors(c_any):
    lam = np.array([0.0, 1.0, 2.0])
    for ne, kT in ((0.0, 1e-3), (6.0, 1e-3), (-1.0, 1e-3), (2.0, 0.0), (2.0, -1e-3)):
        with pytest.raises(sparc.SparcError) as e:
            c_any.occupations(lam, ne, kT)
        assert e.value.status == sparc.SPARC_ERR_ARG
    with pytest.raises(sparc.SparcError) as e:
        c_any.occupations(np.array([0.0, np.nan, 2.0]), 2.0, 1e-3)
    assert e.value.status == sparc.SPARC_ERR_NONFINITE
    mu, g = c_any.occupations(lam, 3.0, 1e-3)  # the context is still usable
    assert abs(mu - 1.0) <= 1e-10 and abs(g[1] - 0.5) <= 1e-10


@pytest.fixture(scope="module")
def c_any():
    w = synth.preset("cluster24")
    cl = synth.make_cluster(w, 2)
    ctx = make_ctx(cl)
    yield ctx
    ctx.close()


# --------------------------------------------------------------------------------------
# density
# --------------------------------------------------------------------------------------
def test_density_f64_and_f32(solved24):
    w, cl, H, ctx, X, ritz = solved24
    mu, g = ctx.occupations(ritz, 9.5, 1e-3)
    Xh = X.cpu().numpy()
    rho = ctx.density(X, g).cpu().numpy()
    ref = OB.density(Xh, g, cl.h)
    assert np.max(np.abs(rho - ref)) <= 1e-14 * np.max(ref)
    assert abs(cl.h ** 3 * rho.sum() - 9.5) <= 1e-9     # orthonormal columns: N_e
    X32 = X.float()
    rho32 = ctx.density(X32, g).cpu().numpy()
    ref32 = OB.density(X32.double().cpu().numpy(), g, cl.h)
    assert np.max(np.abs(rho32 - ref32)) <= 1e-14 * np.max(ref32)


def test_density_ragged_and_padded():
    n3, h = (37, 29, 23), 0.45
    nd = n3[0] * n3[1] * n3[2]
    rng = np.random.default_rng(9)
    ctx = sparc.Context(n3, h, None, None, None, veff=rng.uniform(-1, 0, nd))
    for ncols in (1, 13, 64):
        ld = nd + 7
        X = rng.uniform(-0.5, 0.5, (ncols, ld))
        g = rng.uniform(0, 1, ncols)
        rho = torch.full((nd,), 5.0, dtype=torch.float64, device=DEV)
        ctx.density(to_dev(X), g, rho)
        ref = OB.density(X[:, :nd], g, h)
        got = rho.cpu().numpy()
        assert np.max(np.abs(got - ref)) <= 1e-14 * np.max(ref)
    ctx.close()


# --------------------------------------------------------------------------------------
# non-local force
# --------------------------------------------------------------------------------------
def test_force_matches_oracle(solved24):
    w, cl, H, ctx, X, ritz = solved24
    mu, g = ctx.occupations(ritz, 9.5, 1e-3)
    Xh = X.cpu().numpy()
    f = ctx.nonlocal_force(X, g)
    ref = OB.nonlocal_force(H, Xh, g)
    assert f.shape == ref.shape == (cl.R.shape[0], 3)
    assert np.all(np.abs(f - ref) <= _force_tol(H, Xh, g)), (f, ref)
    # FP32 block: the oracle on the same (rounded) values
    X32 = X.float()
    f32 = ctx.nonlocal_force(X32, g)
    X32h = X32.double().cpu().numpy()
    assert np.all(np.abs(f32 - OB.nonlocal_force(H, X32h, g)) <= _force_tol(H, X32h, g))


def test_force_ragged_grid_atoms_at_the_boundary():
    # projector supports cut by the grid faces: the gradient's zero-Dirichlet values there
    n3, h = (37, 29, 23), 0.45
    nd = n3[0] * n3[1] * n3[2]
    rng = np.random.default_rng(4)
    R = np.array([[0.3, 5.0, 4.4], [15.9, 12.4, 0.2], [8.0, 6.1, 5.0]])
    gamma = rng.uniform(-2, 2, (3, 4))
    V = rng.uniform(-1, 0, nd)
    H = oracle.Hamiltonian(n3, h, V, R, gamma)
    ctx = sparc.Context(n3, h, R, None, gamma, veff=V)
    ld = nd + 3
    X = rng.uniform(-0.5, 0.5, (5, ld))
    g = np.array([1.0, 1.0, 0.7, 0.2, 0.0])
    f = ctx.nonlocal_force(to_dev(X), g)
    Xo = X[:, :nd].copy()
    ref = OB.nonlocal_force(H, Xo, g)
    assert np.all(np.abs(f - ref) <= _force_tol(H, Xo, g)), (f, ref)
    ctx.close()


def test_force_without_atoms_and_repeatable(solved24):
    w, cl, H, ctx, X, ritz = solved24
    g = np.linspace(1.0, 0.0, w.ns)
    a, b = ctx.nonlocal_force(X, g), ctx.nonlocal_force(X, g)
    assert np.array_equal(a, b)          # fixed reduction order
    c0 = sparc.Context(12, 0.5, None, None, None, veff=np.zeros(12 ** 3))
    Xe = torch.rand((2, 12 ** 3), dtype=torch.float64, device=DEV)
    assert c0.nonlocal_force(Xe, [1.0, 0.5]).shape == (0, 3)
    c0.close()


# --------------------------------------------------------------------------------------
# full size: 96^3 grid, 40 atoms, 128 FP64 columns
# --------------------------------------------------------------------------------------
def test_density_and_force_full_size():
    w = synth.preset("cluster96")
    cl = synth.make_cluster(w, 0)
    ctx = make_ctx(cl)
    X = torch.rand((w.ns, w.nd), dtype=torch.float64, device=DEV, generator=torch.Generator(DEV).manual_seed(5)) - 0.5
    X /= torch.linalg.vector_norm(X, dim=1, keepdim=True)
    rng = np.random.default_rng(1)
    g = np.sort(rng.uniform(0, 1, w.ns))[::-1].copy()
    rho = ctx.density(X, g)
    pts = rng.choice(w.nd, 4096, replace=False)
    Xs = X[:, torch.from_numpy(pts).to(DEV)].cpu().numpy()
    ref = OB.density(Xs, g, cl.h)
    got = rho[torch.from_numpy(pts).to(DEV)].cpu().numpy()
    assert np.max(np.abs(got - ref)) <= 1e-14 * np.max(ref)
    # force on every atom from 16 of the columns (the others get g = 0 on both sides)
    cols = np.arange(0, w.ns, 8)
    gs = np.zeros(w.ns)
    gs[cols] = g[cols]
    f = ctx.nonlocal_force(X, gs)
    H = oracle.Hamiltonian.from_cluster(cl, V=np.zeros(w.nd))
    Xc = X[torch.from_numpy(cols).to(DEV)].cpu().numpy()
    ref = OB.nonlocal_force(H, Xc, g[cols])
    assert np.all(np.abs(f - ref) <= _force_tol(H, Xc, g[cols]))
    ctx.close()
