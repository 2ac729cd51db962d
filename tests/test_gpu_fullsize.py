"""Parity at the full sizes of the two headline workloads, through the same C-ABI calls
(and so the same kernels and launch configurations) the benchmark times.

* 96^3 grid, 40 atoms, 128 FP64 columns: H X on sampled (node, column) outputs, each
  evaluated by the oracle from the definition; one complete CheFSI iteration (Lanczos
  bounds, degree-20 filter, Rayleigh-Ritz) against the oracle's iteration.
* 160^3 grid, 400 atoms, 1024 FP32 columns: H X and the degree-24 filter of the whole
  block, checked on sampled columns (H acts column by column, so the oracle's result for a
  column is exact whatever the other columns hold). The block repeats 16 seeded start
  columns 64 times (a 16 GB block would take minutes to draw on the host); the oracle
  filters the sampled columns from the same host data.
"""
import numpy as np
import pytest

import oracle
from paper_1603_04334_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytestmark = [pytest.mark.gpu, pytest.mark.skip(reason="no CUDA device")]

from paper_1603_04334_gb300 import sparc  # noqa: E402


def _ctx(cl, V):
    return sparc.Context(cl.n, cl.h, cl.R, cl.Z, cl.gamma, veff=V, sigma=cl.sigma,
                         rcut=cl.rcut, rc_erf=cl.rc_erf)


@pytest.fixture(scope="module")
def c96():
    w = synth.preset("cluster96")
    cl = synth.make_cluster(w, 0)
    H = oracle.Hamiltonian.from_cluster(cl)
    ctx = _ctx(cl, H.V)
    X0 = synth.initial_block(1, w.nd, w.ns)
    yield w, H, ctx, X0
    ctx.close()


def test_apply_H_f64_cluster96_sampled(c96):
    w, H, ctx, X0 = c96
    Xd = torch.from_numpy(X0).to("cuda")
    HXd = torch.empty_like(Xd)
    ctx.apply_H(Xd, HXd)
    HX = HXd.cpu().numpy()
    rng = np.random.default_rng(7)
    pts = rng.integers(0, w.nd, 4096)
    cols = rng.integers(0, w.ns, 4096)
    # boundary layers and the nodes next to atoms are where mistakes show: add them
    edge = np.array([0, 1, 5, 6, w.n - 7, w.n - 1])
    ii, jj, kk = np.meshgrid(edge, edge, edge, indexing="ij")
    extra = (ii + w.n * (jj + w.n * kk)).reshape(-1)
    pts = np.concatenate([pts, extra])
    cols = np.concatenate([cols, rng.integers(0, w.ns, extra.size)])
    ref = H.apply_at(X0, pts, cols)
    got = HX[cols, pts]
    scale = np.max(np.abs(HX))
    assert np.max(np.abs(got - ref)) <= 1e-12 * scale


def test_chefsi_iteration_cluster96_full(c96):
    w, H, ctx, X0 = c96
    lo_o, hi_o, _ = H.lanczos_bounds(w.lanczos_k, 0)
    lo, hi = ctx.lanczos_bounds(w.lanczos_k, 0)
    assert abs(lo - lo_o) <= 1e-10 and abs(hi - hi_o) <= 1e-10
    b = oracle.chefsi_first_bounds(lo_o, hi_o)
    Xn, ritz_o, resid_o, _ = oracle.chefsi_step(H, X0, w.degree, b)
    Xd = torch.from_numpy(X0).to("cuda")
    ritz, resid, _ = ctx.chefsi_step(Xd, torch.empty_like(Xd), w.degree, b)
    assert np.max(np.abs(ritz - ritz_o)) <= 1e-10
    assert np.max(np.abs(resid - resid_o)) <= 1e-9


def test_filter_f32_cluster160_sampled_columns():
    w = synth.preset("cluster160")
    cl = synth.make_cluster(w, 0)
    H = oracle.Hamiltonian.from_cluster(cl)
    ctx = _ctx(cl, H.V)
    X16 = torch.from_numpy(synth.initial_block(160, w.nd, 16)).to("cuda", torch.float32)
    X = X16.repeat(w.ns // 16, 1)
    del X16
    cols = np.array([0, 517, 1023])
    X0 = X[cols].double().cpu().numpy()
    # H X of the whole block
    HX = torch.empty_like(X)
    ctx.apply_H(X, HX)
    got = HX[cols].double().cpu().numpy()
    del HX
    ref = H.apply(X0)
    assert np.max(np.abs(got - ref)) <= 2e-6 * np.max(np.abs(ref))
    # the degree-24 filter of the whole block
    a, b, a0 = ctx.first_bounds(w.lanczos_k, 0)
    ctx.cheb_filter(X, torch.empty_like(X), w.degree, a, b, a0)
    got = X[cols].double().cpu().numpy()
    ref = H.cheb_filter(X0, w.degree, a, b, a0)
    assert np.max(np.abs(got - ref)) <= 1e-5 * np.max(np.abs(ref))
    ctx.close()
