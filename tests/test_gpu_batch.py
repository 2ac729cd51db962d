"""Batched filter over many uneven clusters: equals the per-cluster filter and the oracle,
across graph replays with new bounds and across every launch variant of the autotuner."""
import numpy as np
import pytest

import oracle
from paper_1603_04334_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytestmark = [pytest.mark.gpu, pytest.mark.skip(reason="no CUDA device")]

from paper_1603_04334_gb300 import batching, sparc  # noqa: E402

# grids with ragged tiles, one without atoms, one smaller than a tile in z; MIXED holds a
# grid the TMA path does not take (n0 not a multiple of 4), so the batch runs the
# shared-memory form; TMA runs the TMA-fed form
MIXED = [((24, 24, 24), 12, 3), ((37, 29, 23), 20, 4), ((32, 20, 40), 7, 0),
         ((20, 33, 18), 33, 2), ((40, 40, 12), 5, 1)]
TMA = [((24, 24, 24), 12, 3), ((44, 29, 23), 20, 4), ((32, 20, 40), 7, 0),
       ((20, 33, 18), 33, 2), ((40, 40, 12), 5, 1)]
SHAPES = MIXED


def _clusters(shapes=MIXED):
    rng = np.random.default_rng(5)
    out = []
    for n3, ns, na in shapes:
        h = 0.45
        R = np.array([[rng.uniform(2, (n - 1) * h - 2) for n in n3] for _ in range(na)]).reshape(-1, 3)
        gamma = rng.uniform(-2, 2, (na, 4))
        V = rng.uniform(-3, 1, int(np.prod(n3)))
        H = oracle.Hamiltonian(n3, h, V, R if na else None, gamma if na else None)
        ctx = sparc.Context(n3, h, R if na else None, None, gamma if na else None, veff=V)
        X = rng.uniform(-0.5, 0.5, (ns, int(np.prod(n3))))
        out.append((H, ctx, X))
    return out


def _bounds(k):
    return [(-4.0 + 0.3 * i + k, 6.0 + 0.5 * i, 45.0 + i) for i in range(len(MIXED))]


def _nrm(a, b):
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


@pytest.mark.parametrize("shapes", [MIXED, TMA], ids=["shared-memory", "tma"])
def test_batched_filter_equals_per_cluster_filter_and_oracle(shapes):
    cl = _clusters(shapes)
    m = 9
    Xb = [torch.from_numpy(X).to("cuda", torch.float32) for _, _, X in cl]
    Wb = [torch.empty_like(x) for x in Xb]
    batch = batching.Batch([c for _, c, _ in cl])
    for k in range(2):  # second call replays the graph with new bounds
        B = [(a, b, a0) for (a0, a, b) in _bounds(k)]
        start = [x.clone() for x in Xb]
        batch.filter(Xb, Wb, m, B)
        for (H, ctx, _), x0, xb, (a, b, a0) in zip(cl, start, Xb, B):
            xr = x0.clone()
            ctx.cheb_filter(xr, torch.empty_like(xr), m, a, b, a0)
            got, ref = xb.double().cpu().numpy(), xr.double().cpu().numpy()
            assert _nrm(got, ref) <= 2e-6
            assert _nrm(got, H.cheb_filter(x0.double().cpu().numpy(), m, a, b, a0)) <= 1e-5
    batch.close()
    for _, c, _ in cl:
        c.close()


@pytest.mark.parametrize("shapes", [MIXED, TMA], ids=["shared-memory", "tma"])
def test_every_variant_agrees_and_tuner_picks_one(shapes):
    cl = _clusters(shapes)
    m = 4
    B = [(a, b, a0) for (a0, a, b) in _bounds(0)]
    X0 = [torch.from_numpy(X).to("cuda", torch.float32) for _, _, X in cl]
    batch = batching.Batch([c for _, c, _ in cl])
    nvar = batch.set_variant(0)
    outs = []
    for v in range(nvar):
        batch.set_variant(v)
        Xb = [x.clone() for x in X0]
        batch.filter(Xb, [torch.empty_like(x) for x in Xb], m, B)
        outs.append([x.double().cpu().numpy() for x in Xb])
    # the shared-memory forms share their per-point arithmetic (bitwise equal); the TMA
    # forms (variants 9-14, when the blocks allow it) agree with each other bitwise and with
    # the shared-memory forms to FP32 rounding
    for v, o in enumerate(outs[1:], start=1):
        for a, b in zip(o, outs[0]):
            if v < 9 or shapes is MIXED:
                assert np.array_equal(a, b)
            else:
                assert _nrm(a, b) <= 2e-6
    if shapes is TMA:
        for v in range(10, nvar):
            for a, b in zip(outs[v], outs[9]):
                assert np.array_equal(a, b)
    Xt = [x.clone() for x in X0]
    v, ms = batch.tune(Xt, [torch.empty_like(x) for x in Xt], m, B)
    assert 0 <= v < nvar and ms > 0
    batch.close()
    for _, c, _ in cl:
        c.close()


def test_batched_filter_64_clusters_of_the_configured_mix():
    # 64 clusters drawn as the batching workload draws them (edge in {32, ..., 96},
    # h = 0.3, 2-60 atoms, Ns 16-160, degree 16): the batched filter of all of them against
    # sparc_cheb_filter on each cluster, and against the oracle on two columns of the four
    # smallest clusters
    spec = batching.draw_clusters(64, 0)
    m = 16
    ctxs, X0, B = [], [], []
    for i, (n, R, Z, gamma, ns) in enumerate(spec):
        ctx = sparc.Context(n, 0.3, R, Z, gamma)
        ctxs.append(ctx)
        B.append(ctx.first_bounds(10, i))
        X0.append(torch.from_numpy(synth.initial_block(i, n ** 3, ns)).to("cuda", torch.float32))
    Xb = [x.clone() for x in X0]
    batch = batching.Batch(ctxs)
    batch.filter(Xb, [torch.empty_like(x) for x in Xb], m, B)
    for ctx, x0, xb, b in zip(ctxs, X0, Xb, B):
        xr = x0.clone()
        ctx.cheb_filter(xr, torch.empty_like(xr), m, *b)
        assert _nrm(xb.double().cpu().numpy(), xr.double().cpu().numpy()) <= 2e-6
    small = sorted(range(64), key=lambda i: (spec[i][0], spec[i][4]))[:4]
    for i in small:
        n, R, Z, gamma, ns = spec[i]
        cl = synth.Cluster(n=n, h=0.3, R=R, Z=Z, gamma=gamma)
        H = oracle.Hamiltonian.from_cluster(cl)
        cols = [0, ns - 1]
        ref = H.cheb_filter(X0[i][cols].double().cpu().numpy(), m, *B[i])
        assert _nrm(Xb[i][cols].double().cpu().numpy(), ref) <= 1e-5
    batch.close()
    for c in ctxs:
        c.close()
