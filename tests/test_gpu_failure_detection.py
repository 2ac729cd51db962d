"""Failure detection on the GPU without a fault.

Every wait inside the library's kernels is bounded. These tests run kernels whose wait can
never complete (an mbarrier that expects an arrival nobody makes, a grid barrier that
expects one CTA more than the grid holds), check that each gives up, that the host reads
SPARC_ERR_TIMEOUT, and that the context keeps working afterwards (H X still matches the
oracle). Nothing here traps, asserts on the device or touches a bad address.
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


@pytest.fixture(scope="module")
def c24():
    w = synth.preset("cluster24")
    cl = synth.make_cluster(w, 0)
    H = oracle.Hamiltonian.from_cluster(cl)
    ctx = sparc.Context(cl.n, cl.h, cl.R, cl.Z, cl.gamma, veff=H.V, sigma=cl.sigma,
                        rcut=cl.rcut, rc_erf=cl.rc_erf)
    yield w, cl, H, ctx
    ctx.close()


def _apply_ok(w, H, ctx):
    X = synth.initial_block(3, w.nd, 4)
    Xd = torch.from_numpy(X).to("cuda:0")
    HXd = torch.empty_like(Xd)
    ctx.apply_H(Xd, HXd)
    ref = H.apply(X)
    got = HXd.cpu().numpy()
    return float(np.max(np.abs(got - ref)) / np.max(np.abs(ref)))


@pytest.mark.parametrize("which", [0, 1], ids=["mbarrier", "grid_barrier"])
def test_bounded_wait_reports_timeout_and_context_survives(c24, which):
    w, cl, H, ctx = c24
    st = ctx.selftest_timeout(which)
    assert st == sparc.SPARC_ERR_TIMEOUT
    # the flag was consumed: the next synchronisation is clean
    ctx.sync()
    assert _apply_ok(w, H, ctx) <= 1e-12
    # and the eigensolver's own grid barrier still completes afterwards
    X0 = torch.from_numpy(synth.initial_block(1, w.nd, w.ns)).to("cuda:0")
    ritz, _, _ = ctx.chefsi_step(X0, torch.empty_like(X0), w.degree, ctx.first_bounds(10, 0))
    assert np.all(np.isfinite(ritz)) and np.all(np.diff(ritz) >= 0)


def test_selftest_rejects_unknown_case(c24):
    _, _, _, ctx = c24
    assert ctx.selftest_timeout(7) == sparc.SPARC_ERR_ARG
