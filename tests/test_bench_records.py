"""The committed measurement records the bench reads stay tied to the code they describe.

The bench's roofline `traffic` is the DRAM byte count of one captured stencil launch,
stored in profiles/stencil_traffic.json with a hash of the kernel's sources; the bench
reports null when the sources have changed since the capture. These tests keep that
record current (re-capture with the command stored in the record after changing the
kernel) and check the algorithmic-byte arithmetic the fractions divide by."""
import importlib.util
import json
import os

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_stencil_traffic_record_matches_current_source(dtype):
    b = _bench()
    ent = b.stencil_traffic(dtype)
    assert ent is not None, (f"profiles/stencil_traffic.json[{dtype}] was taken on other "
                             f"sources of {b.STENCIL_SOURCES[dtype]}: re-capture it")
    # DRAM traffic within a few per cent of the algorithmic bytes of the captured launch
    assert 0.95 <= ent["dram_bytes"] / ent["algorithmic_bytes"] <= 1.1


def test_stencil_algorithmic_bytes_of_the_fp64_solve():
    # per iteration: a 2-stream first step, m - 1 3-stream steps and the 2-stream H Y_f, 8 B
    # elements, plus 8 B of potential per node and launch; k single-column Lanczos steps
    b = _bench()

    class W:
        nd, ns, degree, iters, lanczos_k = 1000, 10, 4, 3, 2

    got = b.stencil_algorithmic(W, "f64", {"stencil": (7, 1.0)}, steps=2)
    it = W.nd * W.ns * 8 * (2 + 3 * (W.degree - 1) + 2) + W.nd * (W.degree * 8 + 8)
    lz = W.lanczos_k * W.nd * 24
    assert got["bytes"] == 2 * (W.iters * it + lz)
    assert got["launches"] == 7


def test_fp32_filter_roofline_object(monkeypatch):
    # the mixed160.f32_filter object: bytes per filter = 8 B per point-orbital for the first
    # step and 12 B for each later one + 4 B of potential per node and step; achieved GB/s =
    # reps x bytes / the stencil launches' CUDA-event time; frac against the measured copy
    torch = pytest.importorskip("torch")
    b = _bench()
    monkeypatch.setattr(torch.cuda, "synchronize", lambda *a, **k: None)

    class W:
        nd, ns, degree = 4096000, 1024, 24

    class Ctx:
        calls = 0

        def profile_reset(self):
            pass

        def profile_enable(self, on=True):
            pass

        def cheb_filter(self, X, work, degree, a, b_, a0):
            Ctx.calls += 1
            assert degree == W.degree and a < b_

        def profile_read(self):
            return {"stencil": (3 * W.degree, 3 * W.degree * 13.0)}

    got = b.f32_filter_roofline(Ctx(), W, None, None, [1.0, 5.0, -1.0], reps=3)
    per = W.nd * W.ns * (2 * 4 + (W.degree - 1) * 3 * 4) + W.nd * W.degree * 4
    assert Ctx.calls == 3
    assert got["bytes_per_filter"] == per == 1191575552000
    assert got["ms_per_step"] == pytest.approx(13.0)
    assert got["achieved_gbs"] == pytest.approx(3 * per / (3 * W.degree * 13.0e-3) / 1e9)
    assert got["frac"] == pytest.approx(got["achieved_gbs"] / got["peak_gbs"])
