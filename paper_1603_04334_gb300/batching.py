"""Batched Chebyshev filter over many uneven clusters (binding of include/sparc_batch.h)
and a driver that compares it with per-cluster filter launches.

    python -m paper_1603_04334_gb300.batching --clusters 64

builds 64 seeded clusters (grid edge in {32, 48, 64, 80, 96}, h = 0.3 bohr, 2-60 atoms,
Ns 16-160, FP32 blocks, degree 16), autotunes the batched launch, and prints one JSON
line with the time of one batched filter (all clusters) against sparc_cheb_filter called
on each cluster in turn. The launches, work lists and graph live in the library.
"""
from __future__ import annotations

import argparse
import ctypes as C
import json
import time

import numpy as np

from . import sparc, synth

EXPORTS = ("sparc_batch_create", "sparc_batch_destroy", "sparc_batch_filter",
           "sparc_batch_tune", "sparc_batch_variant")


def _bind(L):
    if getattr(L, "_batch_bound", False):
        return L
    vp = C.c_void_p
    L.sparc_batch_create.argtypes = [C.POINTER(vp), C.c_int, vp, C.POINTER(vp)]
    L.sparc_batch_filter.argtypes = [vp, C.POINTER(vp), C.POINTER(vp), C.POINTER(C.c_int),
                                     C.POINTER(C.c_long), C.c_int, C.POINTER(C.c_double)]
    L.sparc_batch_tune.argtypes = [vp, C.POINTER(vp), C.POINTER(vp), C.POINTER(C.c_int),
                                   C.POINTER(C.c_long), C.c_int, C.POINTER(C.c_double),
                                   C.POINTER(C.c_int), C.POINTER(C.c_double)]
    L.sparc_batch_variant.argtypes = [vp, C.c_int, C.POINTER(C.c_int)]
    L.sparc_batch_destroy.argtypes = [vp]
    for n in EXPORTS:
        getattr(L, n).restype = C.c_int
    L._batch_bound = True
    return L


class Batch:
    """A sparc_batch over Context objects (FP32 blocks), on the current torch stream."""

    def __init__(self, contexts, stream=None):
        import torch
        self._L = _bind(sparc.load())
        self.contexts = list(contexts)
        hs = (C.c_void_p * len(self.contexts))(*[c._h for c in self.contexts])
        st = stream if stream is not None else torch.cuda.current_stream()
        h = C.c_void_p()
        s = self._L.sparc_batch_create(hs, len(self.contexts), C.c_void_p(st.cuda_stream),
                                       C.byref(h))
        if s != 0:
            raise sparc.SparcError(s, "sparc_batch_create")
        self._h = h

    def _args(self, X, W, bounds):
        import torch
        n = len(self.contexts)
        if len(X) != n or len(W) != n:
            raise ValueError("one X and one W block per cluster")
        for x, w in zip(X, W):
            if x.dtype != torch.float32 or w.shape != x.shape or w.dtype != x.dtype:
                raise ValueError("FP32 blocks of matching shape expected")
        xs = (C.c_void_p * n)(*[x.data_ptr() for x in X])
        ws = (C.c_void_p * n)(*[w.data_ptr() for w in W])
        nc = (C.c_int * n)(*[x.shape[0] for x in X])
        ld = (C.c_long * n)(*[x.shape[1] for x in X])
        b = np.ascontiguousarray(np.asarray(bounds, dtype=np.float64).reshape(n, 3))
        return xs, ws, nc, ld, b

    def filter(self, X, W, degree: int, bounds):
        """bounds: per cluster (a, b, a0)."""
        xs, ws, nc, ld, b = self._args(X, W, bounds)
        s = self._L.sparc_batch_filter(self._h, xs, ws, nc, ld, int(degree),
                                       b.ctypes.data_as(C.POINTER(C.c_double)))
        if s != 0:
            raise sparc.SparcError(s, "sparc_batch_filter")

    def tune(self, X, W, degree: int, bounds):
        """Autotunes the launch variant (X is overwritten); returns (variant, ms)."""
        xs, ws, nc, ld, b = self._args(X, W, bounds)
        v, ms = C.c_int(), C.c_double()
        s = self._L.sparc_batch_tune(self._h, xs, ws, nc, ld, int(degree),
                                     b.ctypes.data_as(C.POINTER(C.c_double)), C.byref(v),
                                     C.byref(ms))
        if s != 0:
            raise sparc.SparcError(s, "sparc_batch_tune")
        return v.value, ms.value

    def set_variant(self, v: int) -> int:
        cnt = C.c_int()
        s = self._L.sparc_batch_variant(self._h, int(v), C.byref(cnt))
        if s != 0:
            raise sparc.SparcError(s, "sparc_batch_variant")
        return cnt.value

    def close(self):
        if getattr(self, "_h", None):
            self._L.sparc_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def draw_clusters(count: int, seed: int, edges=(32, 48, 64, 80, 96), atoms=(2, 60),
                  states=(16, 160), h: float = 0.3):
    """(n, R, Z, gamma, Ns) per cluster from `seed` (placement as synth.place_atoms)."""
    g = np.random.Generator(np.random.PCG64(np.random.SeedSequence(seed).spawn(4)[3]))
    out = []
    for _ in range(count):
        n = int(g.choice(edges))
        R = synth.place_atoms(g, n, h, int(g.integers(atoms[0], atoms[1] + 1)))
        k = R.shape[0]
        Z = g.integers(1, 5, size=k).astype(np.float64)
        gl = g.uniform(-2.0, 2.0, size=(k, 2))
        gamma = np.column_stack([gl[:, 0], gl[:, 1], gl[:, 1], gl[:, 1]]) if k else np.zeros((0, 4))
        out.append((n, R, Z, gamma, int(g.integers(states[0], states[1] + 1))))
    return out


def compare(clusters: int = 64, seed: int = 0, degree: int = 16, reps: int = 5,
            edges=(32, 48, 64, 80, 96)) -> dict:
    """One batched filter of `clusters` seeded clusters (autotuned launch) against
    sparc_cheb_filter on each cluster in turn: best of `reps` CUDA-event timings of each
    after a warm-up (the warm-up captures the batch's graph)."""
    import torch
    h = 0.3
    spec = draw_clusters(clusters, seed, edges=edges)
    ctxs, X, W, bounds = [], [], [], []
    for i, (n, R, Z, gamma, ns) in enumerate(spec):
        ctx = sparc.Context(n, h, R, Z, gamma)
        ctxs.append(ctx)
        bounds.append(ctx.first_bounds(10, i))
        x0 = torch.from_numpy(synth.initial_block(seed + i, n ** 3, ns)).to("cuda",
                                                                         torch.float32)
        X.append(x0)
        W.append(torch.empty_like(x0))
    X0 = [x.clone() for x in X]
    batch = Batch(ctxs)
    variant, tune_ms = batch.tune(X, W, degree, bounds)
    st = torch.cuda.current_stream()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def timed(fn):
        for x, x0 in zip(X, X0):
            x.copy_(x0)
        fn()  # warm-up (graph capture for the batch)
        torch.cuda.synchronize()
        best = None
        for _ in range(reps):
            for x, x0 in zip(X, X0):
                x.copy_(x0)
            torch.cuda.synchronize()
            ev0.record(st)
            fn()
            ev1.record(st)
            torch.cuda.synchronize()
            t = ev0.elapsed_time(ev1)
            best = t if best is None else min(best, t)
        return best

    t_batch = timed(lambda: batch.filter(X, W, degree, bounds))
    t_each = timed(lambda: [c.cheb_filter(x, w, degree, *b)
                            for c, x, w, b in zip(ctxs, X, W, bounds)])
    ptorb = sum(degree * n ** 3 * ns for (n, _, _, _, ns) in spec)
    batch.close()
    for c in ctxs:
        c.close()
    return {"clusters": clusters, "degree": degree, "variant": variant,
            "batched_ms": t_batch, "per_cluster_ms": t_each, "speedup": t_each / t_batch,
            "batched_ptorb_per_s": ptorb / (t_batch / 1e3),
            "per_cluster_ptorb_per_s": ptorb / (t_each / 1e3),
            "workload": f"edge in {{{','.join(str(e) for e in edges)}}}, h=0.3, atoms 2-60, "
                        f"Ns 16-160, FP32, degree {degree}",
            "tune_ms": tune_ms}


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__)
    ap.add_argument("--clusters", type=int, default=64)
    ap.add_argument("--degree", type=int, default=16)
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--reps", type=int, default=5)
    ap.add_argument("--edges", default="32,48,64,80,96")
    a = ap.parse_args(argv)
    out = compare(a.clusters, a.seed, a.degree, a.reps,
                  tuple(int(e) for e in a.edges.split(",")))
    print(json.dumps(dict(out, metric="batched Chebyshev filter, many uneven clusters")),
          flush=True)


if __name__ == "__main__":
    main()
