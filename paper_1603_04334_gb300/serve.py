"""Request loop for cluster eigensolves (binding of include/sparc_server.h) and a driver
that measures it under Poisson arrivals.

The scheduling, admission and device work all run in the library (C++ worker threads,
one CUDA stream each); this module only marshals requests and results.

    python -m paper_1603_04334_gb300.serve --rates 20,100,400 --requests 24

prints one JSON line per arrival rate: p50/p99 latency (completion - arrival), throughput,
and the same request list solved one at a time in FP64 as the baseline.
"""
from __future__ import annotations

import argparse
import ctypes as C
import json
import time
from dataclasses import dataclass
from typing import Optional

import numpy as np

from . import sparc, synth

F32, F64 = 1, 0
EXPORTS = ("sparc_request_bytes", "sparc_server_create", "sparc_server_create_batched",
           "sparc_server_destroy", "sparc_server_stats", "sparc_server_submit",
           "sparc_server_wait")


class _Request(C.Structure):
    _fields_ = [("n", C.c_int * 3), ("h", C.c_double), ("natoms", C.c_int),
                ("R", C.POINTER(C.c_double)), ("Z", C.POINTER(C.c_double)),
                ("gamma", C.POINTER(C.c_double)), ("ns", C.c_int), ("degree", C.c_int),
                ("max_iters", C.c_int), ("tol", C.c_double), ("seed", C.c_ulonglong),
                ("dtype", C.c_int), ("sim_seconds", C.c_double)]


class _Info(C.Structure):
    _fields_ = [("status", C.c_int), ("iters", C.c_int), ("converged", C.c_int),
                ("ns", C.c_int), ("t_submit", C.c_double), ("t_admit", C.c_double),
                ("t_done", C.c_double), ("est_bytes", C.c_size_t), ("used_bytes", C.c_size_t)]


def _bind(L):
    if getattr(L, "_server_bound", False):
        return L
    vp = C.c_void_p
    L.sparc_server_create.argtypes = [C.c_size_t, C.c_int, C.c_int, C.POINTER(vp)]
    L.sparc_server_create_batched.argtypes = [C.c_size_t, C.c_int, C.POINTER(vp)]
    L.sparc_request_bytes.argtypes = [C.POINTER(_Request)]
    L.sparc_request_bytes.restype = C.c_size_t
    L.sparc_server_submit.argtypes = [vp, C.POINTER(_Request), C.POINTER(C.c_longlong)]
    L.sparc_server_wait.argtypes = [vp, C.c_longlong, C.c_double, C.POINTER(_Info),
                                    C.POINTER(C.c_double), C.POINTER(C.c_double)]
    L.sparc_server_stats.argtypes = [vp, C.POINTER(C.c_longlong), C.POINTER(C.c_int),
                                     C.POINTER(C.c_size_t)]
    L.sparc_server_destroy.argtypes = [vp]
    for name in ("sparc_server_create", "sparc_server_create_batched", "sparc_server_submit",
                 "sparc_server_wait", "sparc_server_stats", "sparc_server_destroy"):
        getattr(L, name).restype = C.c_int
    L._server_bound = True
    return L


@dataclass
class Spec:
    """One eigensolve request (the fields of sparc_request)."""
    n: tuple
    h: float
    R: np.ndarray
    Z: np.ndarray
    gamma: np.ndarray
    ns: int
    degree: int = 20
    max_iters: int = 15
    tol: float = 1e-4
    seed: int = 0
    dtype: str = "f32"
    sim_seconds: float = 0.0

    def nd(self) -> int:
        return int(np.prod(self.n))

    def _c(self):
        keep = [np.ascontiguousarray(a, dtype=np.float64) for a in (self.R, self.Z, self.gamma)]
        na = int(keep[1].shape[0])
        ptr = lambda a: a.ctypes.data_as(C.POINTER(C.c_double)) if a.size else None  # noqa: E731
        r = _Request((C.c_int * 3)(*self.n), float(self.h), na, ptr(keep[0]), ptr(keep[1]),
                     ptr(keep[2]), int(self.ns), int(self.degree), int(self.max_iters),
                     float(self.tol), int(self.seed) & 0xFFFFFFFFFFFFFFFF,
                     F32 if self.dtype == "f32" else F64, float(self.sim_seconds))
        return r, keep


def request_bytes(spec: Spec) -> int:
    L = _bind(sparc.load())
    r, _keep = spec._c()
    return int(L.sparc_request_bytes(C.byref(r)))


class Server:
    """A sparc_server: `slots` workers (or, batched=True, one scheduler running rounds over
    at most `slots` active requests whose filters share launches), an HBM budget in bytes;
    simulate=True runs no GPU work (each solve sleeps spec.sim_seconds; worker mode only)."""

    def __init__(self, budget_bytes: int, slots: int = 4, simulate: bool = False,
                 batched: bool = False):
        self._L = _bind(sparc.load())
        h = C.c_void_p()
        if batched:
            if simulate:
                raise ValueError("the batched server has no simulated mode")
            st = self._L.sparc_server_create_batched(int(budget_bytes), int(slots), C.byref(h))
        else:
            st = self._L.sparc_server_create(int(budget_bytes), int(slots),
                                             int(bool(simulate)), C.byref(h))
        if st != 0:
            raise sparc.SparcError(st, "sparc_server_create")
        self._h = h

    def submit(self, spec: Spec) -> int:
        r, _keep = spec._c()
        i = C.c_longlong()
        st = self._L.sparc_server_submit(self._h, C.byref(r), C.byref(i))
        if st != 0:
            raise sparc.SparcError(st, "sparc_server_submit")
        return int(i.value)

    def wait(self, rid: int, timeout: Optional[float] = None, ns: Optional[int] = None) -> dict:
        info = _Info()
        # the result's Ns is only known once it is done: ask for the info first
        st = self._L.sparc_server_wait(self._h, rid, -1.0 if timeout is None else timeout,
                                       C.byref(info), None, None)
        if st != 0:
            raise sparc.SparcError(st, f"sparc_server_wait({rid})")
        ritz = np.zeros(info.ns)
        resid = np.zeros(info.ns)
        self._L.sparc_server_wait(self._h, rid, 0.0, C.byref(info),
                                  ritz.ctypes.data_as(C.POINTER(C.c_double)),
                                  resid.ctypes.data_as(C.POINTER(C.c_double)))
        return {"status": info.status, "iters": info.iters, "converged": bool(info.converged),
                "t_submit": info.t_submit, "t_admit": info.t_admit, "t_done": info.t_done,
                "est_bytes": int(info.est_bytes), "used_bytes": int(info.used_bytes),
                "ritz": ritz, "resid": resid}

    def stats(self) -> dict:
        c, m, p = C.c_longlong(), C.c_int(), C.c_size_t()
        self._L.sparc_server_stats(self._h, C.byref(c), C.byref(m), C.byref(p))
        return {"completed": c.value, "max_running": m.value, "peak_reserved": p.value}

    def close(self):
        if getattr(self, "_h", None):
            self._L.sparc_server_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ----------------------------------------------------------------------------------
# workload of the serving measurement and the driver
# ----------------------------------------------------------------------------------
EDGES = (48, 64, 80, 96, 112, 128)


def draw_requests(count: int, seed: int, edges=EDGES, atoms=(4, 200), states=(32, 512),
                  h: float = 0.3, degree: int = 20, iters: int = 15, tol: float = 1e-4,
                  dtype: str = "f32") -> list:
    """Requests drawn from `seed`: grid edge uniform in `edges`, atom count uniform in
    `atoms` (placed by synth.place_atoms: stops at the first atom that no longer fits),
    Ns uniform in `states` (at most Nd), Z in {1..4}, gamma in [-2, 2]."""
    g = np.random.Generator(np.random.PCG64(np.random.SeedSequence(seed).spawn(3)[2]))
    out = []
    for i in range(count):
        n = int(g.choice(edges))
        na = int(g.integers(atoms[0], atoms[1] + 1))
        R = synth.place_atoms(g, n, h, na)
        k = R.shape[0]
        Z = g.integers(1, 5, size=k).astype(np.float64)
        gl = g.uniform(-2.0, 2.0, size=(k, 2))
        gamma = np.column_stack([gl[:, 0], gl[:, 1], gl[:, 1], gl[:, 1]]) if k else np.zeros((0, 4))
        ns = int(min(g.integers(states[0], states[1] + 1), n ** 3))
        out.append(Spec((n, n, n), h, R, Z, gamma, ns, degree, iters, tol, seed * 1000 + i, dtype))
    return out


def run_arrivals(specs: list, rate: float, budget: int, slots: int, seed: int,
                 batched: bool = False) -> dict:
    """Submits `specs` at Poisson arrival times of the given rate (requests/s) and waits for
    all; latency = completion - arrival (steady-clock seconds in the library)."""
    gaps = np.random.default_rng(seed).exponential(1.0 / rate, size=len(specs))
    arrive = np.cumsum(gaps) - gaps[0]
    srv = Server(budget, slots, batched=batched)
    try:
        t0 = time.perf_counter()
        ids = []
        for t, s in zip(arrive, specs):
            d = t - (time.perf_counter() - t0)
            if d > 0:
                time.sleep(d)
            ids.append(srv.submit(s))
        res = [srv.wait(i) for i in ids]
        st = srv.stats()
    finally:
        srv.close()
    lat = np.array([r["t_done"] - r["t_submit"] for r in res])
    span = max(r["t_done"] for r in res) - min(r["t_submit"] for r in res)
    return {"results": res, "latency_s": lat, "span_s": span, "stats": st}


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__)
    ap.add_argument("--rates", default="20,100,400")
    ap.add_argument("--requests", type=int, default=24)
    ap.add_argument("--budget-gb", type=float, default=150.0)
    ap.add_argument("--slots", type=int, default=4)
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--no-baseline", action="store_true")
    a = ap.parse_args(argv)
    budget = int(a.budget_gb * 2 ** 30)
    specs = draw_requests(a.requests, a.seed)
    pts = sum((s.degree + 1) * s.nd() * s.ns for s in specs)  # per iteration, for context
    base = None
    if not a.no_baseline:
        # serial FP64 per-request solves: one slot, one request at a time
        f64 = [Spec(s.n, s.h, s.R, s.Z, s.gamma, s.ns, s.degree, s.max_iters, s.tol, s.seed,
                    "f64") for s in specs]
        srv = Server(budget, 1)
        try:
            svc = []
            for s in f64:
                r = srv.wait(srv.submit(s))
                svc.append(r["t_done"] - r["t_admit"])
        finally:
            srv.close()
        base = np.array(svc)
    for rate in (float(x) for x in a.rates.split(",")):
        m = run_arrivals(specs, rate, budget, a.slots, a.seed + 1)
        lat = m["latency_s"]
        line = {"metric": "serving latency and throughput", "rate_req_per_s": rate,
                "requests": len(specs), "slots": a.slots, "budget_gb": a.budget_gb,
                "p50_s": float(np.percentile(lat, 50)), "p99_s": float(np.percentile(lat, 99)),
                "throughput_req_per_s": len(specs) / m["span_s"],
                "max_running": m["stats"]["max_running"],
                "peak_reserved_gb": m["stats"]["peak_reserved"] / 2 ** 30,
                "converged": int(sum(r["converged"] for r in m["results"])),
                "failed": int(sum(r["status"] != 0 for r in m["results"])),
                "workload": f"edge in {list(EDGES)}, h=0.3, atoms 4-200, Ns 32-512, "
                            f"degree 20, <= 15 iterations to max residual 1e-4, mixed form",
                "block_point_orbitals_per_iteration": int(pts)}
        if base is not None:
            # the same arrivals served FIFO by serial FP64 solves (measured service times)
            gaps = np.random.default_rng(a.seed + 1).exponential(1.0 / rate, size=len(specs))
            arrive = np.cumsum(gaps) - gaps[0]
            free, blat = 0.0, []
            for t, s in zip(arrive, base):
                start = max(t, free)
                free = start + s
                blat.append(free - t)
            line["serial_fp64"] = {"throughput_req_per_s": len(specs) / float(base.sum()),
                                   "p50_s": float(np.percentile(blat, 50)),
                                   "p99_s": float(np.percentile(blat, 99))}
        print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
