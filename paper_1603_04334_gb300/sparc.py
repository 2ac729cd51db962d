"""ctypes binding of libsparc_gb300.so (the C ABI of include/sparc.h).

Argument marshalling only: every step of the computation runs in the library's CUDA
kernels. Blocks of orbitals are torch tensors of shape (ncols, ld) on the GPU
(row c = column c of the column-major Nd x ncols block), dtype float64 or float32.
There is no CPU fallback: `load()` raises if the library or a CUDA device is missing.
"""
from __future__ import annotations

import ctypes as C
import os
from typing import Optional, Sequence

import numpy as np

from . import build as _build

SPARC_OK = 0
SPARC_ERR_ARG = -1
SPARC_ERR_OOM = -2
SPARC_ERR_CUDA = -3
SPARC_ERR_NOT_SPD = -4
SPARC_ERR_NONFINITE = -5
SPARC_ERR_TIMEOUT = -6
SPARC_ERR_BUDGET = -7
SPARC_F64 = 0
SPARC_F32 = 1

_STATUS = {SPARC_ERR_ARG: "SPARC_ERR_ARG", SPARC_ERR_OOM: "SPARC_ERR_OOM",
           SPARC_ERR_CUDA: "SPARC_ERR_CUDA", SPARC_ERR_NOT_SPD: "SPARC_ERR_NOT_SPD",
           SPARC_ERR_NONFINITE: "SPARC_ERR_NONFINITE", SPARC_ERR_TIMEOUT: "SPARC_ERR_TIMEOUT",
           SPARC_ERR_BUDGET: "SPARC_ERR_BUDGET"}

# Entry points of include/sparc.h (checked by the test suite against the header).
EXPORTS = ("sparc_create", "sparc_destroy", "sparc_last_error", "sparc_get_veff", "sparc_info",
           "sparc_set_kinetic_scale", "sparc_apply_H", "sparc_lanczos_bounds",
           "sparc_first_bounds", "sparc_cheb_filter", "sparc_orth_rr", "sparc_gram",
           "sparc_chefsi_step",
           "sparc_profile_enable",
           "sparc_profile_read", "sparc_profile_reset", "sparc_launch_count",
           "sparc_gram_noalloc", "sparc_sync", "sparc_selftest_timeout",
           "sparc_gram_tc", "sparc_device_bytes", "sparc_occupations", "sparc_density",
           "sparc_nonlocal_force", "sparc_poisson")

PHASES = ("stencil", "project", "scatter", "gram", "dense", "rotate", "other")


class SparcError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{_STATUS.get(status, status)}: {msg}")
        self.status = status


class _Grid(C.Structure):
    _fields_ = [("n", C.c_int * 3), ("h", C.c_double), ("radius", C.c_int)]


class _Atoms(C.Structure):
    _fields_ = [("natoms", C.c_int), ("R", C.POINTER(C.c_double)), ("Z", C.POINTER(C.c_double)),
                ("gamma", C.POINTER(C.c_double)), ("sigma", C.c_double), ("rcut", C.c_double),
                ("rc_erf", C.c_double)]


_lib = None


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load libsparc_gb300.so (building it first if needed); raises if unavailable."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB
    if build_if_missing and (not os.path.exists(path) or _build._stale()):
        path = _build.build()
    if not os.path.exists(path):
        raise RuntimeError(f"libsparc_gb300.so not found at {path}; run build() first")
    L = C.CDLL(path)
    vp, dp, ip = C.c_void_p, C.POINTER(C.c_double), C.c_int
    L.sparc_create.argtypes = [C.POINTER(_Grid), dp, C.POINTER(_Atoms), vp, C.POINTER(vp)]
    L.sparc_destroy.argtypes = [vp]
    L.sparc_last_error.argtypes = [vp]
    L.sparc_last_error.restype = C.c_char_p
    L.sparc_get_veff.argtypes = [vp, dp]
    L.sparc_info.argtypes = [vp, C.POINTER(C.c_long), C.POINTER(C.c_long), C.POINTER(C.c_int)]
    L.sparc_set_kinetic_scale.argtypes = [vp, C.c_double]
    L.sparc_apply_H.argtypes = [vp, ip, vp, vp, ip, C.c_long]
    L.sparc_lanczos_bounds.argtypes = [vp, ip, C.c_ulonglong, dp, dp]
    L.sparc_first_bounds.argtypes = [vp, ip, C.c_ulonglong, dp]
    L.sparc_cheb_filter.argtypes = [vp, ip, vp, vp, ip, C.c_long, ip, C.c_double, C.c_double,
                                    C.c_double]
    L.sparc_orth_rr.argtypes = [vp, ip, vp, vp, ip, C.c_long, dp, dp]
    L.sparc_chefsi_step.argtypes = [vp, ip, vp, vp, ip, C.c_long, ip, dp, dp, dp]
    L.sparc_gram.argtypes = [vp, ip, vp, ip, vp, ip, C.c_long, vp]
    L.sparc_gram_tc.argtypes = [vp, ip, vp, ip, vp, ip, C.c_long, vp]
    L.sparc_profile_enable.argtypes = [vp, ip]
    L.sparc_profile_read.argtypes = [vp, ip, C.POINTER(C.c_longlong), dp]
    L.sparc_profile_reset.argtypes = [vp]
    L.sparc_launch_count.argtypes = [C.POINTER(C.c_longlong)]
    L.sparc_sync.argtypes = [vp]
    L.sparc_selftest_timeout.argtypes = [vp, ip]
    # allocation-free G = A^T B: (A, B, nd, ncols, ld, G, stream)
    L.sparc_gram_noalloc.argtypes = [vp, vp, C.c_long, ip, C.c_long, vp, vp]
    L.sparc_occupations.argtypes = [vp, dp, ip, C.c_double, C.c_double, dp, dp]
    L.sparc_density.argtypes = [vp, ip, vp, ip, C.c_long, dp, vp]
    L.sparc_nonlocal_force.argtypes = [vp, ip, vp, ip, C.c_long, dp, dp]
    L.sparc_poisson.argtypes = [vp, vp, vp, C.c_double, ip, vp, C.POINTER(C.c_int), dp]
    for name in EXPORTS:
        f = getattr(L, name)
        if name != "sparc_last_error" and f.restype is not C.c_char_p:
            f.restype = C.c_int
    _lib = L
    return L


def _dtype_code(t) -> int:
    import torch
    if t.dtype == torch.float64:
        return SPARC_F64
    if t.dtype == torch.float32:
        return SPARC_F32
    raise TypeError(f"blocks must be float64 or float32, got {t.dtype}")


def _block(t, name: str):
    if not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if t.dim() == 1:
        return 1, t.shape[0]
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous with shape (ncols, ld)")
    return t.shape[0], t.shape[1]


def _darr(a):
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a, a.ctypes.data_as(C.POINTER(C.c_double))


class Context:
    """A sparc_ctx: the discrete Hamiltonian of one cluster on the current CUDA device.

    veff: optional host array of Nd values (x fastest); when None the library builds
    V_eff = sum_J -Z_J erf(r/rc_erf)/r itself. stream: a torch.cuda.Stream (default:
    the current stream)."""

    def __init__(self, n, h: float, R=None, Z=None, gamma=None, veff=None, sigma: float = 0.8,
                 rcut: float = 3.0, rc_erf: float = 1.0, radius: int = 6, stream=None):
        import torch
        self._L = load()
        n3 = (n, n, n) if np.isscalar(n) else tuple(int(v) for v in n)
        self.n = n3
        self.nd = n3[0] * n3[1] * n3[2]
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        g = _Grid((C.c_int * 3)(*n3), float(h), int(radius))
        R = np.zeros((0, 3)) if R is None else np.asarray(R, dtype=np.float64).reshape(-1, 3)
        na = R.shape[0]
        self._R, pR = _darr(R if na else np.zeros(3))
        self._Z, pZ = _darr(np.zeros(1) if Z is None or na == 0 else Z)
        self._g, pg = _darr(np.zeros(4) if gamma is None or na == 0 else
                            np.asarray(gamma, dtype=np.float64).reshape(-1, 4))
        at = _Atoms(na, pR, pZ if Z is not None else None, pg, float(sigma), float(rcut),
                    float(rc_erf))
        pv = None
        if veff is not None:
            self._veff, pv = _darr(np.asarray(veff).reshape(-1))
            if self._veff.shape[0] != self.nd:
                raise ValueError("veff must hold Nd values")
        h_ = C.c_void_p()
        st = self._L.sparc_create(C.byref(g), pv, C.byref(at), C.c_void_p(self.stream.cuda_stream),
                                  C.byref(h_))
        if st != SPARC_OK:
            raise SparcError(st, "sparc_create failed")
        self._h = h_

    # ---- plumbing -----------------------------------------------------------------
    def _check(self, st: int):
        if st != SPARC_OK:
            msg = self._L.sparc_last_error(self._h)
            raise SparcError(st, msg.decode() if msg else "")

    def close(self):
        if getattr(self, "_h", None):
            self._L.sparc_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # ---- queries -------------------------------------------------------------------
    def get_veff(self) -> np.ndarray:
        out = np.zeros(self.nd)
        self._check(self._L.sparc_get_veff(self._h, out.ctypes.data_as(C.POINTER(C.c_double))))
        return out

    def info(self):
        nd, ns, na = C.c_long(), C.c_long(), C.c_int()
        self._check(self._L.sparc_info(self._h, C.byref(nd), C.byref(ns), C.byref(na)))
        return {"nd": nd.value, "nsupport": ns.value, "natoms": na.value}

    def set_kinetic_scale(self, kscale: float):
        self._check(self._L.sparc_set_kinetic_scale(self._h, float(kscale)))

    # ---- instrumentation -----------------------------------------------------------
    def profile_enable(self, on: bool = True):
        self._check(self._L.sparc_profile_enable(self._h, 1 if on else 0))

    def profile_reset(self):
        self._check(self._L.sparc_profile_reset(self._h))

    def sync(self):
        """Waits for the context's stream; raises SparcError (SPARC_ERR_TIMEOUT) if a kernel
        of an earlier asynchronous call gave up a bounded wait."""
        self._check(self._L.sparc_sync(self._h))

    def selftest_timeout(self, which: int) -> int:
        """Runs a kernel whose bounded wait cannot complete (0: mbarrier, 1: grid barrier)
        and returns the status code the library reports (SPARC_ERR_TIMEOUT expected)."""
        return int(self._L.sparc_selftest_timeout(self._h, int(which)))

    def profile_read(self) -> dict:
        """{phase: (launches, device ms)} accumulated since the last reset."""
        out = {}
        for i, name in enumerate(PHASES):
            n, ms = C.c_longlong(), C.c_double()
            self._check(self._L.sparc_profile_read(self._h, i, C.byref(n), C.byref(ms)))
            out[name] = (n.value, ms.value)
        return out

    # ---- the hot path ------------------------------------------------------------
    def apply_H(self, X, HX):
        ncols, ld = _block(X, "X")
        if HX.shape != X.shape or HX.dtype != X.dtype:
            raise ValueError("HX must match X in shape and dtype")
        self._check(self._L.sparc_apply_H(self._h, _dtype_code(X), C.c_void_p(X.data_ptr()),
                                          C.c_void_p(HX.data_ptr()), ncols, ld))

    def lanczos_bounds(self, k: int = 10, seed: int = 0):
        lo, hi = C.c_double(), C.c_double()
        self._check(self._L.sparc_lanczos_bounds(self._h, int(k), int(seed) & (2 ** 64 - 1),
                                                 C.byref(lo), C.byref(hi)))
        return lo.value, hi.value

    def first_bounds(self, k: int = 10, seed: int = 0) -> list:
        """[a, b, a0] for the first CheFSI iteration (sparc_first_bounds: k Lanczos steps,
        then the library's cutoff rule)."""
        out = np.zeros(3)
        self._check(self._L.sparc_first_bounds(self._h, int(k), int(seed) & (2 ** 64 - 1),
                                               out.ctypes.data_as(C.POINTER(C.c_double))))
        return [float(v) for v in out]

    def cheb_filter(self, X, work, degree: int, a: float, b: float, a0: float):
        ncols, ld = _block(X, "X")
        if work.shape != X.shape or work.dtype != X.dtype:
            raise ValueError("work must match X in shape and dtype")
        self._check(self._L.sparc_cheb_filter(self._h, _dtype_code(X), C.c_void_p(X.data_ptr()),
                                              C.c_void_p(work.data_ptr()), ncols, ld,
                                              int(degree), float(a), float(b), float(a0)))

    def orth_rr(self, Xf, HXf=None, want_resid: bool = True):
        ncols, ld = _block(Xf, "Xf")
        ritz = np.zeros(ncols)
        resid = np.zeros(ncols) if want_resid else None
        self._check(self._L.sparc_orth_rr(
            self._h, _dtype_code(Xf), C.c_void_p(Xf.data_ptr()),
            C.c_void_p(HXf.data_ptr()) if HXf is not None else None, ncols, ld,
            ritz.ctypes.data_as(C.POINTER(C.c_double)),
            resid.ctypes.data_as(C.POINTER(C.c_double)) if resid is not None else None))
        return ritz, resid

    def gram(self, A, B, G=None):
        """G = A^T B (FP64, ncols x ncols, column-major: G[j, i] in torch indexing is
        entry (i, j)); returns the device tensor G."""
        import torch
        ncols, ld = _block(A, "A")
        if B.shape != A.shape:
            raise ValueError("A and B must have the same shape")
        if G is None:
            G = torch.empty((ncols, ncols), dtype=torch.float64, device=A.device)
        self._check(self._L.sparc_gram(self._h, _dtype_code(A), C.c_void_p(A.data_ptr()),
                                       _dtype_code(B), C.c_void_p(B.data_ptr()), ncols, ld,
                                       C.c_void_p(G.data_ptr())))
        return G

    def gram_tc(self, A, B, G=None):
        """G = A^T B on the tensor cores (23-bit chunk rounding, exact accumulation; see
        sparc_gram_tc); same layout as gram()."""
        import torch
        ncols, ld = _block(A, "A")
        if B.shape != A.shape:
            raise ValueError("A and B must have the same shape")
        if G is None:
            G = torch.empty((ncols, ncols), dtype=torch.float64, device=A.device)
        self._check(self._L.sparc_gram_tc(self._h, _dtype_code(A), C.c_void_p(A.data_ptr()),
                                          _dtype_code(B), C.c_void_p(B.data_ptr()), ncols, ld,
                                          C.c_void_p(G.data_ptr())))
        return G

    def occupations(self, lam, nelec: float, kT: float = 1e-3):
        """Fermi level and occupations of the eigenvalues lam (host array):
        returns (lambda_f, g)."""
        lam, lp = _darr(lam)
        g = np.zeros(lam.shape[0])
        mu = C.c_double()
        self._check(self._L.sparc_occupations(self._h, lp, lam.shape[0], float(nelec),
                                              float(kT), C.byref(mu),
                                              g.ctypes.data_as(C.POINTER(C.c_double))))
        return mu.value, g

    def density(self, X, g, rho=None):
        """rho = (2 / h^3) sum_n g_n x_n^2 on the device (Nd doubles); returns rho."""
        import torch
        ncols, ld = _block(X, "X")
        nd = self.info()["nd"]
        if rho is None:
            rho = torch.empty(nd, dtype=torch.float64, device=X.device)
        if rho.dtype != torch.float64 or rho.numel() < nd or not rho.is_contiguous():
            raise ValueError("rho must be a contiguous float64 tensor of Nd values")
        g, gp = _darr(g)
        if g.shape[0] != ncols:
            raise ValueError("g needs one occupation per column")
        self._check(self._L.sparc_density(self._h, _dtype_code(X), C.c_void_p(X.data_ptr()),
                                          ncols, ld, gp, C.c_void_p(rho.data_ptr())))
        return rho

    def nonlocal_force(self, X, g) -> np.ndarray:
        """Non-local force on each atom, shape (natoms, 3)."""
        ncols, ld = _block(X, "X")
        natoms = self.info()["natoms"]
        g, gp = _darr(g)
        if g.shape[0] != ncols:
            raise ValueError("g needs one occupation per column")
        f = np.zeros((max(natoms, 1), 3))
        self._check(self._L.sparc_nonlocal_force(self._h, _dtype_code(X),
                                                 C.c_void_p(X.data_ptr()), ncols, ld, gp,
                                                 f.ctypes.data_as(C.POINTER(C.c_double))))
        return f[:natoms]

    def poisson(self, rho=None, phi=None, tol: float = 1e-10, maxit: int = 4000,
                want_b: bool = False):
        """Electrostatic potential on the device: returns (phi, iterations, relative
        residual) and, with want_b, the pseudocharge density as a fourth item."""
        import torch
        nd = self.info()["nd"]
        dev = torch.device("cuda", torch.cuda.current_device())
        if phi is None:
            phi = torch.empty(nd, dtype=torch.float64, device=dev)
        for t, name in ((rho, "rho"), (phi, "phi")):
            if t is not None and (t.dtype != torch.float64 or t.numel() < nd or
                                  not t.is_contiguous() or not t.is_cuda):
                raise ValueError(f"{name} must be a contiguous float64 CUDA tensor of Nd values")
        b = torch.empty(nd, dtype=torch.float64, device=phi.device) if want_b else None
        it, rel = C.c_int(), C.c_double()
        self._check(self._L.sparc_poisson(
            self._h, C.c_void_p(rho.data_ptr()) if rho is not None else None,
            C.c_void_p(phi.data_ptr()), float(tol), int(maxit),
            C.c_void_p(b.data_ptr()) if b is not None else None, C.byref(it), C.byref(rel)))
        return (phi, it.value, rel.value, b) if want_b else (phi, it.value, rel.value)

    def chefsi_step(self, X, work, degree: int, bounds: Sequence[float],
                    want_resid: bool = True):
        """One CheFSI iteration; returns (ritz, resid, new bounds [a, b, a0])."""
        ncols, ld = _block(X, "X")
        if work.shape != X.shape or work.dtype != X.dtype:
            raise ValueError("work must match X in shape and dtype")
        b = np.ascontiguousarray(bounds, dtype=np.float64).copy()
        ritz = np.zeros(ncols)
        resid = np.zeros(ncols) if want_resid else None
        self._check(self._L.sparc_chefsi_step(
            self._h, _dtype_code(X), C.c_void_p(X.data_ptr()), C.c_void_p(work.data_ptr()),
            ncols, ld, int(degree), b.ctypes.data_as(C.POINTER(C.c_double)),
            ritz.ctypes.data_as(C.POINTER(C.c_double)),
            resid.ctypes.data_as(C.POINTER(C.c_double)) if resid is not None else None))
        return ritz, resid, list(b)


def launch_count() -> int:
    """Kernels launched by libsparc_gb300 in this process so far."""
    n = C.c_longlong()
    st = load().sparc_launch_count(C.byref(n))
    if st != SPARC_OK:
        raise SparcError(st, "sparc_launch_count")
    return n.value
