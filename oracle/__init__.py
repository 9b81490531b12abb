"""Oracle: plain FP64 CPU reference for the source terms and analytical Jacobian (paper Sections 2-3).

TEST INFRASTRUCTURE ONLY. This package may be imported only by ``tests/``, the smoke check in
``__graft_entry__`` and the CPU-baseline leg of ``bench.py``. The product path (the CUDA library
and its Python binding) never imports it. It shares no code with the CUDA path.

The C implementation lives in ``pyjac_oracle.c`` (with the type-generic source terms in
``source_terms.inc``); this module compiles it on first use with gcc and wraps it with ctypes.
All arrays are host numpy float64 arrays, state-major.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "liboracle.so")
_SRC = [os.path.join(_HERE, f) for f in ("pyjac_oracle.c", "source_terms.inc", "oracle_model.h")]
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile liboracle.so with gcc (FP64, IEEE semantics, OpenMP over states)."""
    newest = max(os.path.getmtime(f) for f in _SRC)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < newest:
        tmp = _SO + ".tmp.%d" % os.getpid()
        cmd = ["gcc", "-O2", "-std=gnu11", "-fopenmp", "-fPIC", "-shared", "-fno-fast-math",
               "-ffp-contract=off", "-o", tmp, os.path.join(_HERE, "pyjac_oracle.c"), "-lm"]
        subprocess.run(cmd, check=True, cwd=_HERE)
        os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    with _lock:
        if _lib is None:
            _lib = _bind(ctypes.CDLL(build()))
    return _lib


def compile_variant(src_dir: str, out_so: str) -> str:
    """Compile the oracle sources found in src_dir (same file names) into out_so. Used by the tests
    that plant mistakes in a copy of the oracle to show that its pins catch them."""
    cmd = ["gcc", "-O2", "-std=gnu11", "-fopenmp", "-fPIC", "-shared", "-fno-fast-math", "-ffp-contract=off",
           "-o", out_so, os.path.join(src_dir, "pyjac_oracle.c"), "-lm"]
    subprocess.run(cmd, check=True, cwd=src_dir, capture_output=True)
    return out_so


def load_variant(so_path: str):
    """ctypes handle of an oracle library compiled by compile_variant (for OracleModel(lib=...))."""
    return _bind(ctypes.CDLL(os.path.abspath(so_path)))


def _bind(lib):
    vp, i64, dp, i32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p, ctypes.c_int
    lib.pjo_mech_load.argtypes = [vp, ctypes.c_size_t, ctypes.POINTER(vp)]
    lib.pjo_mech_load.restype = i32
    lib.pjo_mech_free.argtypes = [vp]
    lib.pjo_mech_free.restype = None
    lib.pjo_mech_info.argtypes = [vp, ctypes.POINTER(i32), ctypes.POINTER(i32), ctypes.POINTER(i32)]
    lib.pjo_mech_info.restype = i32
    lib.pjo_set_threads.argtypes = [i32]
    lib.pjo_set_threads.restype = None
    lib.pjo_max_threads.argtypes = []
    lib.pjo_max_threads.restype = i32
    lib.pjo_eval_dydt.argtypes = [vp, i64, dp, dp, dp, i64, dp, i64]
    lib.pjo_eval_dydt.restype = i32
    lib.pjo_eval_jacobian.argtypes = [vp, i64, dp, dp, dp, i64, dp, i64, dp, dp, i64, dp]
    lib.pjo_eval_jacobian.restype = i32
    lib.pjo_jacobian_complex_step.argtypes = [vp, i64, dp, dp, dp, i64, ctypes.c_double, dp, i64]
    lib.pjo_jacobian_complex_step.restype = i32
    lib.pjo_jacobian_fd.argtypes = [vp, i64, dp, dp, dp, i64, dp, i64, dp]
    lib.pjo_jacobian_fd.restype = i32
    lib.pjo_eval_dydt_cv.argtypes = [vp, i64, dp, dp, dp, i64, dp, i64, dp]
    lib.pjo_eval_dydt_cv.restype = i32
    lib.pjo_jacobian_cv.argtypes = [vp, i64, dp, dp, dp, i64, dp, i64, dp]
    lib.pjo_jacobian_cv.restype = i32
    lib.pjo_eval_dydt_conc.argtypes = [vp, i64, dp, dp, dp, dp, i64, dp, i64]
    lib.pjo_eval_dydt_conc.restype = i32
    lib.pjo_jacobian_conc.argtypes = [vp, i64, dp, dp, dp, dp, i64, dp, i64, dp, dp, i64, dp]
    lib.pjo_jacobian_conc.restype = i32
    lib.pjo_reaction_rates.argtypes = [vp, ctypes.c_double, ctypes.c_double, dp, dp, dp, dp, dp, dp, dp]
    lib.pjo_reaction_rates.restype = i32
    lib.pjo_species_thermo.argtypes = [vp, ctypes.c_double, dp, dp, dp, dp]
    lib.pjo_species_thermo.restype = i32
    return lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _f64(a, shape=None):
    a = np.ascontiguousarray(a, dtype=np.float64)
    if shape is not None:
        a = a.reshape(shape)
    return a


def set_threads(n: int) -> None:
    _load().pjo_set_threads(int(n))


def max_threads() -> int:
    return int(_load().pjo_max_threads())


class OracleModel:
    """A kinetic model loaded into the oracle from the binary model format."""

    def __init__(self, blob: bytes, lib=None):
        lib = lib if lib is not None else _load()
        self._lib = lib
        self._blob = bytes(blob)
        self._buf = ctypes.create_string_buffer(self._blob, len(self._blob))
        h = ctypes.c_void_p()
        rc = lib.pjo_mech_load(self._buf, len(self._blob), ctypes.byref(h))
        if rc != 0:
            raise ValueError("oracle: model load failed (status %d)" % rc)
        self._h = h
        ns, nr, ne = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        lib.pjo_mech_info(h, ctypes.byref(ns), ctypes.byref(nr), ctypes.byref(ne))
        self.n_species, self.n_reactions, self.n_elements = ns.value, nr.value, ne.value

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and getattr(self, "_lib", None) is not None:
            self._lib.pjo_mech_free(h)
            self._h = None

    # -- batch evaluations -------------------------------------------------------------------
    def dydt(self, T, P, Y):
        """f = {dT/dt, dY_1/dt..dY_N/dt} per state: (n, N+1)."""
        T, P, Y = _f64(T).ravel(), _f64(P).ravel(), _f64(Y)
        n, N = Y.shape
        out = np.empty((n, N + 1))
        rc = self._lib.pjo_eval_dydt(self._h, n, _ptr(T), _ptr(P), _ptr(Y), N, _ptr(out), N + 1)
        if rc:
            raise RuntimeError("oracle dydt failed (%d)" % rc)
        return out

    def jacobian(self, T, P, Y, with_scale: bool = False):
        """J per state: (n, N+1, N+1), plus dydt (n, N+1); with scales if requested.

        Returns (J, f) or (J, f, J_scale, f_scale). A scale entry is the sum of the absolute
        values of the terms the oracle added to form that entry."""
        T, P, Y = _f64(T).ravel(), _f64(P).ravel(), _f64(Y)
        n, N = Y.shape
        J = np.empty((n, N + 1, N + 1))
        f = np.empty((n, N + 1))
        Js = np.empty_like(J) if with_scale else None
        fs = np.empty_like(f) if with_scale else None
        rc = self._lib.pjo_eval_jacobian(self._h, n, _ptr(T), _ptr(P), _ptr(Y), N, _ptr(J), (N + 1) ** 2,
                                       _ptr(Js), _ptr(f), N + 1, _ptr(fs))
        if rc:
            raise RuntimeError("oracle jacobian failed (%d)" % rc)
        return (J, f, Js, fs) if with_scale else (J, f)

    def jacobian_complex_step(self, T, P, Y, h: float = 1e-30):
        T, P, Y = _f64(T).ravel(), _f64(P).ravel(), _f64(Y)
        n, N = Y.shape
        J = np.empty((n, N + 1, N + 1))
        rc = self._lib.pjo_jacobian_complex_step(self._h, n, _ptr(T), _ptr(P), _ptr(Y), N, h, _ptr(J),
                                               (N + 1) ** 2)
        if rc:
            raise RuntimeError("oracle complex step failed (%d)" % rc)
        return J

    def jacobian_fd(self, T, P, Y, with_scale: bool = False):
        """First-order forward-difference Jacobian (the paper's finite-difference comparison),
        (n, N+1, N+1); with_scale also returns the per-entry rounding scale (S(y+h) + S(y)) / h."""
        T, P, Y = _f64(T).ravel(), _f64(P).ravel(), _f64(Y)
        n, N = Y.shape
        J = np.empty((n, N + 1, N + 1))
        Js = np.empty_like(J) if with_scale else None
        rc = self._lib.pjo_jacobian_fd(self._h, n, _ptr(T), _ptr(P), _ptr(Y), N, _ptr(J), (N + 1) ** 2, _ptr(Js))
        if rc:
            raise RuntimeError("oracle finite-difference jacobian failed (%d)" % rc)
        return (J, Js) if with_scale else J

    def dydt_cv(self, T, rho, Y, with_scale: bool = False):
        """Constant-volume source terms {dT/dt, dY_k/dt} of states (T, rho, Y): (n, N+1); with
        with_scale also the per-entry sum of the absolute values of the terms."""
        T, rho, Y = _f64(T).ravel(), _f64(rho).ravel(), _f64(Y)
        n, N = Y.shape
        out = np.empty((n, N + 1))
        sc = np.empty_like(out) if with_scale else None
        rc = self._lib.pjo_eval_dydt_cv(self._h, n, _ptr(T), _ptr(rho), _ptr(Y), N, _ptr(out), N + 1, _ptr(sc))
        if rc:
            raise RuntimeError("oracle constant-volume dydt failed (%d)" % rc)
        return (out, sc) if with_scale else out

    def jacobian_cv(self, T, rho, Y, with_scale: bool = False):
        """Constant-volume Jacobian (n, N+1, N+1) by complex-step differentiation of the
        constant-volume source terms; with_scale also returns the per-entry rounding scale."""
        T, rho, Y = _f64(T).ravel(), _f64(rho).ravel(), _f64(Y)
        n, N = Y.shape
        J = np.empty((n, N + 1, N + 1))
        Js = np.empty_like(J) if with_scale else None
        rc = self._lib.pjo_jacobian_cv(self._h, n, _ptr(T), _ptr(rho), _ptr(Y), N, _ptr(J), (N + 1) ** 2, _ptr(Js))
        if rc:
            raise RuntimeError("oracle constant-volume jacobian failed (%d)" % rc)
        return (J, Js) if with_scale else J

    def dydt_conc(self, T, P, V, nmol):
        """Source terms of the molar-concentration basis at constant pressure: states (T, V,
        n_1..n_{N-1}) at pressure P, nmol of shape (n, N-1); returns (n, N+1) in state order
        (dT/dt, dV/dt, dn_1/dt..dn_{N-1}/dt)."""
        T, P, V, nmol = _f64(T).ravel(), _f64(P).ravel(), _f64(V).ravel(), _f64(nmol)
        n = len(T)
        N = self.n_species
        nmol = nmol.reshape(n, N - 1)
        out = np.empty((n, N + 1))
        rc = self._lib.pjo_eval_dydt_conc(self._h, n, _ptr(T), _ptr(P), _ptr(V), _ptr(nmol), N - 1, _ptr(out),
                                          N + 1)
        if rc:
            raise RuntimeError("oracle concentration-basis dydt failed (%d)" % rc)
        return out

    def jacobian_conc(self, T, P, V, nmol, with_scale: bool = False):
        """Jacobian (n, N+1, N+1) of the molar-concentration basis at constant pressure, rows and
        columns (T, V, n_1..n_{N-1}), by complex-step differentiation of its source terms; also the
        source terms. with_scale: (J, f, J_scale, f_scale) with per-entry rounding scales."""
        T, P, V, nmol = _f64(T).ravel(), _f64(P).ravel(), _f64(V).ravel(), _f64(nmol)
        n = len(T)
        N = self.n_species
        nmol = nmol.reshape(n, N - 1)
        J = np.empty((n, N + 1, N + 1))
        f = np.empty((n, N + 1))
        Js = np.empty_like(J) if with_scale else None
        fs = np.empty_like(f) if with_scale else None
        rc = self._lib.pjo_jacobian_conc(self._h, n, _ptr(T), _ptr(P), _ptr(V), _ptr(nmol), N - 1, _ptr(J),
                                         (N + 1) ** 2, _ptr(Js), _ptr(f), N + 1, _ptr(fs))
        if rc:
            raise RuntimeError("oracle concentration-basis jacobian failed (%d)" % rc)
        return (J, f, Js, fs) if with_scale else (J, f)

    # -- single-state introspection ------------------------------------------------------------
    def reaction_rates(self, T: float, P: float, Y):
        Y = _f64(Y).ravel()
        R = self.n_reactions
        kf, kr, c, Rf, Rr, q = (np.empty(R) for _ in range(6))
        rc = self._lib.pjo_reaction_rates(self._h, float(T), float(P), _ptr(Y), _ptr(kf), _ptr(kr), _ptr(c),
                                        _ptr(Rf), _ptr(Rr), _ptr(q))
        if rc:
            raise RuntimeError("oracle rates failed (%d)" % rc)
        return dict(kf=kf, kr=kr, c=c, Rf=Rf, Rr=Rr, q=q)

    def species_thermo(self, T: float):
        N = self.n_species
        cpR, HRT, SR, B = (np.empty(N) for _ in range(4))
        rc = self._lib.pjo_species_thermo(self._h, float(T), _ptr(cpR), _ptr(HRT), _ptr(SR), _ptr(B))
        if rc:
            raise RuntimeError("oracle thermo failed (%d)" % rc)
        return dict(cpR=cpR, HRT=HRT, SR=SR, B=B)


def load_model(blob: bytes, lib=None) -> OracleModel:
    return OracleModel(blob, lib=lib)
