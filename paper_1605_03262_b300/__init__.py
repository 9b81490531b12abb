"""B300-native batched FP64 chemical source terms and analytical Jacobian (pyJac, arXiv:1605.03262).

Thin Python binding of the C ABI in ``include/pyjac_b300.h`` (``libpyjacb300.so``, built for
sm_103a by :mod:`paper_1605_03262_b300.build`). PyTorch provides device memory and streams; every
step of the computation runs in the library's CUDA kernels. There is no CPU fallback: if the
library is missing or cannot be loaded, every call raises.

Main entry points:
    Model(blob)                         load a kinetic model (binary model format, see synth)
    Model.eval_dydt(T, P, Y)            source terms, (n, N+1) CUDA tensor
    Model.eval_jacobian(T, P, Y)        Jacobian (n, N+1, N+1) [and dydt] CUDA tensors
    Model.eval_jacobian_host(...)       same on host (ideally pinned) buffers, copies inside
"""
from __future__ import annotations

import ctypes
import os
import threading
from typing import Optional, Tuple

__all__ = ["Model", "BatchPlan", "LibraryError", "library", "load_library", "PJ_STATUS", "LIB_PATH"]

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libpyjacb300.so")

PJ_STATUS = {0: "PJ_OK", -1: "PJ_EINVAL", -2: "PJ_EFORMAT", -3: "PJ_ECUDA", -4: "PJ_ENOMEM", -5: "PJ_ETIMEOUT",
             -6: "PJ_EUNSUPPORTED"}


class LibraryError(RuntimeError):
    """A C-ABI call returned a negative status."""

    def __init__(self, status: int, message: str):
        super().__init__("%s (%d): %s" % (PJ_STATUS.get(status, "?"), status, message))
        self.status = status


class pj_launch(ctypes.Structure):
    _fields_ = [("warps_per_state", ctypes.c_int), ("states_per_cta", ctypes.c_int), ("ctas_per_sm", ctypes.c_int)]


class pj_batch_item(ctypes.Structure):
    _fields_ = [("mech", ctypes.c_void_p), ("n", ctypes.c_int64), ("T", ctypes.c_void_p), ("P", ctypes.c_void_p),
                ("Y", ctypes.c_void_p), ("ldy", ctypes.c_int64), ("jac", ctypes.c_void_p), ("ldj", ctypes.c_int64),
                ("dydt", ctypes.c_void_p), ("ldd", ctypes.c_int64)]


class pj_batch_shape(ctypes.Structure):
    _fields_ = [("threads_per_cta", ctypes.c_int), ("ctas_per_sm", ctypes.c_int), ("tile_states", ctypes.c_int)]


class pj_batch_item_shape(ctypes.Structure):
    _fields_ = [("warps_per_state", ctypes.c_int), ("states_per_cta", ctypes.c_int), ("tile_states", ctypes.c_int)]


_lock = threading.Lock()
_lib = None


def load_library(path: str = LIB_PATH):
    """Load libpyjacb300.so (raises if it is missing: there is no fallback)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(path):
            raise ImportError("libpyjacb300.so not found at %s; build it with "
                              "`python -m paper_1605_03262_b300.build`" % path)
        lib = ctypes.CDLL(path)
        vp, i64, i32, sz = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_size_t
        sig = {
            "pj_version": ([], i32),
            "pj_last_error": ([], ctypes.c_char_p),
            "pj_mech_load": ([vp, sz, ctypes.POINTER(vp)], i32),
            "pj_mech_load_file": ([ctypes.c_char_p, ctypes.POINTER(vp)], i32),
            "pj_mech_free": ([vp], None),
            "pj_mech_info": ([vp, ctypes.POINTER(i32), ctypes.POINTER(i32), ctypes.POINTER(sz)], i32),
            "pj_eval_dydt": ([vp, i64, vp, vp, vp, i64, vp, i64, vp], i32),
            "pj_eval_jacobian": ([vp, i64, vp, vp, vp, i64, vp, i64, vp, i64, vp], i32),
            "pj_eval_dydt_cv": ([vp, i64, vp, vp, vp, i64, vp, i64, vp], i32),
            "pj_eval_jacobian_cv": ([vp, i64, vp, vp, vp, i64, vp, i64, vp, i64, vp], i32),
            "pj_conc_pattern": ([vp, ctypes.POINTER(i64), vp, vp], i32),
            "pj_eval_jacobian_conc": ([vp, i64, vp, vp, vp, vp, i64, vp, i64, vp, i64, vp], i32),
            "pj_fd_workspace_bytes": ([vp, i64, ctypes.POINTER(sz)], i32),
            "pj_eval_jacobian_fd": ([vp, i64, vp, vp, vp, i64, vp, i64, vp, sz, vp], i32),
            "pj_eval_jacobian_host": ([vp, i64, vp, vp, vp, i64, vp, i64, vp, i64, i64], i32),
            "pj_mech_specialize": ([vp, i32], i32),
            "pj_mech_spec_info": ([vp, ctypes.POINTER(i32), ctypes.POINTER(i32), ctypes.POINTER(ctypes.c_double),
                                   ctypes.POINTER(sz)], i32),
            "pj_set_launch": ([vp, i32, ctypes.POINTER(pj_launch)], i32),
            "pj_get_launch": ([vp, i32, ctypes.POINTER(pj_launch)], i32),
            "pj_launch_smem_bytes": ([vp, i32, ctypes.POINTER(pj_launch), ctypes.POINTER(sz)], i32),
            "pj_batch_create": ([ctypes.POINTER(pj_batch_item), i32, i32, ctypes.POINTER(pj_batch_shape),
                                 ctypes.POINTER(vp)], i32),
            "pj_batch_create_ex": ([ctypes.POINTER(pj_batch_item), i32, i32, ctypes.POINTER(pj_batch_shape),
                                    ctypes.POINTER(pj_batch_item_shape), ctypes.POINTER(vp)], i32),
            "pj_batch_specialize": ([vp, i32], i32),
            "pj_batch_spec_info": ([vp, ctypes.POINTER(i32), ctypes.POINTER(i32), ctypes.POINTER(ctypes.c_double),
                                    ctypes.POINTER(sz)], i32),
            "pj_batch_run": ([vp, vp], i32),
            "pj_batch_info": ([vp, ctypes.POINTER(i32), ctypes.POINTER(sz), ctypes.POINTER(i32)], i32),
            "pj_batch_free": ([vp], None),
            "pj_batch_run_noalloc": ([ctypes.POINTER(pj_batch_item), i32, i32, i32, vp], i32),
            "pj_batch_workspace_bytes": ([], sz),
            "pj_batch_run_ws": ([ctypes.POINTER(pj_batch_item), i32, i32, i32, vp, sz, vp], i32),
        }
        for name, (args, res) in sig.items():
            fn = getattr(lib, name)
            fn.argtypes = args
            fn.restype = res
        _lib = lib
        return lib


def library():
    return load_library()


def _check(status: int):
    if status != 0:
        msg = library().pj_last_error()
        raise LibraryError(status, msg.decode() if msg else "")


def _torch():
    import torch
    return torch


def _ptr(t) -> Optional[int]:
    return None if t is None else t.data_ptr()


def _stream_handle(stream) -> Optional[int]:
    torch = _torch()
    if stream is None:
        stream = torch.cuda.current_stream()
    return stream.cuda_stream


def _as_f64_cuda(x, name, device):
    torch = _torch()
    if not isinstance(x, torch.Tensor):
        x = torch.as_tensor(x, dtype=torch.float64)
    if x.dtype != torch.float64:
        raise TypeError("%s must be float64" % name)
    if x.device.type != "cuda":
        x = x.to(device)
    return x


class Model:
    """A kinetic model resident on the current CUDA device."""

    def __init__(self, blob: bytes):
        lib = library()
        h = ctypes.c_void_p()
        buf = ctypes.create_string_buffer(bytes(blob), len(blob))
        _check(lib.pj_mech_load(buf, len(blob), ctypes.byref(h)))
        self._h = h
        ns, nr, nb = ctypes.c_int(), ctypes.c_int(), ctypes.c_size_t()
        _check(lib.pj_mech_info(h, ctypes.byref(ns), ctypes.byref(nr), ctypes.byref(nb)))
        self.n_species, self.n_reactions, self.device_bytes = ns.value, nr.value, nb.value
        torch = _torch()
        self.device = torch.device("cuda", torch.cuda.current_device())

    @classmethod
    def from_file(cls, path: str) -> "Model":
        with open(path, "rb") as f:
            return cls(f.read())

    def close(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            library().pj_mech_free(h)
        self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def handle(self) -> int:
        return self._h.value

    # -- launch shape ------------------------------------------------------------------------
    def get_launch(self, which: str = "jacobian") -> Tuple[int, int, int]:
        c = pj_launch()
        _check(library().pj_get_launch(self._h, 0 if which == "jacobian" else 1, ctypes.byref(c)))
        return c.warps_per_state, c.states_per_cta, c.ctas_per_sm

    def set_launch(self, warps_per_state: int, states_per_cta: int, ctas_per_sm: int = 1,
                   which: str = "jacobian") -> None:
        c = pj_launch(warps_per_state, states_per_cta, ctas_per_sm)
        _check(library().pj_set_launch(self._h, 0 if which == "jacobian" else 1, ctypes.byref(c)))

    def specialize(self, enable: bool = True) -> dict:
        """Compile (NVRTC) and use kernels specialised for this model and its current launch shapes;
        enable=False returns to the data-driven kernels. Returns spec_info()."""
        _check(library().pj_mech_specialize(self._h, 1 if enable else 0))
        return self.spec_info()

    def spec_info(self) -> dict:
        j, d, sec, nb = ctypes.c_int(), ctypes.c_int(), ctypes.c_double(), ctypes.c_size_t()
        _check(library().pj_mech_spec_info(self._h, ctypes.byref(j), ctypes.byref(d), ctypes.byref(sec),
                                           ctypes.byref(nb)))
        return {"jacobian": bool(j.value), "dydt": bool(d.value), "compile_seconds": sec.value,
                "cubin_bytes": nb.value}

    def launch_smem_bytes(self, warps_per_state: int, states_per_cta: int, ctas_per_sm: int = 1,
                          which: str = "jacobian") -> int:
        c = pj_launch(warps_per_state, states_per_cta, ctas_per_sm)
        b = ctypes.c_size_t()
        _check(library().pj_launch_smem_bytes(self._h, 0 if which == "jacobian" else 1, ctypes.byref(c),
                                              ctypes.byref(b)))
        return b.value

    # -- evaluation on device tensors ----------------------------------------------------------
    def _inputs(self, T, P, Y, width=None):
        T = _as_f64_cuda(T, "T", self.device).contiguous().reshape(-1)
        P = _as_f64_cuda(P, "P", self.device).contiguous().reshape(-1)
        Y = _as_f64_cuda(Y, "Y", self.device)
        width = self.n_species if width is None else width
        if Y.dim() != 2 or Y.shape[1] < width or Y.stride(1) != 1:
            raise ValueError("the per-species input must be (n, >= %d) with unit stride along species" % width)
        n = Y.shape[0]
        if T.shape[0] != n or P.shape[0] != n:
            raise ValueError("T, P and Y must describe the same number of states")
        return T, P, Y, n

    def eval_dydt(self, T, P, Y, out=None, stream=None):
        """Source terms {dT/dt, dY_1/dt..dY_N/dt} for every state: (n, N+1) float64 CUDA tensor."""
        return self._dydt(library().pj_eval_dydt, T, P, Y, out, stream)

    def eval_jacobian(self, T, P, Y, out=None, dydt: bool = False, dydt_out=None, stream=None):
        """Analytical Jacobian (n, N+1, N+1) [, dydt (n, N+1)] as float64 CUDA tensors."""
        return self._jacobian(library().pj_eval_jacobian, T, P, Y, out, dydt, dydt_out, stream)

    def eval_dydt_cv(self, T, rho, Y, out=None, stream=None):
        """Constant-volume source terms (states given by T, density rho, Y): (n, N+1) float64."""
        return self._dydt(library().pj_eval_dydt_cv, T, rho, Y, out, stream)

    def eval_jacobian_cv(self, T, rho, Y, out=None, dydt: bool = False, dydt_out=None, stream=None):
        """Constant-volume analytical Jacobian (n, N+1, N+1) [, dydt (n, N+1)] at fixed density."""
        return self._jacobian(library().pj_eval_jacobian_cv, T, rho, Y, out, dydt, dydt_out, stream)

    def conc_pattern(self):
        """CSR pattern (row_ptr (N+2,), col_idx (nnz,), int32 numpy arrays) of the molar-concentration
        basis Jacobian, rows and columns in state order (T, V, n_1..n_{N-1})."""
        import numpy as np
        nnz = ctypes.c_int64()
        _check(library().pj_conc_pattern(self._h, ctypes.byref(nnz), None, None))
        rp = np.empty(self.n_species + 2, dtype=np.int32)
        ci = np.empty(nnz.value, dtype=np.int32)
        _check(library().pj_conc_pattern(self._h, ctypes.byref(nnz), rp.ctypes.data_as(ctypes.c_void_p),
                                         ci.ctypes.data_as(ctypes.c_void_p)))
        return rp, ci

    def eval_jacobian_conc(self, T, P, V, nmol, out=None, dydt: bool = False, dydt_out=None, stream=None):
        """Sparse Jacobian of the molar-concentration basis at constant pressure for states
        (T, V, n_1..n_{N-1}) at pressures P: the values of every state's CSR entries, (n, nnz) in the
        order of conc_pattern() [, source terms (n, N+1) in state order]."""
        torch = _torch()
        N = self.n_species
        T, P, nmol, n = self._inputs(T, P, nmol, N - 1)
        V = _as_f64_cuda(V, "V", self.device).contiguous().reshape(-1)
        if V.shape[0] != n:
            raise ValueError("V must hold one volume per state")
        nnz = ctypes.c_int64()
        _check(library().pj_conc_pattern(self._h, ctypes.byref(nnz), None, None))
        if out is None:
            out = torch.empty((n, nnz.value), dtype=torch.float64, device=self.device)
        f = None
        if dydt or dydt_out is not None:
            f = dydt_out if dydt_out is not None else torch.empty((n, N + 1), dtype=torch.float64, device=self.device)
        _check(library().pj_eval_jacobian_conc(self._h, n, _ptr(T), _ptr(P), _ptr(V), _ptr(nmol), nmol.stride(0),
                                               _ptr(out), out.stride(0), _ptr(f), f.stride(0) if f is not None else 0,
                                               _stream_handle(stream)))
        return (out, f) if f is not None else out

    def _dydt(self, fn, T, P, Y, out, stream):
        torch = _torch()
        T, P, Y, n = self._inputs(T, P, Y)
        N = self.n_species
        if out is None:
            out = torch.empty((n, N + 1), dtype=torch.float64, device=self.device)
        _check(fn(self._h, n, _ptr(T), _ptr(P), _ptr(Y), Y.stride(0), _ptr(out), out.stride(0), _stream_handle(stream)))
        return out

    def _jacobian(self, fn, T, P, Y, out, dydt, dydt_out, stream):
        torch = _torch()
        T, P, Y, n = self._inputs(T, P, Y)
        N = self.n_species
        if out is None:
            out = torch.empty((n, N + 1, N + 1), dtype=torch.float64, device=self.device)
        ldj = out.stride(0)
        f = None
        if dydt or dydt_out is not None:
            f = dydt_out if dydt_out is not None else torch.empty((n, N + 1), dtype=torch.float64, device=self.device)
        _check(fn(self._h, n, _ptr(T), _ptr(P), _ptr(Y), Y.stride(0), _ptr(out), ldj, _ptr(f),
                  f.stride(0) if f is not None else 0, _stream_handle(stream)))
        return (out, f) if f is not None else out

    def fd_workspace_bytes(self, n: int) -> int:
        """Device workspace (bytes) of eval_jacobian_fd for n states in one pass."""
        b = ctypes.c_size_t()
        _check(library().pj_fd_workspace_bytes(self._h, int(n), ctypes.byref(b)))
        return b.value

    def eval_jacobian_fd(self, T, P, Y, out=None, workspace=None, stream=None):
        """First-order forward-difference Jacobian (n, N+1, N+1) (the paper's finite-difference
        comparison), from the library's source-term kernel. workspace: a CUDA uint8 tensor; a
        smaller one than fd_workspace_bytes(n) makes the library process the states in chunks."""
        torch = _torch()
        T, P, Y, n = self._inputs(T, P, Y)
        N = self.n_species
        if out is None:
            out = torch.empty((n, N + 1, N + 1), dtype=torch.float64, device=self.device)
        if workspace is None:
            workspace = torch.empty(max(8, self.fd_workspace_bytes(n)), dtype=torch.uint8, device=self.device)
        _check(library().pj_eval_jacobian_fd(self._h, n, _ptr(T), _ptr(P), _ptr(Y), Y.stride(0), _ptr(out),
                                             out.stride(0), _ptr(workspace), workspace.numel(), _stream_handle(stream)))
        return out

    # -- evaluation on host buffers (end to end) -----------------------------------------------
    def eval_jacobian_host(self, T, P, Y, jac, dydt=None, chunk_states: int = 0):
        """Jacobian of host (CPU) float64 tensors/arrays into host output ``jac`` (n, N+1, N+1).

        Copies in and out happen inside the call (pinned memory gives full bandwidth)."""
        n = Y.shape[0]
        N = self.n_species
        _check(library().pj_eval_jacobian_host(
            self._h, n, _host_ptr(T), _host_ptr(P), _host_ptr(Y), _host_stride0(Y), _host_ptr(jac),
            _host_stride0(jac), _host_ptr(dydt) if dydt is not None else None,
            _host_stride0(dydt) if dydt is not None else 0, int(chunk_states)))
        return jac


def _host_ptr(a):
    torch = _torch()
    if isinstance(a, torch.Tensor):
        if a.device.type != "cpu" or a.dtype != torch.float64:
            raise TypeError("host buffers must be float64 CPU tensors")
        return a.data_ptr()
    import numpy as np
    if a.dtype != np.float64:
        raise TypeError("host buffers must be float64")
    return a.ctypes.data


def _host_stride0(a):
    torch = _torch()
    if isinstance(a, torch.Tensor):
        return a.stride(0)
    return a.strides[0] // 8


def _batch_items(items, which: int):
    """pj_batch_item array from (Model, T, P, Y, out[, dydt_out]) tuples; returns it and the
    tensors it points into (to keep alive)."""
    keep = []
    arr = (pj_batch_item * len(items))()
    for x, item in enumerate(items):
        model, T, P, Y, out = item[:5]
        f = item[5] if len(item) > 5 else None
        T, P, Y, n = model._inputs(T, P, Y)
        keep += [model, T, P, Y, out, f]
        a = arr[x]
        a.mech = model.handle
        a.n = n
        a.T, a.P, a.Y, a.ldy = T.data_ptr(), P.data_ptr(), Y.data_ptr(), Y.stride(0)
        if which == 0:
            a.jac, a.ldj = out.data_ptr(), out.stride(0)
            a.dydt, a.ldd = (f.data_ptr(), f.stride(0)) if f is not None else (None, 0)
        else:
            a.jac, a.ldj = None, 0
            a.dydt, a.ldd = out.data_ptr(), out.stride(0)
    return arr, keep


def batch_workspace_bytes() -> int:
    return int(library().pj_batch_workspace_bytes())


def run_batch(items, which: str = "jacobian", workspace=None, tile_states: int = 0, stream=None) -> None:
    """One persistent launch over up to 64 (Model, T, P, Y, out[, dydt_out]) items without a plan:
    the item table travels in the kernel's parameter block; the tile counter goes to ``workspace``
    (a CUDA uint8 tensor of at least batch_workspace_bytes(); calls sharing one must be ordered on a
    stream) or, without one, to the library's static array (pj_batch_run_noalloc; calls must not
    overlap on the GPU)."""
    w = 0 if which == "jacobian" else 1
    arr, keep = _batch_items(items, w)
    if workspace is None:
        _check(library().pj_batch_run_noalloc(arr, len(items), w, int(tile_states), _stream_handle(stream)))
    else:
        _check(library().pj_batch_run_ws(arr, len(items), w, int(tile_states), _ptr(workspace), workspace.numel(),
                                         _stream_handle(stream)))
    del keep


class BatchPlan:
    """One persistent launch over several (model, states, outputs) items (the batched form).

    items: sequence of (Model, T, P, Y, out[, dydt_out]) with CUDA float64 tensors; for
    which="jacobian" out is (n, N+1, N+1) (dydt_out optional), for which="dydt" out is (n, N+1).
    The plan keeps pointers to these tensors: refill them in place and call run() again, or
    capture run() into a CUDA graph with capture() and replay it."""

    def __init__(self, items, which: str = "jacobian", threads_per_cta: int = 0, ctas_per_sm: int = 0,
                 tile_states: int = 0, item_shapes=None):
        """item_shapes: optional per-item (warps_per_state, states_per_cta, tile_states), 0 = default."""
        self.which = 0 if which == "jacobian" else 1
        arr, self._keep = _batch_items(items, self.which)
        shape = pj_batch_shape(threads_per_cta, ctas_per_sm, tile_states)
        h = ctypes.c_void_p()
        if item_shapes is None:
            _check(library().pj_batch_create(arr, len(items), self.which, ctypes.byref(shape), ctypes.byref(h)))
        else:
            if len(item_shapes) != len(items):
                raise ValueError("one item shape per item")
            ish = (pj_batch_item_shape * len(items))(*[pj_batch_item_shape(*map(int, x)) for x in item_shapes])
            _check(library().pj_batch_create_ex(arr, len(items), self.which, ctypes.byref(shape), ish,
                                                ctypes.byref(h)))
        self._h = h
        nt, sm, th = ctypes.c_int(), ctypes.c_size_t(), ctypes.c_int()
        _check(library().pj_batch_info(h, ctypes.byref(nt), ctypes.byref(sm), ctypes.byref(th)))
        self.n_tiles, self.smem_bytes, self.threads_per_cta = nt.value, sm.value, th.value

    def run(self, stream=None) -> None:
        _check(library().pj_batch_run(self._h, _stream_handle(stream)))

    def specialize(self, enable: bool = True) -> dict:
        """Compile (NVRTC) and use the plan's kernel specialised for its models (pj_batch_specialize);
        returns spec_info()."""
        _check(library().pj_batch_specialize(self._h, 1 if enable else 0))
        return self.spec_info()

    def spec_info(self) -> dict:
        a, n, t, b = ctypes.c_int(), ctypes.c_int(), ctypes.c_double(), ctypes.c_size_t()
        _check(library().pj_batch_spec_info(self._h, ctypes.byref(a), ctypes.byref(n), ctypes.byref(t), ctypes.byref(b)))
        return {"active": bool(a.value), "slots": n.value, "compile_seconds": t.value, "cubin_bytes": b.value}

    def capture(self):
        """CUDA graph of one run (counter reset + persistent launch); replay() re-evaluates."""
        torch = _torch()
        side = torch.cuda.Stream()
        side.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(side):
            self.run(stream=side)
        torch.cuda.current_stream().wait_stream(side)
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph):
            self.run()
        return graph

    def close(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            library().pj_batch_free(h)
        self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
