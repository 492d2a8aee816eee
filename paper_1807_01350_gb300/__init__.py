"""Python binding of the GB300 OCTen online CP update library.

Argument marshalling only: every step of the update runs in the CUDA library
(`_build/libocten.so`, C ABI in include/octen.h).  Arrays may be torch tensors
(CUDA or CPU) or numpy arrays; CPU arrays are copied to the device by the
library itself.  There is no fallback: if the library is missing or fails to
load, every call raises.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

__all__ = ["Octen", "OctenN", "OctenError", "append_many", "compress", "lib", "library_path",
           "PREC", "launch_count"]

PREC = {"fp32": 0, "bf16": 1, "fp8": 2}
_STATUS = {0: "OCTEN_OK", 1: "OCTEN_EINVAL", 2: "OCTEN_ENOMEM", 3: "OCTEN_ECUDA",
           4: "OCTEN_ETIMEOUT", 5: "OCTEN_ENUMERIC", 6: "OCTEN_ESTATE"}


class OctenError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{_STATUS.get(status, status)}: {msg}")
        self.status = status


MAX_MODES = 6


class _NConfig(ctypes.Structure):
    _fields_ = [("N", ctypes.c_int32), ("R", ctypes.c_int32), ("P", ctypes.c_int32),
                ("Q", ctypes.c_int32), ("S", ctypes.c_int32), ("als_iters", ctypes.c_int32),
                ("dims", ctypes.c_int64 * (MAX_MODES - 1)), ("prec", ctypes.c_int32)]


class _Config(ctypes.Structure):
    _fields_ = [("I", ctypes.c_int64), ("J", ctypes.c_int64), ("R", ctypes.c_int32),
                ("P", ctypes.c_int32), ("Q", ctypes.c_int32), ("S", ctypes.c_int32),
                ("als_iters", ctypes.c_int32), ("prec", ctypes.c_int32)]


_LIB = None


def library_path() -> str:
    return _build.LIB


def lib() -> ctypes.CDLL:
    """The loaded CUDA library (build it first with `build.build()`)."""
    global _LIB
    if _LIB is None:
        path = library_path()
        if not os.path.exists(path):
            raise OctenError(3, f"CUDA library not built: {path} is missing "
                                "(run paper_1807_01350_gb300.build.build())")
        L = ctypes.CDLL(path)
        vp, i64, f32p = ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p
        L.octen_create.argtypes = [ctypes.POINTER(_Config), vp, ctypes.POINTER(vp)]
        L.octen_init.argtypes = [vp, vp, i64, f32p, f32p, f32p, f32p, f32p, f32p]
        L.octen_append.argtypes = [vp, vp, i64, f32p]
        L.octen_append_many.argtypes = [vp, ctypes.c_int, vp, vp, vp]
        L.octen_append_async.argtypes = [vp, vp, i64, f32p, f32p, f32p, f32p,
                                         ctypes.POINTER(i64)]
        L.octen_wait.argtypes = [vp, i64]
        L.octen_get_factors.argtypes = [vp, f32p, f32p, f32p, ctypes.POINTER(i64)]
        L.octen_rows.argtypes = [vp]
        L.octen_rows.restype = i64
        L.octen_device_bytes.argtypes = [vp]
        L.octen_device_bytes.restype = ctypes.c_uint64
        L.octen_fit.argtypes = [vp, vp, i64, ctypes.POINTER(ctypes.c_double)]
        L.octen_get_replicas.argtypes = [vp, f32p]
        L.octen_get_replica_factors.argtypes = [vp, ctypes.c_int, f32p, f32p, f32p, vp, vp]
        L.octen_compress.argtypes = [ctypes.POINTER(_Config), vp, vp, i64, f32p, f32p, f32p, f32p]
        L.octen_compress_noalloc.argtypes = [ctypes.POINTER(_Config), vp, vp, i64, f32p, f32p,
                                             f32p, f32p]
        L.octen_save.argtypes = [vp, ctypes.c_char_p]
        L.octen_load.argtypes = [ctypes.c_char_p, vp, ctypes.POINTER(vp)]
        L.octen_destroy.argtypes = [vp]
        L.octen_destroy.restype = None
        L.octen_last_error.argtypes = [vp]
        L.octen_last_error.restype = ctypes.c_char_p
        L.octen_status_name.argtypes = [ctypes.c_int]
        L.octen_status_name.restype = ctypes.c_char_p
        L.octen_launch_count.argtypes = []
        L.octen_launch_count.restype = ctypes.c_uint64
        L.octen_tc_launch_count.argtypes = []
        L.octen_tc_launch_count.restype = ctypes.c_uint64
        L.octen_tc_fallback_count.argtypes = []
        L.octen_tc_fallback_count.restype = ctypes.c_uint64
        L.octen_stage_count.argtypes = []
        L.octen_stage_count.restype = ctypes.c_int
        L.octen_stage_name.argtypes = [ctypes.c_int]
        L.octen_stage_name.restype = ctypes.c_char_p
        L.octen_set_timing.argtypes = [vp, ctypes.c_int]
        L.octen_stage_times.argtypes = [vp, vp, vp]
        L.octen_reset_stage_times.argtypes = [vp]
        L.octen_n_create.argtypes = [ctypes.POINTER(_NConfig), vp, ctypes.POINTER(vp)]
        L.octen_n_init.argtypes = [vp, vp, i64, vp, f32p, vp, f32p]
        L.octen_n_append.argtypes = [vp, vp, i64, f32p]
        L.octen_n_get_factors.argtypes = [vp, vp, f32p, ctypes.POINTER(i64)]
        L.octen_n_get_replicas.argtypes = [vp, f32p]
        L.octen_n_get_replica_factors.argtypes = [vp, ctypes.c_int, vp, vp, vp]
        L.octen_n_rows.argtypes = [vp]
        L.octen_n_rows.restype = i64
        L.octen_n_fit.argtypes = [vp, f32p, i64, ctypes.POINTER(ctypes.c_double)]
        L.octen_n_save.argtypes = [vp, ctypes.c_char_p]
        L.octen_n_load.argtypes = [ctypes.c_char_p, vp, ctypes.POINTER(vp)]
        L.octen_n_destroy.argtypes = [vp]
        L.octen_n_destroy.restype = None
        L.octen_n_last_error.argtypes = [vp]
        L.octen_n_last_error.restype = ctypes.c_char_p
        L.octen_n_stage_count.argtypes = []
        L.octen_n_stage_count.restype = ctypes.c_int
        L.octen_n_stage_name.argtypes = [ctypes.c_int]
        L.octen_n_stage_name.restype = ctypes.c_char_p
        L.octen_n_set_timing.argtypes = [vp, ctypes.c_int]
        L.octen_n_stage_times.argtypes = [vp, vp, vp]
        for name in ("octen_n_create", "octen_n_init", "octen_n_append", "octen_n_get_factors",
                     "octen_n_get_replicas", "octen_n_get_replica_factors",
                     "octen_n_set_timing", "octen_n_stage_times", "octen_n_fit",
                     "octen_n_save", "octen_n_load"):
            getattr(L, name).restype = ctypes.c_int
        for name in ("octen_create", "octen_init", "octen_append", "octen_append_many",
                     "octen_append_async", "octen_wait",
                     "octen_get_factors",
                     "octen_fit", "octen_get_replicas", "octen_get_replica_factors",
                     "octen_compress", "octen_compress_noalloc", "octen_set_timing",
                     "octen_save", "octen_load",
                     "octen_stage_times",
                     "octen_reset_stage_times"):
            getattr(L, name).restype = ctypes.c_int
        _LIB = L
    return _LIB


def launch_count() -> int:
    return int(lib().octen_launch_count())


def tc_launch_count() -> int:
    return int(lib().octen_tc_launch_count())


def tc_fallback_count() -> int:
    """Wanted tensor-core contractions that ran on the SIMT kernels instead."""
    return int(lib().octen_tc_fallback_count())


def _stream_handle(stream) -> int | None:
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return int(stream.cuda_stream)


def _ptr(a, keep: list):
    """Pointer to the data of a torch tensor or numpy array (contiguous)."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        a = np.ascontiguousarray(a)
        keep.append(a)
        return a.ctypes.data
    if not a.is_contiguous():
        a = a.contiguous()
    keep.append(a)
    return a.data_ptr()


def _numel(a) -> int:
    return int(a.size) if isinstance(a, np.ndarray) else int(a.numel())


def _need(a, count: int, what: str, required: bool = True):
    """The library reads exactly `count` elements behind each array pointer:
    an array of another size is refused here (EINVAL), before a kernel could
    read past its end."""
    if a is None:
        if required:
            raise OctenError(1, f"{what} is required")
        return
    if _numel(a) != count:
        raise OctenError(1, f"{what}: {_numel(a)} elements, expected {count}")


def _out(a, count: int, what: str):
    """A destination buffer: contiguous fp32 of exactly `count` elements (a
    converted copy would receive the result instead of the caller's array)."""
    if a is None:
        return
    _need(a, count, what)
    if isinstance(a, np.ndarray):
        ok = a.dtype == np.float32 and a.flags["C_CONTIGUOUS"] and a.flags["WRITEABLE"]
    else:
        import torch
        ok = a.dtype == torch.float32 and a.is_contiguous()
    if not ok:
        raise OctenError(1, f"{what}: must be a contiguous, writable float32 array")


def _as_is(a, dtype: str, what: str):
    """An array the library reads after the call returns: it must be passed
    as it is (contiguous, of the element type the library reads), since a
    converted copy would be freed before the library reads it."""
    if isinstance(a, np.ndarray):
        ok = a.dtype == np.dtype(dtype) if dtype != "bfloat16" else False
        ok = ok and a.flags["C_CONTIGUOUS"]
    else:
        import torch
        ok = a.dtype == getattr(torch, dtype) and a.is_contiguous()
    if not ok:
        raise OctenError(1, f"{what}: must be a contiguous {dtype} array")


def _f32(a, keep: list):
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        return _ptr(np.ascontiguousarray(a, dtype=np.float32), keep)
    import torch
    return _ptr(a.to(torch.float32), keep)


def _slices(a, prec: str, keep: list):
    """Slice batch in the element type the precision takes (fp32 or bf16)."""
    if isinstance(a, np.ndarray):
        if prec == "fp32":
            return _ptr(np.ascontiguousarray(a, dtype=np.float32), keep)
        import torch
        a = torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32))
    import torch
    want = torch.float32 if prec == "fp32" else torch.bfloat16
    return _ptr(a.to(want), keep)


class Octen:
    """One online CP decomposition (see include/octen.h)."""

    def __init__(self, I, J, R, P, Q, S, als_iters, prec="fp32", stream=None):
        self._lib = lib()
        self.prec = prec
        self.cfg = _Config(int(I), int(J), int(R), int(P), int(Q), int(S), int(als_iters),
                           PREC[prec])
        self.I, self.J, self.R, self.P, self.Q, self.S = I, J, R, P, Q, S
        self.Qd = S + P * (Q - S)
        h = ctypes.c_void_p()
        st = self._lib.octen_create(ctypes.byref(self.cfg), _stream_handle(stream),
                                    ctypes.byref(h))
        if st != 0:
            raise OctenError(st, "octen_create failed")
        self._h = h

    def _check(self, st: int):
        if st != 0:
            raise OctenError(st, self._lib.octen_last_error(self._h).decode())

    def init(self, X_old, U_all, V_all, W_old, A0, B0, C0=None):
        """octen_init; with C0 None the existing decomposition is computed on
        the GPU by CP-ALS of X_old from the starting guesses A0, B0."""
        keep: list = []
        t_old = int(X_old.shape[0])
        I, J, R, Qd = self.I, self.J, self.R, self.Qd
        _need(X_old, t_old * I * J, "X_old")
        _need(U_all, I * Qd, "U_all")
        _need(V_all, J * Qd, "V_all")
        _need(W_old, t_old * Qd, "W_old")
        _need(A0, I * R, "A0")
        _need(B0, J * R, "B0")
        _need(C0, t_old * R, "C0", required=False)
        self._check(self._lib.octen_init(
            self._h, _slices(X_old, self.prec, keep), t_old, _f32(U_all, keep),
            _f32(V_all, keep), _f32(W_old, keep), _f32(A0, keep), _f32(B0, keep),
            _f32(C0, keep)))

    def append(self, X_new, W_new):
        keep: list = []
        t = int(X_new.shape[0])
        _need(X_new, t * self.I * self.J, "X_new")
        _need(W_new, t * self.Qd, "W_new")
        self._check(self._lib.octen_append(self._h, _slices(X_new, self.prec, keep),
                                           int(X_new.shape[0]), _f32(W_new, keep)))

    def append_ptr(self, x_ptr: int, t: int, w_ptr: int):
        """Append from raw pointers (device or host) already in the right types."""
        self._check(self._lib.octen_append(self._h, x_ptr, int(t), w_ptr))

    def append_async(self, X_new, W_new, A_out=None, B_out=None, C_new_out=None) -> int:
        """octen_append_async: enqueue an append and return its ticket.  X_new
        must already be in the precision's element type (fp32, or bf16 for the
        bf16 / fp8 modes) and stay alive and unchanged, with W_new, until
        wait(ticket); the optional fp32 outputs receive A, B and the new rows
        of C once the append has run."""
        t = int(X_new.shape[0])
        _need(X_new, t * self.I * self.J, "X_new")
        _need(W_new, t * self.Qd, "W_new")
        _as_is(X_new, "float32" if self.prec == "fp32" else "bfloat16", "X_new")
        _as_is(W_new, "float32", "W_new")
        _out(A_out, self.I * self.R, "A_out")
        _out(B_out, self.J * self.R, "B_out")
        _out(C_new_out, t * self.R, "C_new_out")
        return self.append_async_ptr(_ptr(X_new, []), t, _ptr(W_new, []), _ptr(A_out, []),
                                     _ptr(B_out, []), _ptr(C_new_out, []))

    def append_async_ptr(self, x_ptr, t, w_ptr, a_ptr=None, b_ptr=None, c_ptr=None) -> int:
        """octen_append_async from raw pointers; returns the ticket."""
        tk = ctypes.c_int64()
        self._check(self._lib.octen_append_async(self._h, x_ptr, int(t), w_ptr, a_ptr, b_ptr,
                                                 c_ptr, ctypes.byref(tk)))
        return int(tk.value)

    def wait(self, ticket: int):
        """octen_wait: block until the append of `ticket` has run."""
        self._check(self._lib.octen_wait(self._h, int(ticket)))

    @property
    def rows(self) -> int:
        return int(self._lib.octen_rows(self._h))

    @property
    def device_bytes(self) -> int:
        """Bytes of device memory the context holds (octen_device_bytes)."""
        return int(self._lib.octen_device_bytes(self._h))

    def factors(self):
        K = self.rows
        A = np.empty((self.I, self.R), np.float32)
        B = np.empty((self.J, self.R), np.float32)
        C = np.empty((K, self.R), np.float32)
        k = ctypes.c_int64()
        self._check(self._lib.octen_get_factors(self._h, A.ctypes.data, B.ctypes.data,
                                                C.ctypes.data, ctypes.byref(k)))
        return A, B, C

    def factors_into(self, A, B, C):
        """Copy the factors into caller buffers (torch device tensors allowed)."""
        keep: list = []
        _out(A, self.I * self.R, "A")
        _out(B, self.J * self.R, "B")
        _out(C, self.rows * self.R, "C")
        k = ctypes.c_int64()
        self._check(self._lib.octen_get_factors(self._h, _ptr(A, keep), _ptr(B, keep),
                                                _ptr(C, keep), ctypes.byref(k)))
        return int(k.value)

    def fit(self, X_all) -> float:
        keep: list = []
        out = ctypes.c_double()
        _need(X_all, int(X_all.shape[0]) * self.I * self.J, "X_all")
        self._check(self._lib.octen_fit(self._h, _slices(X_all, self.prec, keep),
                                        int(X_all.shape[0]), ctypes.byref(out)))
        return float(out.value)

    def replicas(self):
        Y = np.empty((self.P, self.Q, self.Q, self.Q), np.float32)
        self._check(self._lib.octen_get_replicas(self._h, Y.ctypes.data))
        return Y

    def replica_factors(self, which: int = 0):
        shp = (self.P, self.Q, self.R)
        At, Bt, Ct = (np.empty(shp, np.float32) for _ in range(3))
        perm = np.empty((self.P, self.R), np.int32)
        scales = np.empty((self.P, 2, self.R), np.float64)
        self._check(self._lib.octen_get_replica_factors(
            self._h, int(which), At.ctypes.data, Bt.ctypes.data, Ct.ctypes.data,
            perm.ctypes.data, scales.ctypes.data))
        return At, Bt, Ct, perm, scales

    def save(self, path: str):
        """Checkpoint the whole state to `path`."""
        self._check(self._lib.octen_save(self._h, os.fsencode(path)))

    @classmethod
    def load(cls, path: str, stream=None) -> "Octen":
        """A context resumed from a checkpoint written by `save`."""
        L = lib()
        h = ctypes.c_void_p()
        st = L.octen_load(os.fsencode(path), _stream_handle(stream), ctypes.byref(h))
        if st != 0:
            raise OctenError(st, f"octen_load({path!r}) failed")
        self = cls.__new__(cls)
        self._lib = L
        self._h = h
        # read the shape back from the file header (magic, then octen_config)
        with open(path, "rb") as f:
            f.read(8)
            cfg = _Config.from_buffer_copy(f.read(ctypes.sizeof(_Config)))
        self.cfg = cfg
        self.prec = {v: k for k, v in PREC.items()}[cfg.prec]
        self.I, self.J, self.R, self.P, self.Q, self.S = cfg.I, cfg.J, cfg.R, cfg.P, cfg.Q, cfg.S
        self.Qd = cfg.S + cfg.P * (cfg.Q - cfg.S)
        return self

    def set_timing(self, on: bool = True):
        self._check(self._lib.octen_set_timing(self._h, int(bool(on))))

    def reset_stage_times(self):
        self._check(self._lib.octen_reset_stage_times(self._h))

    def stage_times(self) -> dict:
        """{stage: (milliseconds, timed intervals)} accumulated while timing is on."""
        n = self._lib.octen_stage_count()
        ms = np.zeros(n, np.float64)
        cnt = np.zeros(n, np.uint64)
        self._check(self._lib.octen_stage_times(self._h, ms.ctypes.data, cnt.ctypes.data))
        return {self._lib.octen_stage_name(i).decode(): (float(ms[i]), int(cnt[i]))
                for i in range(n)}

    def close(self):
        if getattr(self, "_h", None):
            self._lib.octen_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class OctenN:
    """One online CP decomposition of an N-mode tensor growing in its last
    (time) mode (octen_n_* in include/octen.h), fp32 or bf16 slices.  dims are
    the N - 1 non-temporal sizes; slices are [k][i_1]...[i_{N-1}]."""

    def __init__(self, dims, R, P, Q, S, als_iters, prec="fp32", stream=None):
        self._lib = lib()
        if prec not in ("fp32", "bf16"):
            raise OctenError(1, f"N-mode precision {prec!r}: fp32 or bf16")
        self.prec = prec
        self.dims = [int(d) for d in dims]
        self.N = len(self.dims) + 1
        if not 3 <= self.N <= MAX_MODES:
            raise OctenError(1, f"N = {self.N} modes: 3 <= N <= {MAX_MODES}")
        dd = (ctypes.c_int64 * (MAX_MODES - 1))(*(self.dims + [0] * (MAX_MODES - self.N)))
        self.cfg = _NConfig(self.N, int(R), int(P), int(Q), int(S), int(als_iters), dd,
                            PREC[prec])
        self.R, self.P, self.Q, self.S = R, P, Q, S
        self.Qd = S + P * (Q - S)
        h = ctypes.c_void_p()
        st = self._lib.octen_n_create(ctypes.byref(self.cfg), _stream_handle(stream),
                                      ctypes.byref(h))
        if st != 0:
            raise OctenError(st, "octen_n_create failed")
        self._h = h

    def _check(self, st: int):
        if st != 0:
            raise OctenError(st, self._lib.octen_n_last_error(self._h).decode())

    @property
    def _slice(self) -> int:
        """Elements of one slice (I_1 x ... x I_{N-1})."""
        return int(np.prod(self.dims, dtype=np.int64))

    def _ptrs(self, arrays, keep):
        return (ctypes.c_void_p * len(arrays))(*[_f32(a, keep) for a in arrays])

    def init(self, X_old, Us, W_old, A0s, C0):
        keep: list = []
        t_old = int(X_old.shape[0])
        nm = self.N - 1
        if len(Us) != nm or len(A0s) != nm:
            raise OctenError(1, f"{nm} projections and {nm} factors expected")
        _need(X_old, t_old * self._slice, "X_old")
        for n in range(nm):
            _need(Us[n], self.dims[n] * self.Qd, f"U_all[{n}]")
            _need(A0s[n], self.dims[n] * self.R, f"A0[{n}]")
        _need(W_old, t_old * self.Qd, "W_old")
        _need(C0, t_old * self.R, "C0", required=False)
        us = self._ptrs(Us, keep)
        a0 = self._ptrs(A0s, keep)
        keep += [us, a0]
        self._check(self._lib.octen_n_init(self._h, _slices(X_old, self.prec, keep),
                                           int(X_old.shape[0]), us, _f32(W_old, keep), a0,
                                           _f32(C0, keep)))

    def append(self, X_new, W_new):
        keep: list = []
        t = int(X_new.shape[0])
        _need(X_new, t * self._slice, "X_new")
        _need(W_new, t * self.Qd, "W_new")
        self._check(self._lib.octen_n_append(self._h, _slices(X_new, self.prec, keep),
                                             int(X_new.shape[0]), _f32(W_new, keep)))

    def append_ptr(self, x_ptr: int, t: int, w_ptr: int):
        """Append from raw fp32 pointers (device or host)."""
        self._check(self._lib.octen_n_append(self._h, x_ptr, int(t), w_ptr))

    @property
    def rows(self) -> int:
        return int(self._lib.octen_n_rows(self._h))

    def factors(self):
        """([A_1, ..., A_{N-1}], C) as numpy arrays."""
        As = [np.empty((d, self.R), np.float32) for d in self.dims]
        C = np.empty((self.rows, self.R), np.float32)
        ap = (ctypes.c_void_p * len(As))(*[a.ctypes.data for a in As])
        k = ctypes.c_int64()
        self._check(self._lib.octen_n_get_factors(self._h, ap, C.ctypes.data, ctypes.byref(k)))
        return As, C

    def save(self, path: str):
        """Checkpoint the whole state to `path` (octen_n_save)."""
        self._check(self._lib.octen_n_save(self._h, os.fsencode(path)))

    @classmethod
    def load(cls, path: str, stream=None) -> "OctenN":
        """A context resumed from a checkpoint written by `save`."""
        L = lib()
        h = ctypes.c_void_p()
        st = L.octen_n_load(os.fsencode(path), _stream_handle(stream), ctypes.byref(h))
        if st != 0:
            raise OctenError(st, f"octen_n_load({path!r}) failed")
        self = cls.__new__(cls)
        self._lib = L
        self._h = h
        with open(path, "rb") as f:   # the shape, from the header (magic, then octen_nconfig)
            f.read(8)
            cfg = _NConfig.from_buffer_copy(f.read(ctypes.sizeof(_NConfig)))
        self.cfg = cfg
        self.prec = {v: k for k, v in PREC.items()}[cfg.prec]
        self.N = cfg.N
        self.dims = [int(cfg.dims[n]) for n in range(cfg.N - 1)]
        self.R, self.P, self.Q, self.S = cfg.R, cfg.P, cfg.Q, cfg.S
        self.Qd = cfg.S + cfg.P * (cfg.Q - cfg.S)
        return self

    def fit(self, X_all) -> float:
        """Fitness of the current factors on all slices so far (octen_n_fit)."""
        keep: list = []
        out = ctypes.c_double()
        _need(X_all, int(X_all.shape[0]) * self._slice, "X_all")
        self._check(self._lib.octen_n_fit(self._h, _slices(X_all, self.prec, keep),
                                          int(X_all.shape[0]), ctypes.byref(out)))
        return float(out.value)

    def replicas(self):
        Y = np.empty((self.P,) + (self.Q,) * self.N, np.float32)
        self._check(self._lib.octen_n_get_replicas(self._h, Y.ctypes.data))
        return Y

    def replica_factors(self, which: int = 0):
        """([F_1, ..., F_{N-1}, C_rep] each P x Q x R, perm P x R, scales P x (N-1) x R)."""
        Fs = [np.empty((self.P, self.Q, self.R), np.float32) for _ in range(self.N)]
        fp = (ctypes.c_void_p * self.N)(*[f.ctypes.data for f in Fs])
        perm = np.empty((self.P, self.R), np.int32)
        scales = np.empty((self.P, self.N - 1, self.R), np.float64)
        self._check(self._lib.octen_n_get_replica_factors(self._h, int(which), fp,
                                                          perm.ctypes.data, scales.ctypes.data))
        return Fs, perm, scales

    def set_timing(self, on: bool = True):
        self._check(self._lib.octen_n_set_timing(self._h, int(bool(on))))

    def stage_times(self) -> dict:
        """{stage: (milliseconds, timed intervals)} accumulated while timing is on."""
        n = self._lib.octen_n_stage_count()
        ms = np.zeros(n, np.float64)
        cnt = np.zeros(n, np.uint64)
        self._check(self._lib.octen_n_stage_times(self._h, ms.ctypes.data, cnt.ctypes.data))
        return {self._lib.octen_n_stage_name(i).decode(): (float(ms[i]), int(cnt[i]))
                for i in range(n)}

    def close(self):
        if getattr(self, "_h", None):
            self._lib.octen_n_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def append_many(streams, batches, ws):
    """One append on each of several Octen contexts (see octen_append_many)."""
    L = lib()
    keep: list = []
    n = len(streams)
    if len(batches) != n or len(ws) != n:
        raise OctenError(1, "one batch and one W_new per stream expected")
    for i, (g, x, w) in enumerate(zip(streams, batches, ws)):
        t = int(x.shape[0])
        _need(x, t * g.I * g.J, f"X_new[{i}]")
        _need(w, t * g.Qd, f"W_new[{i}]")
    hs = (ctypes.c_void_p * n)(*[s._h.value for s in streams])
    xs = (ctypes.c_void_p * n)(*[_slices(x, s.prec, keep) for x, s in zip(batches, streams)])
    ts = (ctypes.c_int64 * n)(*[int(x.shape[0]) for x in batches])
    wp = (ctypes.c_void_p * n)(*[_f32(w, keep) for w in ws])
    st = L.octen_append_many(hs, n, xs, ts, wp)
    if st != 0:
        msgs = "; ".join(L.octen_last_error(s._h).decode() for s in streams)
        raise OctenError(st, msgs)


def compress(I, J, P, Q, S, X, U_all, V_all, W_all, prec="fp32", R=1, stream=None):
    """Stateless compression of one batch into P summaries (P x Q x Q x Q)."""
    L = lib()
    cfg = _Config(int(I), int(J), int(R), int(P), int(Q), int(S), 1, PREC[prec])
    keep: list = []
    t, Qd = int(X.shape[0]), S + P * (Q - S)
    _need(X, t * I * J, "X")
    _need(U_all, I * Qd, "U_all")
    _need(V_all, J * Qd, "V_all")
    _need(W_all, t * Qd, "W_all")
    Z = np.empty((P, Q, Q, Q), np.float32)
    st = L.octen_compress(ctypes.byref(cfg), _stream_handle(stream), _slices(X, prec, keep),
                          int(X.shape[0]), _f32(U_all, keep), _f32(V_all, keep),
                          _f32(W_all, keep), Z.ctypes.data)
    if st != 0:
        raise OctenError(st, "octen_compress failed")
    return Z
