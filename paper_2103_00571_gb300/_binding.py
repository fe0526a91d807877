"""ctypes binding of libsu3 (include/su3.h): argument marshalling only.

Every step of the operation runs in libsu3's CUDA kernels. PyTorch is used by callers for device
memory and streams; this module only turns tensors into pointers and stream handles. If the
library cannot be built or loaded, every entry point raises: there is no fallback path.
"""
import ctypes
import os
import re
import threading

import numpy as np

from . import build as _build

F64, F32, F16, BF16 = 0, 1, 2, 3
FULL18, TWOROW12 = 0, 1
AOS, AOSOA32, SOA = 0, 1, 2
NATIVE, F32PAIR, HYBRID = 0, 1, 2
OP_NN, OP_NA, OP_AN = 0, 1, 2
HOST_AUTO, HOST_DIRECT, HOST_STAGED = 0, 1, 2

OK, ERR_INVALID_ARG, ERR_UNSUPPORTED, ERR_CUDA, ERR_NOT_INITIALIZED, ERR_TIMEOUT, ERR_FAULT_INJECTED = range(7)

DTYPE_NAMES = {"f64": F64, "f32": F32, "f16": F16, "bf16": BF16}
REAL_BYTES = {F64: 8, F32: 4, F16: 2, BF16: 2}


class Su3Error(RuntimeError):
    def __init__(self, status, message):
        self.status = status
        super().__init__("%s: %s" % (_status_name(status), message))


class Desc(ctypes.Structure):
    _fields_ = [("dtype", ctypes.c_int32), ("repr", ctypes.c_int32), ("layout", ctypes.c_int32),
                ("arith", ctypes.c_int32), ("n_sites", ctypes.c_int64),
                ("site_stride_bytes", ctypes.c_int64)]

    def __init__(self, dtype=F64, repr=FULL18, layout=AOS, n_sites=0, site_stride_bytes=0, arith=NATIVE):
        super().__init__(dtype, repr, layout, arith, n_sites, site_stride_bytes)

    def key(self):
        return (self.dtype, self.repr, self.layout, self.arith, self.n_sites, self.site_stride_bytes)

    def __repr__(self):
        return "Desc(dtype=%d, repr=%d, layout=%d, arith=%d, n_sites=%d, stride=%d)" % self.key()


class LaunchCfg(ctypes.Structure):
    _fields_ = [("block", ctypes.c_int32), ("tile_sites", ctypes.c_int32), ("stages", ctypes.c_int32),
                ("ctas_per_sm", ctypes.c_int32), ("native_permille", ctypes.c_int32),
                ("threads_per_link", ctypes.c_int32)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class BatchItem(ctypes.Structure):
    _fields_ = [("desc", Desc), ("a_dev", ctypes.c_void_p), ("c_dev", ctypes.c_void_p),
                ("b", ctypes.c_double * 72)]


_lock = threading.Lock()
_lib = None

_SIGS = {
    "su3_init": (ctypes.c_int, [ctypes.c_int, ctypes.c_void_p]),
    "su3_finalize": (ctypes.c_int, [ctypes.c_void_p]),
    "su3_mult": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(Desc), ctypes.c_void_p, ctypes.c_void_p,
                                ctypes.POINTER(Desc), ctypes.c_void_p, ctypes.c_void_p]),
    "su3_mult_host": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(Desc), ctypes.c_void_p, ctypes.c_void_p,
                                     ctypes.POINTER(Desc), ctypes.c_void_p, ctypes.c_void_p]),
    "su3_mult_batched": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.POINTER(BatchItem),
                                        ctypes.c_void_p, ctypes.c_int32]),
    "su3_pack": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.POINTER(Desc), ctypes.c_void_p,
                                ctypes.c_void_p]),
    "su3_unpack": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(Desc), ctypes.c_void_p, ctypes.c_void_p,
                                  ctypes.c_void_p]),
    "su3_sync": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32]),
    "su3_status_string": (ctypes.c_char_p, [ctypes.c_int]),
    "su3_last_error": (ctypes.c_char_p, [ctypes.c_void_p]),
    "su3_link_bytes": (ctypes.c_int64, [ctypes.c_int32, ctypes.c_int32]),
    "su3_array_bytes": (ctypes.c_int64, [ctypes.POINTER(Desc)]),
    "su3_check_desc": (ctypes.c_int, [ctypes.POINTER(Desc)]),
    "su3_set_launch_cfg": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(Desc), ctypes.POINTER(LaunchCfg)]),
    "su3_get_launch_cfg": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(Desc), ctypes.POINTER(LaunchCfg)]),
    "su3_launch_count": (ctypes.c_int64, [ctypes.c_void_p]),
    "su3_mult_batched_static": (ctypes.c_int, [ctypes.c_int32, ctypes.POINTER(BatchItem), ctypes.c_void_p]),
    "su3_set_batched_cfg": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(LaunchCfg)]),
    "su3_get_batched_cfg": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(LaunchCfg)]),
    "su3_abi_version": (ctypes.c_int32, []),
    "su3_selftest_wait_timeout": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p]),
    "su3_mult_op": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.POINTER(Desc), ctypes.c_void_p,
                                   ctypes.c_void_p, ctypes.POINTER(Desc), ctypes.c_void_p, ctypes.c_void_p]),
    "su3_mat_vec": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.POINTER(Desc), ctypes.c_void_p,
                                   ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "su3_set_launch_cfg_for": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(Desc), ctypes.POINTER(Desc),
                                              ctypes.POINTER(LaunchCfg)]),
    "su3_get_launch_cfg_for": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(Desc), ctypes.POINTER(Desc),
                                              ctypes.POINTER(LaunchCfg)]),
    "su3_measure_fp64_rate": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.POINTER(ctypes.c_double)]),
    "su3_set_host_path": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32]),
    "su3_last_host_path": (ctypes.c_int32, [ctypes.c_void_p]),
    "su3_host_pageable_access": (ctypes.c_int32, [ctypes.c_void_p]),
}


def library_path():
    return _build.LIB


def lib():
    """Loads libsu3 (building it first if it is missing or older than its sources)."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.build()
            L = ctypes.CDLL(path)
            for name, (res, args) in _SIGS.items():
                f = getattr(L, name)
                f.restype = res
                f.argtypes = args
            _lib = L
    return _lib


def header_functions():
    """Names of the functions include/su3.h declares."""
    hdr = open(os.path.join(_build.INCLUDE, "su3.h")).read()
    return sorted(set(re.findall(r"^\s*(?:const\s+)?[a-z0-9_]+\s*\*?\s*(su3_[a-z0-9_]+)\s*\(", hdr, re.M)))


def _status_name(s):
    try:
        return lib().su3_status_string(s).decode()
    except Exception:  # noqa: BLE001 - only used for messages
        return "status %d" % s


def _stream_ptr(stream):
    if stream is None:
        import torch
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


def _ptr(x):
    if x is None:
        return ctypes.c_void_p(0)
    if isinstance(x, int):
        return ctypes.c_void_p(x)
    if isinstance(x, np.ndarray):
        return ctypes.c_void_p(x.ctypes.data)
    return ctypes.c_void_p(x.data_ptr())


def _b72(b):
    b = np.ascontiguousarray(b, dtype=np.float64).reshape(-1)
    if b.size != 72:
        raise ValueError("b must hold 4 x 3 x 3 complex = 72 doubles")
    return b


def link_bytes(dtype, repr_):
    return int(lib().su3_link_bytes(dtype, repr_))


def array_bytes(desc):
    n = int(lib().su3_array_bytes(ctypes.byref(desc)))
    if n < 0:
        raise Su3Error(ERR_INVALID_ARG, "invalid descriptor %r" % (desc,))
    return n


def check_desc(desc):
    return int(lib().su3_check_desc(ctypes.byref(desc)))


class Handle:
    """One libsu3 handle bound to a CUDA device (not thread-safe: one per host thread)."""

    def __init__(self, device=0):
        self._h = ctypes.c_void_p()
        s = lib().su3_init(device, ctypes.byref(self._h))
        if s != OK:
            raise Su3Error(s, "su3_init(%d) failed" % device)

    def close(self):
        if self._h:
            lib().su3_finalize(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:  # noqa: BLE001 - interpreter shutdown
            pass

    def _check(self, s, what):
        if s != OK:
            raise Su3Error(s, "%s: %s" % (what, lib().su3_last_error(self._h).decode()))

    def mult(self, a_desc, a, b, c_desc, c, stream=None):
        b = _b72(b)
        self._check(lib().su3_mult(self._h, ctypes.byref(a_desc), _ptr(a), _ptr(b),
                                   ctypes.byref(c_desc) if c_desc is not None else None, _ptr(c),
                                   _stream_ptr(stream)), "su3_mult")

    def mult_op(self, op, a_desc, a, b, c_desc, c, stream=None):
        b = _b72(b)
        self._check(lib().su3_mult_op(self._h, op, ctypes.byref(a_desc), _ptr(a), _ptr(b),
                                      ctypes.byref(c_desc) if c_desc is not None else None, _ptr(c),
                                      _stream_ptr(stream)), "su3_mult_op")

    def mat_vec(self, a_desc, a, v, w, adjoint=False, stream=None):
        v = np.ascontiguousarray(v, dtype=np.float64).reshape(-1)
        if v.size != 24:
            raise ValueError("v holds 4 colour vectors x 3 complex = 24 doubles")
        self._check(lib().su3_mat_vec(self._h, int(bool(adjoint)), ctypes.byref(a_desc), _ptr(a), _ptr(v), _ptr(w),
                                      _stream_ptr(stream)), "su3_mat_vec")

    def mult_host(self, a_desc, a_host, b, c_desc, c_host, stream=0):
        b = _b72(b)
        self._check(lib().su3_mult_host(self._h, ctypes.byref(a_desc), _ptr(a_host), _ptr(b),
                                        ctypes.byref(c_desc) if c_desc is not None else None, _ptr(c_host),
                                        _stream_ptr(stream)), "su3_mult_host")

    def mult_batched(self, items, stream=None, use_graph=True):
        arr = (BatchItem * len(items))(*items)
        self._check(lib().su3_mult_batched(self._h, len(items), arr, _stream_ptr(stream), int(bool(use_graph))),
                    "su3_mult_batched")

    def pack(self, src_f64, dst_desc, dst, stream=None):
        self._check(lib().su3_pack(self._h, _ptr(src_f64), ctypes.byref(dst_desc), _ptr(dst), _stream_ptr(stream)),
                    "su3_pack")

    def unpack(self, src_desc, src, dst_f64, stream=None):
        self._check(lib().su3_unpack(self._h, ctypes.byref(src_desc), _ptr(src), _ptr(dst_f64),
                                     _stream_ptr(stream)), "su3_unpack")

    def sync(self, stream=None, timeout_ms=-1):
        self._check(lib().su3_sync(self._h, _stream_ptr(stream), timeout_ms), "su3_sync")

    def set_launch_cfg(self, form, **cfg):
        c = LaunchCfg(cfg.get("block", 0), cfg.get("tile_sites", 0), cfg.get("stages", 0), cfg.get("ctas_per_sm", 0),
                      cfg.get("native_permille", 0), cfg.get("threads_per_link", 0))
        self._check(lib().su3_set_launch_cfg(self._h, ctypes.byref(form), ctypes.byref(c)), "su3_set_launch_cfg")

    def get_launch_cfg(self, form):
        c = LaunchCfg()
        self._check(lib().su3_get_launch_cfg(self._h, ctypes.byref(form), ctypes.byref(c)), "su3_get_launch_cfg")
        return c.as_dict()

    def set_launch_cfg_for(self, a_form, c_form, **cfg):
        """Launch configuration of one (a, c) repr pair, e.g. two-row in, full out."""
        c = LaunchCfg(cfg.get("block", 0), cfg.get("tile_sites", 0), cfg.get("stages", 0), cfg.get("ctas_per_sm", 0),
                      cfg.get("native_permille", 0), cfg.get("threads_per_link", 0))
        self._check(lib().su3_set_launch_cfg_for(self._h, ctypes.byref(a_form), ctypes.byref(c_form), ctypes.byref(c)),
                    "su3_set_launch_cfg_for")

    def get_launch_cfg_for(self, a_form, c_form):
        c = LaunchCfg()
        self._check(lib().su3_get_launch_cfg_for(self._h, ctypes.byref(a_form), ctypes.byref(c_form), ctypes.byref(c)),
                    "su3_get_launch_cfg_for")
        return c.as_dict()

    def set_batched_cfg(self, **cfg):
        c = LaunchCfg(cfg.get("block", 0), cfg.get("tile_sites", 0), cfg.get("stages", 0), cfg.get("ctas_per_sm", 0),
                      0, cfg.get("threads_per_link", 0))
        self._check(lib().su3_set_batched_cfg(self._h, ctypes.byref(c)), "su3_set_batched_cfg")

    def get_batched_cfg(self):
        c = LaunchCfg()
        self._check(lib().su3_get_batched_cfg(self._h, ctypes.byref(c)), "su3_get_batched_cfg")
        return c.as_dict()

    def measure_fp64_rate(self, steps=8192):
        """Sustained FP64 FMA rate of the device in TFLOP/s (a diagnostic kernel)."""
        out = ctypes.c_double()
        self._check(lib().su3_measure_fp64_rate(self._h, int(steps), ctypes.byref(out)), "su3_measure_fp64_rate")
        return out.value

    def set_host_path(self, path):
        """HOST_AUTO, HOST_DIRECT (the kernel streams pinned host buffers, or pageable ones on a
        device with coherent pageable access) or HOST_STAGED (chunked copies through HBM)."""
        self._check(lib().su3_set_host_path(self._h, int(path)), "su3_set_host_path")

    def last_host_path(self):
        return int(lib().su3_last_host_path(self._h))

    def pageable_host_access(self):
        """Whether the device reads pageable host memory coherently (the direct path then also
        takes pageable buffers)."""
        return bool(lib().su3_host_pageable_access(self._h))

    def selftest_wait_timeout(self, limit_ms=50, stream=None):
        self._check(lib().su3_selftest_wait_timeout(self._h, limit_ms, _stream_ptr(stream)),
                    "su3_selftest_wait_timeout")

    def launch_count(self):
        return int(lib().su3_launch_count(self._h))

    @property
    def raw(self):
        return self._h
