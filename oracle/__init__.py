"""CPU FP64 oracle for the SU3_Bench link multiply (arXiv 2103.00571).

TEST INFRASTRUCTURE ONLY. The tests, ``__graft_entry__.smoke()``, and the CPU-baseline leg and
reference arm (``--impl reference``) of ``bench.py`` may call it; the product library never does,
and the two share no code.

The arithmetic lives in ``su3_oracle.c`` (plain C, FP64, no FMA contraction); this module builds
it with gcc on first use and wraps it with ctypes and numpy. Every function states the passage of
the paper it follows.
"""
import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "su3_oracle.c")
_OUT = os.path.join(_HERE, "_build", "libsu3oracle.so")
_lock = threading.Lock()
_lib = None


def build(force=False):
    """Compile the oracle (gcc, -O2 -fopenmp -ffp-contract=off) into oracle/_build/."""
    os.makedirs(os.path.dirname(_OUT), exist_ok=True)
    if (not force and os.path.exists(_OUT)
            and os.path.getmtime(_OUT) >= os.path.getmtime(_SRC)):
        return _OUT
    tmp = _OUT + ".%d.tmp" % os.getpid()
    cmd = ["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
           "-shared", "-std=c11", _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _OUT)
    return _OUT


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = ctypes.CDLL(build())
            i64, dp, vp = ctypes.c_int64, ctypes.POINTER(ctypes.c_double), ctypes.c_void_p
            for name, args in [
                ("su3o_mult", [i64, i64, vp, vp, vp]),
                ("su3o_mult_sites", [i64, vp, vp, vp]),
                ("su3o_tworow_expand", [i64, vp, vp]),
                ("su3o_tworow_compress", [i64, vp, vp]),
                ("su3o_unitarity", [i64, vp, vp]),
                ("su3o_round_half", [i64, vp, vp]),
                ("su3o_round_bf16", [i64, vp, vp]),
                ("su3o_round_float", [i64, vp, vp]),
                ("su3o_widen_half", [i64, vp, vp]),
                ("su3o_widen_bf16", [i64, vp, vp]),
                ("su3o_error", [i64, vp, vp, vp]),
                ("su3o_mult_an", [i64, i64, vp, vp, vp]),
                ("su3o_mult_na", [i64, i64, vp, vp, vp]),
                ("su3o_mat_vec", [i64, i64, ctypes.c_int, vp, vp, vp]),
            ]:
                f = getattr(L, name)
                f.argtypes = args
                f.restype = None
            L.su3o_threads.argtypes = []
            L.su3o_threads.restype = ctypes.c_int
            L.su3o_set_threads.argtypes = [ctypes.c_int]
            L.su3o_set_threads.restype = None
            _lib = L
    return _lib


def _ptr(x):
    return ctypes.c_void_p(x.ctypes.data)


def _f64(x):
    return np.ascontiguousarray(x, dtype=np.float64)


def mult(a, b, site_stride=72):
    """c[i][j] = a[i][j] x b[j] for every site i and link j (§Background, the SU3_Bench kernel).

    ``a``: float64 array of n_sites * site_stride doubles (sites of 4 links x 18 doubles, then
    ``site_stride - 72`` untouched doubles); ``b``: 72 doubles (4 matrices). Returns ``c`` shaped
    like ``a``; the doubles past the links of each site stay zero, since the kernel never writes
    them.
    """
    a = _f64(a)
    b = _f64(b)
    assert b.size == 72, "b holds four 3x3 complex matrices"
    assert a.size % site_stride == 0 and site_stride >= 72
    n = a.size // site_stride
    c = np.zeros_like(a)
    lib().su3o_mult(n, site_stride, _ptr(a), _ptr(b), _ptr(c))
    return c


def mult_an(a, b, site_stride=72):
    """c = a^dagger b per link (MILC's mult_su3_an): sum_m conj(a[m][k]) b[j][m][l]."""
    a, b = _f64(a), _f64(b)
    n = a.size // site_stride
    c = np.zeros_like(a)
    lib().su3o_mult_an(n, site_stride, _ptr(a), _ptr(b), _ptr(c))
    return c


def mult_na(a, b, site_stride=72):
    """c = a b^dagger per link (MILC's mult_su3_na): sum_m a[k][m] conj(b[j][l][m])."""
    a, b = _f64(a), _f64(b)
    n = a.size // site_stride
    c = np.zeros_like(a)
    lib().su3o_mult_na(n, site_stride, _ptr(a), _ptr(b), _ptr(c))
    return c


def mat_vec(a, v, adjoint=False, site_stride=72):
    """w[i][j] = a[i][j] v[j] (or a[i][j]^dagger v[j]); v: 24 doubles, w: n_sites*24 doubles."""
    a, v = _f64(a), _f64(v)
    assert v.size == 24, "v holds four colour vectors"
    n = a.size // site_stride
    w = np.zeros(n * 24, dtype=np.float64)
    lib().su3o_mat_vec(n, site_stride, int(bool(adjoint)), _ptr(a), _ptr(v), _ptr(w))
    return w


def mult_sites(a_sel, b):
    """The kernel on a list of sites a_sel[n][72] (sampled checks of large lattices)."""
    a_sel = _f64(a_sel)
    b = _f64(b)
    n = a_sel.size // 72
    c = np.empty_like(a_sel)
    lib().su3o_mult_sites(n, _ptr(a_sel), _ptr(b), _ptr(c))
    return c


def tworow_expand(m12):
    """Rebuild row 2 = conj(row0 x row1) of two-row matrices m12[n][12] -> [n][18]."""
    m12 = _f64(m12)
    n = m12.size // 12
    out = np.empty(n * 18, dtype=np.float64)
    lib().su3o_tworow_expand(n, _ptr(m12), _ptr(out))
    return out.reshape(m12.shape[:-1] + (18,)) if m12.shape[-1] == 12 else out


def tworow_compress(m18):
    """Keep rows 0 and 1 of matrices m18[n][18] -> [n][12]."""
    m18 = _f64(m18)
    n = m18.size // 18
    out = np.empty(n * 12, dtype=np.float64)
    lib().su3o_tworow_compress(n, _ptr(m18), _ptr(out))
    return out.reshape(m18.shape[:-1] + (12,)) if m18.shape[-1] == 18 else out


def unitarity(m18):
    """(max |M M^dagger - I|, max |det M - 1|) over matrices m18[n][18]."""
    m18 = _f64(m18)
    out = np.zeros(2, dtype=np.float64)
    lib().su3o_unitarity(m18.size // 18, _ptr(m18), _ptr(out))
    return float(out[0]), float(out[1])


def round_half(x):
    """FP64 -> binary16 bit patterns, one rounding to nearest even."""
    x = _f64(x)
    out = np.empty(x.shape, dtype=np.uint16)
    lib().su3o_round_half(x.size, _ptr(x), _ptr(out))
    return out


def round_bf16(x):
    """FP64 -> bfloat16 bit patterns, one rounding to nearest even."""
    x = _f64(x)
    out = np.empty(x.shape, dtype=np.uint16)
    lib().su3o_round_bf16(x.size, _ptr(x), _ptr(out))
    return out


def round_float(x):
    """FP64 -> binary32, rounding to nearest even."""
    x = _f64(x)
    out = np.empty(x.shape, dtype=np.float32)
    lib().su3o_round_float(x.size, _ptr(x), _ptr(out))
    return out


def widen_half(h):
    h = np.ascontiguousarray(h, dtype=np.uint16)
    out = np.empty(h.shape, dtype=np.float64)
    lib().su3o_widen_half(h.size, _ptr(h), _ptr(out))
    return out


def widen_bf16(h):
    h = np.ascontiguousarray(h, dtype=np.uint16)
    out = np.empty(h.shape, dtype=np.float64)
    lib().su3o_widen_bf16(h.size, _ptr(h), _ptr(out))
    return out


def threads():
    """OpenMP threads the oracle's parallel loops use."""
    return int(lib().su3o_threads())


def set_threads(n):
    """Sets the OpenMP thread count of the oracle's parallel loops."""
    lib().su3o_set_threads(int(n))


def error(x, ref):
    """(max abs, RMS) of x - ref over all reals; a NaN counts as an infinite error."""
    x = _f64(x).ravel()
    ref = _f64(ref).ravel()
    assert x.size == ref.size
    out = np.zeros(2, dtype=np.float64)
    lib().su3o_error(x.size, _ptr(x), _ptr(ref), _ptr(out))
    return float(out[0]), float(out[1])
