"""Seeded synthetic SU(3) inputs for the SU3_Bench link multiply.

A module of its own: it builds input matrices (random SU(3) by Gram-Schmidt, plus the paper's
constant initialisation) and holds none of the multiply's arithmetic. The CPU oracle and the CUDA
path both consume its bytes. The C source (``su3gen.c``) documents the recipe; this file compiles
it with gcc on first use and wraps it with ctypes.
"""
import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "su3gen.c")
_OUT = os.path.join(_HERE, "_build", "libsu3gen.so")
_lock = threading.Lock()
_lib = None

#: seed of the single-lattice workloads; lattice k of a batch uses lattice id k
DEFAULT_SEED = 2103


def build(force=False):
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
            u64, u32, i64, i32, vp = (ctypes.c_uint64, ctypes.c_uint32, ctypes.c_int64,
                                      ctypes.c_int32, ctypes.c_void_p)
            L.su3gen_philox4x32_10.argtypes = [vp, vp, vp]
            L.su3gen_normals.argtypes = [u64, u32, u64, vp]
            L.su3gen_matrices.argtypes = [u64, u32, u64, i64, vp]
            L.su3gen_sites.argtypes = [u64, u32, i64, i64, i64, vp]
            L.su3gen_sites_at.argtypes = [u64, u32, vp, i64, vp]
            L.su3gen_extents.argtypes = [u64, i32, vp]
            for f in (L.su3gen_philox4x32_10, L.su3gen_normals, L.su3gen_matrices,
                      L.su3gen_sites, L.su3gen_sites_at, L.su3gen_extents):
                f.restype = None
            _lib = L
    return _lib


def _p(x):
    return ctypes.c_void_p(x.ctypes.data)


def philox4x32_10(ctr, key):
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    lib().su3gen_philox4x32_10(_p(c), _p(k), _p(out))
    return out


def normals(seed, lattice, mat_id):
    out = np.zeros(12, dtype=np.float64)
    lib().su3gen_normals(seed, lattice, mat_id, _p(out))
    return out


def matrices(seed, lattice, first_id, count):
    """Random SU(3) matrices with ids first_id..first_id+count-1, shape [count, 18]."""
    out = np.empty((count, 18), dtype=np.float64)
    if count:
        lib().su3gen_matrices(seed, lattice, first_id, count, _p(out))
    return out


def sites(seed, lattice, n_sites, first_site=0, count=None, stride=72, out=None):
    """Sites first_site..first_site+count-1 of a lattice (FP64 AoS, ``stride`` doubles each).

    With ``out`` given (a float64 array of count*stride doubles, possibly pinned memory), it is
    filled in place; the doubles past the 72 link doubles of each site are left untouched.
    """
    count = n_sites - first_site if count is None else count
    if out is None:
        out = np.zeros(count * stride, dtype=np.float64)
    assert out.dtype == np.float64 and out.size >= count * stride and out.flags.c_contiguous
    if count:
        lib().su3gen_sites(seed, lattice, first_site, count, stride, _p(out))
    return out


def sites_at(seed, lattice, idx):
    """The 4 links of the sites at indices ``idx``: array [len(idx), 72]."""
    idx = np.ascontiguousarray(idx, dtype=np.int64)
    out = np.empty((idx.size, 72), dtype=np.float64)
    if idx.size:
        lib().su3gen_sites_at(seed, lattice, _p(idx), idx.size, _p(out))
    return out


def bmat(seed, lattice, n_sites):
    """The four fixed matrices b[0..3] of a lattice of ``n_sites`` sites: 72 doubles."""
    return matrices(seed, lattice, 4 * n_sites, 4).reshape(72)


def lattice(seed, n_sites, lattice_id=0, stride=72):
    """(a, b) of one lattice: a has n_sites*stride doubles, b has 72."""
    return sites(seed, lattice_id, n_sites, stride=stride), bmat(seed, lattice_id, n_sites)


def extents(seed, n):
    """Extents (Lx, Ly, Lz, Lt) of n lattices, uniform over {4, 6, ..., 24}: int32 [n, 4]."""
    out = np.zeros((n, 4), dtype=np.int32)
    lib().su3gen_extents(seed, n, _p(out))
    return out


def paper_constant(n_sites, stride=72):
    """The paper's initialisation (§Performance on Xeon, the data-allocation table): every element
    of every link of a equal to 1+0i and every element of b equal to 1/3+0i. Not SU(3); with it
    every element of c equals 1+0i."""
    a = np.zeros((n_sites, stride), dtype=np.float64)
    a[:, 0:72:2] = 1.0
    b = np.zeros(72, dtype=np.float64)
    b[0::2] = 1.0 / 3.0
    return a.reshape(-1), b
