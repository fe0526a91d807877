"""The C-ABI library without a GPU: it loads, exports every function include/su3.h declares, and
its host-side logic (descriptor validation, sizes, status strings, fault injection, null handles)
behaves as documented. No compute call is made."""
import ctypes
import os
import re
import subprocess
import sys

import pytest

import paper_2103_00571_gb300 as su3
from paper_2103_00571_gb300 import _binding as B

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_library_exports_header():
    L = su3.lib()
    names = su3.header_functions()
    assert len(names) >= 18
    missing = [n for n in names if not hasattr(L, n)]
    assert not missing, missing
    hdr = open(os.path.join(ROOT, "include", "su3.h")).read()
    assert L.su3_abi_version() == int(re.search(r"#define SU3_ABI_VERSION (\d+)", hdr).group(1)) == 4


def test_header_is_plain_c_and_links(tmp_path):
    """include/su3.h compiles as strict C99 and a C caller links against libsu3 (no torch types)."""
    src = tmp_path / "caller.c"
    src.write_text(
        '#include "su3.h"\n'
        "int run(const void* a, void* c, void* stream, long long n) {\n"
        "  double b[4][3][3][2] = {{{{0}}}};\n"
        "  su3_handle* h;\n"
        "  if (su3_init(0, &h) != SU3_OK) return 1;\n"
        "  su3_desc d = {SU3_F64, SU3_REPR_FULL18, SU3_LAYOUT_AOS, SU3_ARITH_NATIVE, n, 0};\n"
        "  su3_status s = su3_mult(h, &d, a, &b[0][0][0][0], &d, c, stream);\n"
        "  if (s == SU3_OK) s = su3_sync(h, stream, -1);\n"
        "  su3_finalize(h);\n"
        "  return (int)s;\n"
        "}\n")
    lib = su3.library_path()
    out = tmp_path / "caller.so"
    r = subprocess.run(["gcc", "-std=c99", "-Wall", "-Werror", "-pedantic", "-shared", "-fPIC", "-I",
                        os.path.join(ROOT, "include"), str(src), "-o", str(out), "-L", os.path.dirname(lib),
                        "-lsu3"], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr


def test_status_strings():
    L = su3.lib()
    for s, name in enumerate(["SU3_OK", "SU3_ERR_INVALID_ARG", "SU3_ERR_UNSUPPORTED", "SU3_ERR_CUDA",
                              "SU3_ERR_NOT_INITIALIZED", "SU3_ERR_TIMEOUT", "SU3_ERR_FAULT_INJECTED"]):
        assert L.su3_status_string(s).decode() == name
    assert L.su3_status_string(99).decode() == "SU3_ERR_UNKNOWN"


def test_link_and_site_bytes_match_the_paper():
    """su3_matrix is 144 B in FP64 and 72 B in FP32 (§Background); the packed site is 4 links."""
    assert su3.link_bytes(su3.F64, su3.FULL18) == 144
    assert su3.link_bytes(su3.F32, su3.FULL18) == 72
    assert su3.link_bytes(su3.F16, su3.FULL18) == 36
    assert su3.link_bytes(su3.F64, su3.TWOROW12) == 96
    assert su3.site_update_bytes(su3.F64) == 1152
    assert su3.site_update_bytes(su3.F32) == 576
    assert su3.site_update_bytes(su3.BF16) == 288
    assert su3.site_update_bytes(su3.F64, su3.TWOROW12) == 768
    assert su3.site_update_bytes(su3.F64, su3.TWOROW12, su3.FULL18) == 960
    # 32^4 sites of the paper's padded 320-byte FP32 Site = 320 MiB (§Background)
    d = su3.Desc(su3.F32, su3.FULL18, su3.AOS, 32 ** 4, 320)
    assert su3.array_bytes(d) == 320 * 2 ** 20
    d = su3.Desc(su3.F64, su3.FULL18, su3.AOS, 32 ** 4, 640)
    assert su3.array_bytes(d) == 640 * 2 ** 20


def test_array_bytes_layouts():
    V = 10
    assert su3.array_bytes(su3.Desc(su3.F64, su3.FULL18, su3.SOA, V)) == 40 * 144
    assert su3.array_bytes(su3.Desc(su3.F64, su3.FULL18, su3.AOSOA32, V)) == 64 * 144  # padded to 32 links
    assert su3.array_bytes(su3.Desc(su3.F16, su3.TWOROW12, su3.AOSOA32, 8)) == 32 * 24


@pytest.mark.parametrize("bad", [
    dict(dtype=7), dict(repr=2), dict(layout=3), dict(arith=3), dict(n_sites=-1),
    dict(site_stride_bytes=8), dict(site_stride_bytes=584), dict(layout=su3.SOA, site_stride_bytes=576),
    dict(dtype=su3.F32, arith=su3.F32PAIR), dict(dtype=su3.F16, arith=su3.HYBRID),
])
def test_descriptor_validation(bad):
    kw = dict(dtype=su3.F64, repr=su3.FULL18, layout=su3.AOS, n_sites=16, site_stride_bytes=0, arith=su3.NATIVE)
    kw.update(bad)
    assert su3.check_desc(su3.Desc(**kw)) == B.ERR_INVALID_ARG
    assert su3.lib().su3_array_bytes(ctypes.byref(su3.Desc(**kw))) == -1


def test_valid_descriptors():
    for dt in (su3.F64, su3.F32, su3.F16, su3.BF16):
        for rep in (su3.FULL18, su3.TWOROW12):
            for lay in (su3.AOS, su3.AOSOA32, su3.SOA):
                assert su3.check_desc(su3.Desc(dt, rep, lay, 1000)) == B.OK
    assert su3.check_desc(su3.Desc(su3.F64, su3.FULL18, su3.AOS, 5, 640)) == B.OK


def test_null_handle():
    L = su3.lib()
    d = su3.Desc(su3.F64, su3.FULL18, su3.AOS, 1)
    assert L.su3_mult(None, ctypes.byref(d), None, None, None, None, None) == B.ERR_NOT_INITIALIZED
    assert L.su3_sync(None, None, 0) == B.ERR_NOT_INITIALIZED
    assert L.su3_finalize(None) == B.OK
    assert L.su3_last_error(None).decode() == "null handle"
    assert L.su3_init(0, None) == B.ERR_INVALID_ARG


def test_fault_injection_on_init_touches_no_gpu():
    code = ("import sys, ctypes; sys.path.insert(0, %r); import paper_2103_00571_gb300 as s;"
            "h = ctypes.c_void_p(); print(s.lib().su3_init(0, ctypes.byref(h)))" % ROOT)
    env = dict(os.environ, SU3_FAULT_INJECT="alloc")
    out = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, check=True)
    assert out.stdout.strip() == str(B.ERR_FAULT_INJECTED)


def test_init_without_gpu_fails_cleanly():
    """On a machine without a GPU, su3_init reports a CUDA error instead of crashing."""
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    h = ctypes.c_void_p()
    assert su3.lib().su3_init(0, ctypes.byref(h)) == B.ERR_CUDA
    assert not h.value
