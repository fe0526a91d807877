"""su3_mult_host, the entry point for a and c in host memory, on both of its paths.

DIRECT: a and c in pinned, mapped host memory (and, on a device that reads pageable host memory
coherently, ordinary pageable memory) are streamed by the kernel itself over the host link. STAGED: chunks are copied through HBM. Both must give, bit for bit, what su3_mult gives on
device copies of the same data (the same per-link operations), for every arithmetic, repr pair and
site stride, in place too; the path taken is reported, and pad bytes of padded sites in c are
never written."""
import numpy as np
import pytest

import oracle
import paper_2103_00571_gb300 as su3
import su3_inputs as gen
from gpu_helpers import empty_bytes, to_dev

pytestmark = pytest.mark.gpu

FORMS = [  # dtype, repr in, repr out, arith, site stride (0 = packed)
    (su3.F64, su3.FULL18, su3.FULL18, su3.NATIVE, 0),
    (su3.F64, su3.FULL18, su3.FULL18, su3.F32PAIR, 0),
    (su3.F64, su3.FULL18, su3.FULL18, su3.NATIVE, 640),
    (su3.F64, su3.TWOROW12, su3.FULL18, su3.F32PAIR, 0),
    (su3.F32, su3.FULL18, su3.FULL18, su3.NATIVE, 0),
    (su3.F16, su3.TWOROW12, su3.TWOROW12, su3.NATIVE, 0),
    (su3.BF16, su3.FULL18, su3.FULL18, su3.NATIVE, 0),
]


@pytest.fixture(scope="module")
def h():
    hh = su3.Handle(0)
    yield hh
    hh.close()


def _device_result(h, da, dc, abuf_host, b):
    """su3_mult on device copies of the same bytes; returns the bytes of c."""
    import torch
    a_dev = to_dev(np.frombuffer(abuf_host, dtype=np.uint8))
    c_dev = empty_bytes(su3.array_bytes(dc), fill=0xA5)
    h.mult(da, a_dev, b, dc, c_dev)
    h.sync()
    return c_dev.cpu().numpy()


def _packed_host(h, a64, d):
    """a64 (FP64 AOS sites) converted to the form d describes, as host bytes."""
    import torch
    V = d.n_sites
    src = to_dev(a64)
    if d.site_stride_bytes:  # a padded FP64 site: links at offset 0, pad bytes a marker
        buf = empty_bytes(su3.array_bytes(d), fill=0x3C)
    else:
        buf = empty_bytes(su3.array_bytes(d))
    h.pack(src, d, buf)
    h.sync()
    return buf.cpu().numpy()


@pytest.mark.parametrize("form", FORMS, ids=lambda f: "dt%d-r%d%d-ar%d-s%d" % f)
@pytest.mark.parametrize("path", [su3.HOST_AUTO, su3.HOST_STAGED])
def test_host_paths_match_device(h, form, path):
    import torch
    dt, ri, ro, ar, stride = form
    V = 20000 + 7
    a64, b = gen.lattice(31, V)
    da = su3.Desc(dt, ri, su3.AOS, V, stride, ar)
    dc = su3.Desc(dt, ro, su3.AOS, V, stride, ar)
    a_bytes = _packed_host(h, a64, da)
    want = _device_result(h, da, dc, a_bytes, b)
    a_pin = torch.from_numpy(a_bytes.copy()).pin_memory()
    c_pin = torch.full((su3.array_bytes(dc),), 0xA5, dtype=torch.uint8).pin_memory()
    h.set_host_path(path)
    try:
        h.mult_host(da, a_pin.data_ptr(), b, dc, c_pin.data_ptr())
        assert h.last_host_path() == (su3.HOST_DIRECT if path == su3.HOST_AUTO else su3.HOST_STAGED)
    finally:
        h.set_host_path(su3.HOST_AUTO)
    assert np.array_equal(c_pin.numpy(), want)  # same bits, pad bytes (0xA5) untouched too
    if stride:
        assert np.all(c_pin.numpy().reshape(V, stride)[:, 576:] == 0xA5)


def test_direct_in_place_and_pageable(h):
    """In place on pinned memory takes the direct path. Pageable numpy arrays take the direct path
    on a device with coherent pageable access and the staged path elsewhere (the same bits either
    way); forcing the direct path on pageable memory is refused before anything runs where the
    device cannot read it."""
    import torch
    V = 9001
    a64, b = gen.lattice(32, V)
    d = su3.Desc(su3.F64, su3.FULL18, su3.AOS, V)
    ref = oracle.mult(a64, b)
    pin = torch.from_numpy(a64.copy()).pin_memory()
    h.mult_host(d, pin.data_ptr(), b, d, pin.data_ptr())
    assert h.last_host_path() == su3.HOST_DIRECT
    assert oracle.error(pin.numpy(), ref)[0] <= 1e-13
    page = a64.copy()
    out = np.full_like(page, np.nan)
    h.mult_host(d, page, b, d, out)
    assert h.last_host_path() == (su3.HOST_DIRECT if h.pageable_host_access() else su3.HOST_STAGED)
    assert np.array_equal(out, pin.numpy())
    for path in (su3.HOST_STAGED, su3.HOST_DIRECT):
        out2 = np.full_like(page, np.nan)
        h.set_host_path(path)
        try:
            if path == su3.HOST_DIRECT and not h.pageable_host_access():
                with pytest.raises(su3.Su3Error):
                    h.mult_host(d, page, b, d, out2)
                continue
            h.mult_host(d, page, b, d, out2)
            assert h.last_host_path() == path
            assert np.array_equal(out2, pin.numpy())
        finally:
            h.set_host_path(su3.HOST_AUTO)
    with pytest.raises(su3.Su3Error):
        h.set_host_path(7)


@pytest.mark.parametrize("form", FORMS, ids=lambda f: "dt%d-r%d%d-ar%d-s%d" % f)
def test_pageable_direct_matches_device(h, form):
    """Ordinary (pageable) numpy buffers on a device that reads them coherently: AUTO takes the
    direct path, the kernel streams them as it streams pinned ones, so c has su3_mult's bits and
    pad bytes stay untouched; in place too."""
    if not h.pageable_host_access():
        pytest.skip("this device does not read pageable host memory coherently")
    dt, ri, ro, ar, stride = form
    V = 20000 + 7
    a64, b = gen.lattice(33, V)
    da = su3.Desc(dt, ri, su3.AOS, V, stride, ar)
    dc = su3.Desc(dt, ro, su3.AOS, V, stride, ar)
    a_bytes = _packed_host(h, a64, da)
    want = _device_result(h, da, dc, a_bytes, b)
    a_page = a_bytes.copy()
    c_page = np.full(su3.array_bytes(dc), 0xA5, dtype=np.uint8)
    h.mult_host(da, a_page, b, dc, c_page)
    assert h.last_host_path() == su3.HOST_DIRECT
    assert np.array_equal(c_page, want)
    assert np.array_equal(a_page, a_bytes)  # a is only read
    if ri == ro:
        h.mult_host(da, a_page, b, dc, a_page)  # in place: links replaced, a's pad bytes kept
        assert h.last_host_path() == su3.HOST_DIRECT
        exp = want.copy()
        if stride:
            exp.reshape(V, stride)[:, 576:] = a_bytes.reshape(V, stride)[:, 576:]
        assert np.array_equal(a_page, exp)


def test_misaligned_host_buffers_take_the_staged_path(h):
    """The kernel streams 16-byte words, so buffers that are not 16-byte aligned (pinned or
    pageable) are copied through HBM under AUTO, with the same bits; a forced direct path is
    refused before anything runs."""
    import torch
    V = 3001
    n = V * 72
    a64, b = gen.lattice(34, V)
    d = su3.Desc(su3.F64, su3.FULL18, su3.AOS, V)
    a_al = torch.from_numpy(a64.copy()).pin_memory()
    c_al = torch.empty(n, dtype=torch.float64).pin_memory()
    h.mult_host(d, a_al.data_ptr(), b, d, c_al.data_ptr())
    assert h.last_host_path() == su3.HOST_DIRECT
    want = c_al.numpy().copy()
    pa = torch.zeros(n + 2, dtype=torch.float64).pin_memory()
    pc = torch.zeros(n + 2, dtype=torch.float64).pin_memory()
    pa.numpy()[1:1 + n] = a64
    h.mult_host(d, pa.data_ptr() + 8, b, d, pc.data_ptr() + 8)  # both 8 bytes off a 16-byte boundary
    assert h.last_host_path() == su3.HOST_STAGED
    assert np.array_equal(pc.numpy()[1:1 + n], want)
    page_a = np.zeros(n + 2)
    page_a[1:1 + n] = a64
    page_c = np.zeros(n + 2)
    a_view, c_view = page_a[1:1 + n], page_c[1:1 + n]
    assert a_view.ctypes.data % 16 == 8
    h.mult_host(d, a_view, b, d, c_view)
    assert h.last_host_path() == su3.HOST_STAGED
    assert np.array_equal(c_view, want)
    h.set_host_path(su3.HOST_DIRECT)
    try:
        for args in ((pa.data_ptr() + 8, pc.data_ptr() + 8), (a_view, c_view), (a_al.data_ptr(), pc.data_ptr() + 8)):
            with pytest.raises(su3.Su3Error):
                h.mult_host(d, args[0], b, d, args[1])
    finally:
        h.set_host_path(su3.HOST_AUTO)


def test_direct_large_lattice_vs_oracle(h):
    """A lattice far larger than L2 (L=40, 1.47 GB each way) through the direct path, checked
    against the oracle on a sample of sites spread over the whole lattice."""
    import torch
    V = 40 ** 4
    a_pin = torch.empty(V * 72, dtype=torch.float64).pin_memory()
    gen.sites(2103, 0, V, out=a_pin.numpy())
    b = gen.bmat(2103, 0, V)
    c_pin = torch.empty(V * 72, dtype=torch.float64).pin_memory()
    for arith, tol in ((su3.NATIVE, 1e-13), (su3.F32PAIR, 1e-13)):
        d = su3.Desc(su3.F64, su3.FULL18, su3.AOS, V, 0, arith)
        h.mult_host(d, a_pin.data_ptr(), b, d, c_pin.data_ptr())
        assert h.last_host_path() == su3.HOST_DIRECT
        idx = np.unique(np.linspace(0, V - 1, 5000).astype(np.int64))
        got = c_pin.numpy().reshape(V, 72)[idx]
        want = oracle.mult_sites(a_pin.numpy().reshape(V, 72)[idx], b)
        assert oracle.error(got, want)[0] <= tol, arith
