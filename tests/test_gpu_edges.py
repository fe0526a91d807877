"""Edge cases and invariants of the CUDA path, all through the C ABI."""
import numpy as np
import pytest

import oracle
import paper_2103_00571_gb300 as su3
import su3_inputs as gen
from gpu_helpers import empty_bytes, run_form, to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def h():
    return su3.Handle(0)


def test_identity_b_bitwise(h):
    V = 4099
    a, _ = gen.lattice(1, V)
    eye = np.zeros((4, 9, 2))
    eye[:, [0, 4, 8], 0] = 1.0
    got = run_form(h, a, eye.reshape(72), su3.F64)
    assert np.array_equal(got.view(np.uint64), a.view(np.uint64))


def test_paper_constant_case(h):
    """a = 1+0i, b = 1/3+0i everywhere (the paper's initialisation) => c = 1+0i."""
    a, b = gen.paper_constant(4096)
    for dt, tl in ((su3.F64, 1e-15), (su3.F32, 1e-6), (su3.F16, 1e-3), (su3.BF16, 1e-2)):
        got = run_form(h, a, b, dt).reshape(-1, 72)
        assert np.max(np.abs(got[:, 0::2] - 1.0)) <= tl and np.max(np.abs(got[:, 1::2])) <= tl


def test_iterations_are_idempotent(h):
    """Each iteration recomputes c from the unchanged a: 10 iterations == 1, bit for bit."""
    V = 5000
    a, b = gen.lattice(2, V)
    assert np.array_equal(run_form(h, a, b, su3.F64, iters=1), run_form(h, a, b, su3.F64, iters=10))


def test_in_place(h):
    import torch
    V = 3001
    a, b = gen.lattice(3, V)
    for dt in (su3.F64, su3.F32):
        d = su3.Desc(dt, su3.FULL18, su3.AOS, V)
        buf = empty_bytes(su3.array_bytes(d))
        h.pack(to_dev(a), d, buf)
        h.mult(d, buf, b, d, buf)
        out = torch.empty(V * 72, dtype=torch.float64, device="cuda")
        h.unpack(d, buf, out)
        h.sync()
        ref = oracle.mult(a, b)
        assert oracle.error(out.cpu().numpy(), ref)[0] <= (1e-13 if dt == su3.F64 else 2e-6)


@pytest.mark.parametrize("arith", [su3.NATIVE, su3.F32PAIR])
@pytest.mark.parametrize("cfg", [None, dict(block=256, tile_sites=64, stages=3, ctas_per_sm=2)])
def test_stride_640_keeps_pads_and_canaries(h, arith, cfg):
    """The paper's padded 640-byte FP64 site: the kernel never writes bytes 576..639 of a site,
    nor anything outside c (4 KiB canaries on both sides). The second shape is the packed-stride
    tuned one, which at 640 B needs a smaller tile to keep two CTAs per SM."""
    import torch
    V = 20051
    a, b = gen.lattice(4, V)
    stride = 640
    a640 = np.full((V, 80), -3.25)
    a640[:, :72] = a.reshape(V, 72)
    canary = 4096
    d = su3.Desc(su3.F64, su3.FULL18, su3.AOS, V, stride, arith)
    saved = h.get_launch_cfg(d)
    if cfg:
        h.set_launch_cfg(d, **cfg)
    try:
        cbig = torch.full((canary * 2 + V * stride,), 0xA5, dtype=torch.uint8, device="cuda")
        cview_ptr = cbig.data_ptr() + canary
        # pads of c pre-filled with a pattern
        cbig[canary:canary + V * stride].view(torch.float64).view(V, 80)[:, 72:] = 9.5
        a_dev = to_dev(a640.reshape(-1))
        h.mult(d, a_dev, b, d, cview_ptr)
        h.sync()
    finally:
        h.set_launch_cfg(d, **saved)
    host = cbig.cpu().numpy()
    assert np.all(host[:canary] == 0xA5) and np.all(host[-canary:] == 0xA5)
    c = host[canary:canary + V * stride].view(np.float64).reshape(V, 80)
    assert np.all(c[:, 72:] == 9.5)
    assert oracle.error(c[:, :72].reshape(-1), oracle.mult(a, b))[0] <= 1e-13


@pytest.mark.parametrize("dtype,stride", [(su3.F64, 592), (su3.F64, 1024), (su3.F32, 304), (su3.F16, 160),
                                          (su3.BF16, 208)])
def test_generic_site_strides(h, dtype, stride):
    """Any 16-byte-multiple site stride at least the link bytes: links land at each site's start,
    the bytes after them are left alone, for one and three threads per link, and for a tile wider
    than the 256 sites one tensor copy moves (the launcher narrows it)."""
    import torch
    V = 3001
    a, b = gen.lattice(14, V)
    d = su3.Desc(dtype, su3.FULL18, su3.AOS, V, stride)
    dp = su3.Desc(dtype, su3.FULL18, su3.AOS, V)
    packed = empty_bytes(su3.array_bytes(dp))
    h.pack(to_dev(a), dp, packed)
    lb = su3.array_bytes(dp) // V
    src = torch.full((V * stride,), 0x3C, dtype=torch.uint8, device="cuda")
    src.view(V, stride)[:, :lb] = packed.view(V, lb)
    ref = oracle.mult(a, b)
    tol = {su3.F64: 1e-13, su3.F32: 2e-6, su3.F16: 5e-3, su3.BF16: 3e-2}[dtype]
    saved = h.get_launch_cfg(d)
    try:
        for tiles, tpl in ((48, 1), (48, 3), (300, 1)):
            h.set_launch_cfg(d, block=128, tile_sites=tiles, stages=3, ctas_per_sm=1, threads_per_link=tpl)
            dst = torch.full((V * stride,), 0xC3, dtype=torch.uint8, device="cuda")
            h.mult(d, src, b, d, dst)
            h.sync()
            host = dst.view(V, stride).cpu()
            assert bool(torch.all(host[:, lb:] == 0xC3)), "bytes after the links were written"
            out = torch.empty(V * 72, dtype=torch.float64, device="cuda")
            h.unpack(dp, host[:, :lb].contiguous().view(-1).cuda(), out)
            h.sync()
            assert oracle.error(out.cpu().numpy(), ref)[0] <= tol, tpl
    finally:
        h.set_launch_cfg(d, **saved)


@pytest.mark.parametrize("arith", [su3.NATIVE, su3.F32PAIR])
@pytest.mark.parametrize("reprs", [(su3.FULL18, su3.FULL18), (su3.TWOROW12, su3.FULL18), (su3.TWOROW12, su3.TWOROW12)],
                         ids=["full", "2row-to-full", "2row"])
def test_mixed_site_strides_bitwise(arith, reprs):
    """a and c with site strides of their own (padded a into packed c, packed a into padded c, two
    different padded strides): each gives the packed-stride bits, leaves the bytes after c's links
    alone, for one and three threads per link and tiles narrower and wider than the 32 sites one
    warp copies per pass."""
    import torch
    h = su3.Handle(0)  # its own handle: the configurations below stay local to it
    ri, ro = reprs
    V = 2777
    a, b = gen.lattice(15, V)
    dpa, dpc = su3.Desc(su3.F64, ri, su3.AOS, V, 0, arith), su3.Desc(su3.F64, ro, su3.AOS, V, 0, arith)
    la, lc = su3.array_bytes(dpa) // V, su3.array_bytes(dpc) // V  # link bytes per site
    packed_a = empty_bytes(su3.array_bytes(dpa))
    h.pack(to_dev(a), dpa, packed_a)
    ref = empty_bytes(su3.array_bytes(dpc))
    h.mult(dpa, packed_a, b, dpc, ref)
    out = torch.empty(V * 72, dtype=torch.float64, device="cuda")
    h.unpack(dpc, ref, out)
    h.sync()
    assert oracle.error(out.cpu().numpy(), oracle.mult(a, b))[0] <= (1e-13 if ri == su3.FULL18 else 1e-12)
    ref = ref.cpu()
    for sa, sc in ((la + 64, 0), (0, lc + 128), (la + 16, lc + 64)):
        da, dc = su3.Desc(su3.F64, ri, su3.AOS, V, sa, arith), su3.Desc(su3.F64, ro, su3.AOS, V, sc, arith)
        src = packed_a
        if sa:
            src = torch.full((V * sa,), 0x3C, dtype=torch.uint8, device="cuda")
            src.view(V, sa)[:, :la] = packed_a.view(V, la)
        for tiles, tpl in ((24, 1), (80, 1), (40, 3), (72, 3)):
            h.set_launch_cfg(da, block=128, tile_sites=tiles, stages=3, ctas_per_sm=2, threads_per_link=tpl)
            h.set_launch_cfg_for(da, dc, block=128, tile_sites=tiles, stages=3, ctas_per_sm=2, threads_per_link=tpl)
            dst = torch.full((V * (sc or lc),), 0xC3, dtype=torch.uint8, device="cuda")
            h.mult(da, src, b, dc, dst)
            h.sync()
            host = dst.view(V, sc or lc).cpu()
            assert torch.equal(host[:, :lc].contiguous().view(-1), ref), (sa, sc, tiles, tpl)
            if sc:
                assert bool(torch.all(host[:, lc:] == 0xC3)), "bytes after the links were written"
    h.close()


@pytest.mark.parametrize("arith", [su3.NATIVE, su3.F32PAIR])
@pytest.mark.parametrize("V", [1, 7, 65])
def test_padded_arrays_smaller_than_a_tile(h, arith, V):
    """Padded sites fewer than one tile's rows: the tensor copy's box reaches past the array (rows
    there arrive as zeros and are never stored), and the bytes after each site's links stay."""
    import torch
    a, b = gen.lattice(16, V)
    d = su3.Desc(su3.F64, su3.FULL18, su3.AOS, V, 640, arith)
    saved = h.get_launch_cfg(d)
    try:
        h.set_launch_cfg(d, block=256, tile_sites=64, stages=3, ctas_per_sm=2, threads_per_link=1)
        abuf = torch.full((V * 640,), 0x3C, dtype=torch.uint8, device="cuda")
        h.pack(to_dev(a), d, abuf)
        cbuf = torch.full_like(abuf, 0xC3)
        h.mult(d, abuf, b, d, cbuf)
        h.sync()
    finally:
        h.set_launch_cfg(d, **saved)
    host = cbuf.view(V, 640).cpu()
    assert bool(torch.all(host[:, 576:] == 0xC3)), "bytes after the links were written"
    got = host[:, :576].contiguous().view(torch.float64).numpy().reshape(-1)
    assert oracle.error(got, oracle.mult(a, b))[0] <= 1e-13


def test_canaries_packed(h):
    import torch
    V = 1237
    a, b = gen.lattice(5, V)
    for dt in (su3.F64, su3.F16):
        d = su3.Desc(dt, su3.FULL18, su3.AOS, V)
        n = su3.array_bytes(d)
        abuf = empty_bytes(n)
        h.pack(to_dev(a), d, abuf)
        cbig = torch.full((n + 8192,), 0x5A, dtype=torch.uint8, device="cuda")
        h.mult(d, abuf, b, d, cbig.data_ptr() + 4096)
        h.sync()
        host = cbig.cpu().numpy()
        assert np.all(host[:4096] == 0x5A) and np.all(host[-4096:] == 0x5A)


def test_empty_is_noop(h):
    d = su3.Desc(su3.F64, su3.FULL18, su3.AOS, 0)
    h.mult(d, 0, np.zeros(72), d, 0)
    h.sync()


def test_invalid_arguments_rejected(h):
    V = 100
    d = su3.Desc(su3.F64, su3.FULL18, su3.AOS, V)
    buf = empty_bytes(su3.array_bytes(d) + 64)
    b = np.zeros(72)
    with pytest.raises(su3.Su3Error) as e:
        h.mult(d, buf.data_ptr() + 8, b, d, buf.data_ptr() + 8)  # misaligned
    assert e.value.status == 1
    with pytest.raises(su3.Su3Error) as e:
        h.mult(d, buf.data_ptr(), b, d, buf.data_ptr() + 16)  # partial overlap
    assert e.value.status == 1
    dc = su3.Desc(su3.F32, su3.FULL18, su3.AOS, V)
    with pytest.raises(su3.Su3Error):
        h.mult(d, buf.data_ptr(), b, dc, buf.data_ptr())  # dtype mismatch
    with pytest.raises(su3.Su3Error):
        h.mult(su3.Desc(su3.F64, su3.FULL18, su3.AOS, V, 600), buf.data_ptr(), b, None, buf.data_ptr())
    with pytest.raises(su3.Su3Error):
        h.set_launch_cfg(d, block=100)
    h.sync()


def test_default_launch_cfg_reported_per_arithmetic():
    """su3_get_launch_cfg on a fresh handle reports the default each arithmetic actually runs with."""
    h = su3.Handle(0)
    nat = h.get_launch_cfg(su3.Desc(su3.F64, su3.FULL18, su3.AOS, 10, 0, su3.NATIVE))
    hyb = h.get_launch_cfg(su3.Desc(su3.F64, su3.FULL18, su3.AOS, 10, 0, su3.HYBRID))
    assert nat["native_permille"] == 0
    assert hyb["native_permille"] == 125 and hyb["block"] == 256 and hyb["tile_sites"] == 64 and hyb["stages"] == 3
    h.close()


def test_launch_cfg_variants_agree():
    """Every tile size / stage depth / block / threads per link gives the same bits (sites are
    independent, and a row computed by its own thread follows the same operation order)."""
    h = su3.Handle(0)  # its own handle: the configurations below stay local to it
    V = 7000
    a, b = gen.lattice(6, V)
    for dt, lay in ((su3.F64, su3.AOS), (su3.F16, su3.AOS), (su3.F32, su3.SOA)):
        base = run_form(h, a, b, dt, layout=lay)
        cfgs = ({"tile_sites": 7, "stages": 2, "block": 64, "threads_per_link": 1},
                {"tile_sites": 64, "stages": 3, "block": 256},
                {"tile_sites": 33, "stages": 8, "block": 128, "ctas_per_sm": 1},
                {"tile_sites": 21, "stages": 3, "block": 256, "threads_per_link": 3},
                {"tile_sites": 5, "stages": 2, "block": 64, "threads_per_link": 3})
        if lay != su3.AOS:
            cfgs = ({"tile_sites": 1, "block": 64}, {"tile_sites": 2, "block": 256}, {"tile_sites": 4, "ctas_per_sm": 1})
        for cfg in cfgs:
            assert np.array_equal(run_form(h, a, b, dt, layout=lay, cfg=cfg), base), (dt, cfg)
    h.close()


@pytest.mark.parametrize("form", [(su3.F64, su3.FULL18, su3.FULL18, su3.F32PAIR, 3),
                                  (su3.F64, su3.FULL18, su3.FULL18, su3.HYBRID, 3),
                                  (su3.F64, su3.TWOROW12, su3.TWOROW12, su3.NATIVE, 3),
                                  (su3.F64, su3.TWOROW12, su3.TWOROW12, su3.F32PAIR, 3),
                                  (su3.F32, su3.TWOROW12, su3.FULL18, su3.NATIVE, 3),
                                  (su3.F64, su3.TWOROW12, su3.FULL18, su3.NATIVE, 3),
                                  (su3.F64, su3.TWOROW12, su3.FULL18, su3.F32PAIR, 3),
                                  (su3.F64, su3.TWOROW12, su3.FULL18, su3.HYBRID, 3)],
                         ids=["pair", "hybrid", "f64-2row", "pair-2row", "f32-2row-to-full", "f64-2row-to-full",
                              "pair-2row-to-full", "hybrid-2row-to-full"])
def test_row_split_is_bitwise(form):
    """One thread per output row (threads_per_link 3; two threads for two-row output) gives the bits
    of one thread per link, for every op with rows."""
    h = su3.Handle(0)
    dt, ri, ro, arith, rows = form
    V = 3333
    a, b = gen.lattice(12, V)
    cfg1 = {"tile_sites": 64, "stages": 3, "block": 256, "threads_per_link": 1}
    cfgr = {"tile_sites": 24, "stages": 3, "block": 256, "threads_per_link": rows}
    if arith == su3.HYBRID:
        cfg1["native_permille"] = cfgr["native_permille"] = 250
    one = run_form(h, a, b, dt, ri, ro, arith=arith, cfg=cfg1)
    split = run_form(h, a, b, dt, ri, ro, arith=arith, cfg=cfgr)
    if arith == su3.HYBRID:  # warps take the native role per tile: each row is one or the other
        nat = run_form(h, a, b, dt, ri, ro, arith=su3.NATIVE).reshape(-1, 6)
        pair = run_form(h, a, b, dt, ri, ro, arith=su3.F32PAIR).reshape(-1, 6)
        s = split.reshape(-1, 6)
        assert np.all(np.all(s == nat, axis=1) | np.all(s == pair, axis=1))
    else:
        assert np.array_equal(one, split)
    h.close()


def test_threads_per_link_validation(h):
    """threads_per_link must be 1 or 3 (row split); adjacent ops keep one thread per link."""
    import torch
    d = su3.Desc(su3.F64, su3.FULL18, su3.AOS, 64)
    h2 = su3.Handle(0)
    with pytest.raises(su3.Su3Error):
        h2.set_launch_cfg(d, threads_per_link=2)
    with pytest.raises(su3.Su3Error):
        h2.set_launch_cfg(su3.Desc(su3.F64, su3.FULL18, su3.SOA, 64), threads_per_link=3)
    with pytest.raises(su3.Su3Error):
        h2.set_batched_cfg(threads_per_link=2)
    # a^dagger b and a v on a form whose configuration asks for a row split still run (one thread per link)
    h2.set_launch_cfg(d, tile_sites=24, stages=3, block=256, threads_per_link=3)
    V = 64
    a, b = gen.lattice(13, V)
    a_dev = to_dev(a)
    c = torch.empty_like(a_dev)
    h2.mult_op(su3.OP_AN, d, a_dev, b, d, c)
    w = torch.empty(V * 24, dtype=torch.float64, device="cuda")
    h2.mat_vec(d, a_dev, np.linspace(-1, 1, 24), w)
    h2.sync()
    assert oracle.error(c.cpu().numpy(), oracle.mult_an(a, b))[0] <= 1e-13
    h2.close()


def test_host_path_matches_device_path(h):
    import torch
    V = 70001
    a, b = gen.lattice(7, V)
    d = su3.Desc(su3.F64, su3.FULL18, su3.AOS, V)
    a_pin = torch.from_numpy(a).pin_memory()
    c_pin = torch.empty(V * 72, dtype=torch.float64).pin_memory()
    h.mult_host(d, a_pin.data_ptr(), b, d, c_pin.data_ptr())
    dev = run_form(h, a, b, su3.F64)
    assert np.array_equal(c_pin.numpy(), dev)
    # pageable host memory and in place
    a_page = a.copy()
    h.mult_host(d, a_page, b, d, a_page)
    assert np.array_equal(a_page, dev)


def test_sync_host_deadline(h):
    """A host deadline shorter than the queued work returns TIMEOUT; a later sync succeeds."""
    import torch
    V = 1 << 21
    d = su3.Desc(su3.F64, su3.FULL18, su3.AOS, V)
    buf = torch.zeros(su3.array_bytes(d), dtype=torch.uint8, device="cuda")
    out = torch.empty_like(buf)
    for _ in range(20):
        h.mult(d, buf, np.zeros(72), d, out)
    with pytest.raises(su3.Su3Error) as e:
        h.sync(timeout_ms=0)
    assert e.value.status == 5
    h.sync()


def test_device_bounded_wait_times_out_cleanly(h):
    """The bounded mbarrier wait gives up, the status word reports TIMEOUT, the context lives on."""
    h.selftest_wait_timeout(50)
    with pytest.raises(su3.Su3Error) as e:
        h.sync()
    assert e.value.status == 5
    h.sync()  # status word was cleared
    V = 100
    a, b = gen.lattice(8, V)
    assert oracle.error(run_form(h, a, b, su3.F64), oracle.mult(a, b))[0] <= 1e-13


def test_launch_count(h):
    n0 = h.launch_count()
    V = 100
    a, b = gen.lattice(8, V)
    run_form(h, a, b, su3.F64, iters=3)
    assert h.launch_count() - n0 == 5  # pack + 3 mult + unpack


def test_launch_cfg_per_repr_pair():
    """Two-row in, full out keeps a launch shape of its own (su3_set_launch_cfg_for); without one it
    uses the two-row in and out shape. Every shape gives the same bits."""
    h = su3.Handle(0)
    V = 4 * 8 ** 3 + 3
    a, b = gen.lattice(44, V)
    for arith in (su3.NATIVE, su3.F32PAIR):
        d2 = su3.Desc(su3.F64, su3.TWOROW12, su3.AOS, V, 0, arith)
        df = su3.Desc(su3.F64, su3.FULL18, su3.AOS, V, 0, arith)
        h.set_launch_cfg(d2, block=128, tile_sites=64, stages=3, ctas_per_sm=2, threads_per_link=1)
        assert h.get_launch_cfg_for(d2, df)["tile_sites"] == 64  # falls back to the two-row shape
        base = run_form(h, a, b, su3.F64, su3.TWOROW12, su3.FULL18, arith=arith)
        h.set_launch_cfg_for(d2, df, block=256, tile_sites=24, stages=2, ctas_per_sm=1, threads_per_link=3)
        assert h.get_launch_cfg_for(d2, df)["tile_sites"] == 24 and h.get_launch_cfg_for(d2, df)["threads_per_link"] == 3
        assert h.get_launch_cfg(d2)["tile_sites"] == 64  # the two-row in/out shape is untouched
        got = run_form(h, a, b, su3.F64, su3.TWOROW12, su3.FULL18, arith=arith)
        assert np.array_equal(got, base)
        assert oracle.error(got, oracle.mult(a, b))[0] <= 1e-12
    with pytest.raises(su3.Su3Error):  # full in, two-row out is not a supported pair
        h.set_launch_cfg_for(su3.Desc(su3.F64, su3.FULL18, su3.AOS, 8), su3.Desc(su3.F64, su3.TWOROW12, su3.AOS, 8),
                             block=128)
    h.close()


def test_measure_fp64_rate(h):
    """The FP64 FMA-rate diagnostic: a plausible rate for a GB300 (about 1.25 TFLOP/s nominal) and
    argument checks."""
    tf = h.measure_fp64_rate(2048)
    assert 0.3 < tf < 3.0, tf
    with pytest.raises(su3.Su3Error):
        h.measure_fp64_rate(0)
