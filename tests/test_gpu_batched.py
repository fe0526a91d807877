"""Batched path: 96 lattices with extents drawn from {4, 6, ..., 24}, mixed FP64/FP32, one
persistent launch (optionally a CUDA graph), each lattice against its own oracle and bitwise
against the single-lattice kernel."""
import ctypes

import numpy as np
import pytest

import oracle
import paper_2103_00571_gb300 as su3
import su3_inputs as gen
from gpu_helpers import empty_bytes, to_dev

pytestmark = pytest.mark.gpu


def make_batch(h, n, seed=2103, max_extent=None):
    import torch
    ext = gen.extents(seed, n)
    if max_extent:
        ext = np.minimum(ext, max_extent)
    lat = []
    for k in range(n):
        V = int(np.prod(ext[k]))
        a, b = gen.lattice(seed, V, lattice_id=k)
        dt = su3.F64 if k % 2 == 0 else su3.F32
        d = su3.Desc(dt, su3.FULL18, su3.AOS, V)
        abuf = empty_bytes(su3.array_bytes(d))
        h.pack(to_dev(a), d, abuf)
        cbuf = empty_bytes(su3.array_bytes(d))
        item = su3.BatchItem(d, abuf.data_ptr(), cbuf.data_ptr(), (ctypes.c_double * 72)(*b))
        lat.append(dict(a=a, b=b, d=d, abuf=abuf, cbuf=cbuf, item=item, V=V, dt=dt))
    h.sync()
    return lat


def unpack(h, L):
    import torch
    out = torch.empty(L["V"] * 72, dtype=torch.float64, device="cuda")
    h.unpack(L["d"], L["cbuf"], out)
    h.sync()
    return out.cpu().numpy()


@pytest.fixture(scope="module")
def h():
    return su3.Handle(0)


@pytest.mark.parametrize("use_graph", [False, True])
def test_batched_vs_oracle_and_single(h, use_graph):
    lat = make_batch(h, 96, max_extent=12)
    h.mult_batched([L["item"] for L in lat], use_graph=use_graph)
    h.sync()
    outs = [unpack(h, L) for L in lat]
    for L, got in zip(lat, outs):
        tol = 1e-13 if L["dt"] == su3.F64 else 2e-6
        assert oracle.error(got, oracle.mult(L["a"], L["b"]))[0] <= tol
    # bitwise equal to the single-lattice kernel
    for L, got in zip(lat[:12], outs[:12]):
        single = empty_bytes(su3.array_bytes(L["d"]))
        h.mult(L["d"], L["abuf"], L["b"], L["d"], single)
        import torch
        o = torch.empty(L["V"] * 72, dtype=torch.float64, device="cuda")
        h.unpack(L["d"], single, o)
        h.sync()
        assert np.array_equal(o.cpu().numpy(), got)


def test_graph_replay_and_rebuild(h):
    lat = make_batch(h, 10, seed=7)
    items = [L["item"] for L in lat]
    n0 = h.launch_count()
    for _ in range(3):
        h.mult_batched(items, use_graph=True)
    h.sync()
    assert h.launch_count() - n0 == 3
    for L in lat:
        assert oracle.error(unpack(h, L), oracle.mult(L["a"], L["b"]))[0] <= 2e-6
    # a changed b forces a new graph
    b2 = gen.bmat(99, 0, 1)
    items[0].b[:] = list(b2)
    h.mult_batched(items, use_graph=True)
    h.sync()
    tol = 1e-13 if lat[0]["dt"] == su3.F64 else 2e-6
    assert oracle.error(unpack(h, lat[0]), oracle.mult(lat[0]["a"], b2))[0] <= tol


def test_batched_empty_and_rejects(h):
    h.mult_batched([], use_graph=False)
    d = su3.Desc(su3.F16, su3.FULL18, su3.AOS, 10)
    buf = empty_bytes(su3.array_bytes(d))
    with pytest.raises(su3.Su3Error):
        h.mult_batched([su3.BatchItem(d, buf.data_ptr(), buf.data_ptr())], use_graph=False)
    z = su3.Desc(su3.F64, su3.FULL18, su3.AOS, 0)
    h.mult_batched([su3.BatchItem(z, 0, 0)], use_graph=False)
    h.sync()


def test_batched_f32pair_items(h):
    """FP64 lattices in FP32-pair arithmetic inside the batched launch: within the FP64 tolerance
    of the oracle and bit for bit the single-lattice F32PAIR kernel's result."""
    import torch
    lat = make_batch(h, 16, seed=31, max_extent=10)
    for L in lat:
        if L["dt"] == su3.F64:
            L["d"] = su3.Desc(su3.F64, su3.FULL18, su3.AOS, L["V"], 0, su3.F32PAIR)
            L["item"].desc = L["d"]
    for use_graph in (False, True):
        h.mult_batched([L["item"] for L in lat], use_graph=use_graph)
        h.sync()
        for L in lat:
            got = unpack(h, L)
            tol = 1e-13 if L["dt"] == su3.F64 else 2e-6
            assert oracle.error(got, oracle.mult(L["a"], L["b"]))[0] <= tol
            if L["dt"] == su3.F64:
                single = empty_bytes(su3.array_bytes(L["d"]))
                h.mult(L["d"], L["abuf"], L["b"], L["d"], single)
                o = torch.empty(L["V"] * 72, dtype=torch.float64, device="cuda")
                h.unpack(L["d"], single, o)
                h.sync()
                assert np.array_equal(o.cpu().numpy(), got)


def test_batched_many_small_lattices(h):
    """Hundreds of lattices of 1..97 sites (FP64, FP32 and FP64 in FP32 pairs) under small tiles:
    many lattices fall between two tiles of one CTA, FP32 lattices take twice the sites per tile,
    and most tiles are ragged. Each lattice against its own oracle, with and without a graph."""
    import torch
    saved = h.get_batched_cfg()
    try:
        h.set_batched_cfg(block=64, tile_sites=8, stages=3, ctas_per_sm=2)
        lat = []
        for k in range(300):
            V = 1 + (k * 37) % 97
            a, b = gen.lattice(41, V, lattice_id=k)
            kind = k % 3
            dt = su3.F32 if kind == 1 else su3.F64
            d = su3.Desc(dt, su3.FULL18, su3.AOS, V, 0, su3.F32PAIR if kind == 2 else su3.NATIVE)
            abuf = empty_bytes(su3.array_bytes(d))
            h.pack(to_dev(a), d, abuf)
            cbuf = empty_bytes(su3.array_bytes(d))
            item = su3.BatchItem(d, abuf.data_ptr(), cbuf.data_ptr(), (ctypes.c_double * 72)(*b))
            lat.append(dict(a=a, b=b, d=d, abuf=abuf, cbuf=cbuf, item=item, V=V, dt=dt))
        h.sync()
        for use_graph in (False, True):
            for L in lat:
                L["cbuf"].fill_(0)
            h.mult_batched([L["item"] for L in lat], use_graph=use_graph)
            h.sync()
            for L in lat:
                tol = 1e-13 if L["dt"] == su3.F64 else 2e-6
                assert oracle.error(unpack(h, L), oracle.mult(L["a"], L["b"]))[0] <= tol
    finally:
        h.set_batched_cfg(**saved)
        torch.cuda.synchronize()


def test_batched_row_split_is_bitwise(h):
    """threads_per_link 3 (one thread per output row) in the batched kernel gives the bits of one
    thread per link, for FP64, FP32 and FP32-pair lattices, with and without a graph."""
    saved = h.get_batched_cfg()
    try:
        lat = make_batch(h, 24, seed=53, max_extent=10)
        for k, L in enumerate(lat):
            if L["dt"] == su3.F64 and k % 4 == 0:
                L["d"] = su3.Desc(su3.F64, su3.FULL18, su3.AOS, L["V"], 0, su3.F32PAIR)
                L["item"].desc = L["d"]
        outs = {}
        for tpl in (1, 3):
            h.set_batched_cfg(block=128, tile_sites=16, stages=3, ctas_per_sm=2, threads_per_link=tpl)
            for use_graph in (False, True):
                h.mult_batched([L["item"] for L in lat], use_graph=use_graph)
                h.sync()
                outs[(tpl, use_graph)] = [unpack(h, L) for L in lat]
        for key, got in outs.items():
            for x, y in zip(got, outs[(1, False)]):
                assert np.array_equal(x, y), key
        for L, got in zip(lat, outs[(3, True)]):
            tol = 1e-13 if L["dt"] == su3.F64 else 2e-6
            assert oracle.error(got, oracle.mult(L["a"], L["b"]))[0] <= tol
    finally:
        h.set_batched_cfg(**saved)


@pytest.mark.parametrize("f64_arith", ["native", "f32pair"])
def test_batched_full_bench_mix_vs_oracle(h, f64_arith):
    """The 96-lattice workload exactly as bench.py times it: extents drawn from {4, 6, ..., 24}
    with no cap (2,972,320 sites, lattices up to 331,776 sites), even lattices FP64 and odd FP32,
    one persistent launch replayed from a CUDA graph, the FP64 lattices in plain FP64 or in FP32
    pairs. Every element of every lattice is compared with the oracle (1e-13 FP64, 2e-6 FP32)."""
    import torch
    lat = make_batch(h, 96)
    assert sum(L["V"] for L in lat) == int(np.prod(gen.extents(2103, 96), axis=1).sum())
    assert max(L["V"] for L in lat) > 100000  # the large lattices the capped tests never reach
    if f64_arith == "f32pair":
        for L in lat:
            if L["dt"] == su3.F64:
                L["d"] = su3.Desc(su3.F64, su3.FULL18, su3.AOS, L["V"], 0, su3.F32PAIR)
                L["item"].desc = L["d"]
    items = [L["item"] for L in lat]
    for rep in range(2):  # the capture, then a replay of the same graph
        for L in lat:
            L["cbuf"].fill_(0xFF)  # NaN bytes: every output must be rewritten
        h.mult_batched(items, use_graph=True)
        h.sync()
        for L in lat:
            ref = oracle.mult(L["a"], L["b"])
            tol = 1e-13 if L["dt"] == su3.F64 else 2e-6
            err = oracle.error(unpack(h, L), ref)[0]
            assert err <= tol, (rep, L["V"], L["dt"], err)
    del lat
    torch.cuda.empty_cache()
