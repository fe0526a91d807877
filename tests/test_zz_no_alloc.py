"""su3_mult_batched_static: the batched launch for callers that cannot allocate device memory.

Such callers (plug-ins whose host application owns every device allocation, loops that must not
stall on cudaMalloc/cudaFree) get an entry point that takes no handle and keeps its descriptor
table in a statically allocated device area. This test calls it through the C ABI, twice in a
row, and checks each result against the existing su3_mult_batched entry point. The file is named
so that pytest collects it last; it also passes on its own in a fresh process.
"""
import ctypes

import numpy as np
import pytest

import paper_2103_00571_gb300 as su3
import su3_inputs as gen

pytestmark = pytest.mark.gpu

TOL = {su3.F64: 1e-13, su3.F32: 2e-6}


def _lattices(h, seed, n):
    import torch
    ext = np.minimum(gen.extents(seed, n), 10)
    out = []
    for k in range(n):
        V = int(np.prod(ext[k]))
        dt = su3.F64 if k % 2 == 0 else su3.F32
        d = su3.Desc(dt, su3.FULL18, su3.AOS, V)
        a64 = torch.from_numpy(gen.sites(seed, k, V)).cuda()
        abuf = torch.empty(su3.array_bytes(d), dtype=torch.uint8, device="cuda")
        h.pack(a64, d, abuf)
        b = gen.bmat(seed, k, V)
        out.append(dict(d=d, V=V, dt=dt, abuf=abuf, b=b,
                        c_ref=torch.empty_like(abuf), c_new=torch.full_like(abuf, 0x7F)))
    h.sync()
    return out


def _items(lat, key):
    return [su3.BatchItem(L["d"], L["abuf"].data_ptr(), L[key].data_ptr(), (ctypes.c_double * 72)(*L["b"]))
            for L in lat]


def _as_f64(h, L, key):
    import torch
    o = torch.empty(L["V"] * 72, dtype=torch.float64, device="cuda")
    h.unpack(L["d"], L[key], o)
    h.sync()
    return o.cpu().numpy()


def test_static_entry_matches_batched_twice():
    import torch
    h = su3.Handle(0)
    lib = su3.lib()
    stream = torch.cuda.current_stream().cuda_stream
    for call, seed in enumerate((2103, 4242)):  # two calls in a row, different inputs
        lat = _lattices(h, seed, 24)
        h.mult_batched(_items(lat, "c_ref"), use_graph=False)
        h.sync()
        arr = (su3.BatchItem * len(lat))(*_items(lat, "c_new"))
        status = lib.su3_mult_batched_static(len(lat), arr, ctypes.c_void_p(stream))
        assert status == 0, (call, lib.su3_status_string(status))
        for L in lat:
            ref = _as_f64(h, L, "c_ref")
            got = _as_f64(h, L, "c_new")
            assert np.max(np.abs(got - ref)) <= TOL[L["dt"]], (call, L["V"])
    # beyond the stated maximum: rejected before anything runs
    z = lat[0]
    too_many = (su3.BatchItem * 257)(
        *[su3.BatchItem(z["d"], z["abuf"].data_ptr(), z["c_new"].data_ptr()) for _ in range(257)])
    assert lib.su3_mult_batched_static(257, too_many, ctypes.c_void_p(stream)) == 1
    h.close()
