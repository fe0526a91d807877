"""su3_mult_batched_static: the batched launch for callers that cannot allocate device memory.

Such callers (plug-ins whose host application owns every device allocation, loops that must not
stall on cudaMalloc/cudaFree) get an entry point that takes no handle and keeps its descriptor
table in a statically allocated device area. This test calls it through the C ABI, twice in a
row on different inputs, and checks that each result equals, bit for bit, what the existing
su3_mult_batched entry point produces (both run the same kernel with the same configuration), and
that every lattice matches the FP64 oracle. The batch holds 40 lattices mixing FP64, FP32 and
FP64 in FP32-pair arithmetic. The file is named so that pytest collects it last; it also passes on
its own in a fresh process.
"""
import ctypes

import numpy as np
import pytest

import oracle
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
        kind = k % 3  # 0: FP64 native, 1: FP32, 2: FP64 in FP32 pairs
        dt = su3.F32 if kind == 1 else su3.F64
        d = su3.Desc(dt, su3.FULL18, su3.AOS, V, 0, su3.F32PAIR if kind == 2 else su3.NATIVE)
        a, b = gen.lattice(seed, V, lattice_id=k)
        abuf = torch.empty(su3.array_bytes(d), dtype=torch.uint8, device="cuda")
        h.pack(torch.from_numpy(a).cuda(), d, abuf)
        out.append(dict(d=d, V=V, dt=dt, a=a, abuf=abuf, b=b,
                        c_ref=torch.full_like(abuf, 0x7F), c_new=torch.full_like(abuf, 0x7F)))
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
        lat = _lattices(h, seed, 40)
        assert len(lat) > 16 and any(L["d"].arith == su3.F32PAIR for L in lat)
        h.mult_batched(_items(lat, "c_ref"), use_graph=False)
        h.sync()
        arr = (su3.BatchItem * len(lat))(*_items(lat, "c_new"))
        status = lib.su3_mult_batched_static(len(lat), arr, ctypes.c_void_p(stream))
        assert status == 0, (call, lib.su3_status_string(status))
        for L in lat:
            assert torch.equal(L["c_new"], L["c_ref"]), (call, L["V"], L["d"].arith)  # same bytes
            got = _as_f64(h, L, "c_new")
            err = oracle.error(got, oracle.mult(L["a"], L["b"]))[0]
            assert err <= TOL[L["dt"]], (call, L["V"], err)
    # beyond the stated maximum: rejected before anything runs
    z = lat[0]
    too_many = (su3.BatchItem * 257)(
        *[su3.BatchItem(z["d"], z["abuf"].data_ptr(), z["c_new"].data_ptr()) for _ in range(257)])
    assert lib.su3_mult_batched_static(257, too_many, ctypes.c_void_p(stream)) == 1
    h.close()
