"""The element-major layouts (AOSOA32, SOA) through the staged kernel: tiles moved between HBM and
shared memory by bulk copies (whole 32-link blocks for AOSOA32; for SOA one 2-D tensor copy of
every element plane's 256 links when a tile is 64 sites of 4- or 8-byte elements, one copy per
element plane otherwise; V = 1 puts a whole array inside one box), computed in place with the
element stride of the layout, and stored back the same way.

Every form against the oracle and bit for bit against the direct-load kernel (both run the same
per-link operations in the same order), ragged sizes whose last AOSOA32 block is partial, the row
split, FP32-pair arithmetic, and canaries: bytes outside c and the padding links of c's last
AOSOA32 block are never written."""
import numpy as np
import pytest

import oracle
import paper_2103_00571_gb300 as su3
import su3_inputs as gen
from gpu_helpers import empty_bytes, run_form, to_dev, tol

pytestmark = pytest.mark.gpu

FORMS = [
    (su3.F64, su3.FULL18, su3.FULL18, su3.NATIVE),
    (su3.F64, su3.FULL18, su3.FULL18, su3.F32PAIR),
    (su3.F32, su3.FULL18, su3.FULL18, su3.NATIVE),
    (su3.F16, su3.FULL18, su3.FULL18, su3.NATIVE),
    (su3.BF16, su3.FULL18, su3.FULL18, su3.NATIVE),
    (su3.F64, su3.TWOROW12, su3.TWOROW12, su3.NATIVE),
    (su3.F64, su3.TWOROW12, su3.TWOROW12, su3.F32PAIR),
    (su3.F32, su3.TWOROW12, su3.FULL18, su3.NATIVE),
    (su3.F64, su3.TWOROW12, su3.FULL18, su3.F32PAIR),
    (su3.F16, su3.TWOROW12, su3.TWOROW12, su3.NATIVE),
]
STAGED = {
    su3.AOSOA32: [{"tile_sites": 64, "stages": 3, "block": 256},
                  {"tile_sites": 8, "stages": 2, "block": 32},
                  {"tile_sites": 40, "stages": 4, "block": 128, "threads_per_link": 3}],
    su3.SOA: [{"tile_sites": 64, "stages": 3, "block": 256},
              {"tile_sites": 13, "stages": 2, "block": 64},
              {"tile_sites": 32, "stages": 3, "block": 128, "threads_per_link": 3}],
}
DIRECT = {"stages": 0, "tile_sites": 1, "block": 256}
SIZES = [1, 4096 + 13, 3 * 8 ** 3 + 5]


def _name(f):
    return "%s-%s-%s-%s" % ({0: "f64", 1: "f32", 2: "f16", 3: "bf16"}[f[0]], f[1], f[2],
                            {0: "native", 1: "pair", 2: "hybrid"}[f[3]])


@pytest.fixture(scope="module")
def h():
    hh = su3.Handle(0)
    yield hh
    hh.close()


@pytest.mark.parametrize("layout", [su3.AOSOA32, su3.SOA], ids=["aosoa32", "soa"])
@pytest.mark.parametrize("form", FORMS, ids=[_name(f) for f in FORMS])
@pytest.mark.parametrize("V", SIZES)
def test_staged_matches_oracle_and_direct(h, form, layout, V):
    dt, ri, ro, arith = form
    a, b = gen.lattice(21, V)
    ref = oracle.mult(a, b)
    direct = run_form(h, a, b, dt, ri, ro, layout, cfg=DIRECT, arith=arith)
    for cfg in STAGED[layout]:
        got = run_form(h, a, b, dt, ri, ro, layout, cfg=cfg, arith=arith)
        assert oracle.error(got, ref)[0] <= tol(dt, ri, ro), cfg
        assert np.array_equal(got, direct), cfg


@pytest.mark.parametrize("layout", [su3.AOSOA32, su3.SOA], ids=["aosoa32", "soa"])
@pytest.mark.parametrize("dt", [su3.F64, su3.F16])
def test_staged_canaries_and_padding(h, layout, dt):
    """c sits 4 KiB inside a buffer of canary bytes: nothing outside c changes, and for AOSOA32 the
    padding links of the last, partial block keep their bytes (only c's real links are written)."""
    import torch
    V = 4096 + 13  # 16,436 links: the last AOSOA32 block holds 20 real links and 12 padding links
    a, b = gen.lattice(22, V)
    d = su3.Desc(dt, su3.FULL18, layout, V)
    n = su3.array_bytes(d)
    abuf = empty_bytes(n)
    h.pack(to_dev(a), d, abuf)
    h.set_launch_cfg(d, tile_sites=64, stages=3, block=256)
    try:
        cbig = torch.full((n + 8192,), 0x5A, dtype=torch.uint8, device="cuda")
        h.mult(d, abuf, b, d, cbig.data_ptr() + 4096)
        h.sync()
        host = cbig.cpu().numpy()
        assert np.all(host[:4096] == 0x5A) and np.all(host[-4096:] == 0x5A)
        if layout == su3.AOSOA32:
            vec = 16 if dt == su3.F64 else 4
            n_links, blk = 4 * V, (4 * V) // 32
            real = n_links - 32 * blk
            tail = host[4096 + blk * 9 * 32 * vec: 4096 + n].reshape(9, 32 * vec)
            assert real == 20
            assert np.all(tail[:, real * vec:] == 0x5A)  # padding links untouched
            assert not np.all(tail[:, :real * vec] == 0x5A)
        # and the real links are right
        out = torch.empty(V * 72, dtype=torch.float64, device="cuda")
        h.unpack(d, cbig[4096:4096 + n], out)
        h.sync()
        assert oracle.error(out.cpu().numpy(), oracle.mult(a, b))[0] <= tol(dt, su3.FULL18)
    finally:
        h.set_launch_cfg(d, **DIRECT)


def test_staged_config_validation(h):
    with pytest.raises(su3.Su3Error):  # AOSOA32 tiles are whole 32-link blocks
        h.set_launch_cfg(su3.Desc(su3.F64, su3.FULL18, su3.AOSOA32, 64), tile_sites=12, stages=3)
    with pytest.raises(su3.Su3Error):  # an SOA tile's element planes hold 256 links
        h.set_launch_cfg(su3.Desc(su3.F32, su3.FULL18, su3.SOA, 64), tile_sites=65, stages=3)
    with pytest.raises(su3.Su3Error):  # direct loads: one thread per link
        h.set_launch_cfg(su3.Desc(su3.F32, su3.FULL18, su3.SOA, 64), tile_sites=2, threads_per_link=3)
    d = su3.Desc(su3.F32, su3.FULL18, su3.SOA, 64)
    h.set_launch_cfg(d, tile_sites=16, stages=2, threads_per_link=3)
    assert h.get_launch_cfg(d)["stages"] == 2
    h.set_launch_cfg(d, **DIRECT)
    assert h.get_launch_cfg(d)["stages"] == 0
