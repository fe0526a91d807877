"""su3_mult captured in a CUDA graph and replayed: the launch path (descriptor checks, launch
configuration, tensor-map encoding for SoA tiles and padded sites) only enqueues work on the given
stream, so a captured call replays to the same bits as the eager call. The eager call comes first
and warms the launch path, as a capture's warm-up does."""
import numpy as np
import pytest

import oracle
import paper_2103_00571_gb300 as su3
import su3_inputs as gen
from gpu_helpers import empty_bytes, to_dev

pytestmark = pytest.mark.gpu

# (dtype, repr in, repr out, layout, site stride, arith, launch configuration or None)
CASES = [
    (su3.F64, su3.FULL18, su3.FULL18, su3.AOS, 0, su3.NATIVE, None),
    (su3.F64, su3.FULL18, su3.FULL18, su3.AOS, 0, su3.F32PAIR, None),
    (su3.F32, su3.FULL18, su3.FULL18, su3.SOA, 0, su3.NATIVE, dict(tile_sites=64, stages=3, block=128)),
    (su3.F64, su3.FULL18, su3.FULL18, su3.AOS, 640, su3.F32PAIR, None),
    (su3.F64, su3.TWOROW12, su3.FULL18, su3.AOS, 0, su3.F32PAIR, None),
]
IDS = ["f64-native", "f64-f32pair", "f32-soa-tensor", "f64-f32pair-site640", "f64-f32pair-2row-to-full"]


@pytest.mark.parametrize("case", CASES, ids=IDS)
def test_mult_replays_from_a_cuda_graph(case):
    import torch
    dt, ri, ro, lay, stride, arith, cfg = case
    h = su3.Handle(0)
    V = 3 * 8 ** 3 + 5
    a, b = gen.lattice(17, V)
    da = su3.Desc(dt, ri, lay, V, stride, arith)
    dc = su3.Desc(dt, ro, lay, V, stride, arith)
    if cfg:
        h.set_launch_cfg_for(da, dc, **cfg)
    abuf = empty_bytes(su3.array_bytes(da), fill=0)
    h.pack(to_dev(a), da, abuf)
    eager = empty_bytes(su3.array_bytes(dc), fill=0xFF)  # padded sites: the tails keep this byte
    captured = empty_bytes(su3.array_bytes(dc), fill=0xFF)
    h.mult(da, abuf, b, dc, eager)
    h.sync()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        h.mult(da, abuf, b, dc, captured, s)
    for _ in range(2):
        captured.fill_(0xFF)
        g.replay()
        torch.cuda.synchronize()
        assert torch.equal(captured, eager), "the replayed graph differs from the eager call"
    out = torch.empty(V * 72, dtype=torch.float64, device="cuda")
    h.unpack(dc, captured, out)
    h.sync()
    tol = 1e-13 if (dt, ri) == (su3.F64, su3.FULL18) else (1e-12 if dt == su3.F64 else 2e-6)
    assert oracle.error(out.cpu().numpy(), oracle.mult(a, b))[0] <= tol
    assert np.isfinite(out.cpu().numpy()).all()
    del g
    h.close()
