"""Helpers shared by the GPU tests: move FP64 sites to the device, run one form of the operation
through the C ABI (pack -> mult -> unpack), and the tolerances each form is held to."""
import numpy as np

import paper_2103_00571_gb300 as su3

# Max-abs tolerance of each form against the FP64 oracle (values are SU(3) entries, |x| <= 1).
# FP64: the analytic error of three complex MACs is a few ulp (~1e-15); 1e-13 leaves margin for
# FMA contraction. FP32 storage + math: input/output rounding 2^-24 relative through sum |b| <= sqrt3
# gives ~5e-7. Two-row: row 2 rebuilt from rounded rows adds a few ulp. FP16: half-ulp 2^-12 on
# [0.5, 1) through sqrt3 plus output rounding ~1e-3. BF16: half-ulp 2^-9 -> ~8e-3.
TOL = {
    (su3.F64, su3.FULL18): 1e-13,
    (su3.F64, su3.TWOROW12): 1e-12,
    (su3.F32, su3.FULL18): 2e-6,
    (su3.F32, su3.TWOROW12): 5e-6,
    (su3.F16, su3.FULL18): 5e-3,
    (su3.F16, su3.TWOROW12): 5e-3,
    (su3.BF16, su3.FULL18): 3e-2,
    (su3.BF16, su3.TWOROW12): 3e-2,
}


def torch():
    import torch as t
    return t


def to_dev(x):
    t = torch()
    return t.from_numpy(np.ascontiguousarray(x)).cuda()


def empty_bytes(n, fill=None):
    t = torch()
    buf = t.empty(max(int(n), 16), dtype=t.uint8, device="cuda")
    if fill is not None:
        buf.fill_(fill)
    return buf


def run_form(h, a64, b, dtype, repr_in=su3.FULL18, repr_out=None, layout=su3.AOS, stride=0, cfg=None,
             iters=1, stream=None, arith=su3.NATIVE):
    """pack(a64) -> mult x iters -> unpack; returns the FP64 result as a numpy array [V*72]."""
    t = torch()
    repr_out = repr_in if repr_out is None else repr_out
    V = a64.size // 72
    a_src = to_dev(a64)
    da = su3.Desc(dtype, repr_in, layout, V, stride, arith)
    dc = su3.Desc(dtype, repr_out, layout, V, stride, arith)
    abuf = empty_bytes(su3.array_bytes(da))
    cbuf = empty_bytes(su3.array_bytes(dc))
    h.pack(a_src, da, abuf, stream)
    if cfg:
        h.set_launch_cfg(da, **cfg)
    for _ in range(iters):
        h.mult(da, abuf, b, dc, cbuf, stream)
    out = t.empty(V * 72, dtype=t.float64, device="cuda")
    h.unpack(dc, cbuf, out, stream)
    h.sync(stream)
    return out.cpu().numpy()


def tol(dtype, repr_in, repr_out=None):
    r = repr_in if repr_out is None or repr_in == repr_out else su3.TWOROW12
    return TOL[(dtype, r)]
