"""The benchmark's own sizes, in the launch configuration bench.py times (tuned or default):
L=32, L=48 and the FP64 L=64 step compared element by element over the whole lattice; every
other L=64 form on sampled sites the oracle recomputes one by one."""
import numpy as np
import pytest

import oracle
import paper_2103_00571_gb300 as su3
import su3_inputs as gen
from gpu_helpers import run_form, tol

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def h():
    from paper_2103_00571_gb300 import tune
    hd = su3.Handle(0)
    tune.apply_cached(hd)
    return hd


def test_L32_f64_aos_full_compare(h):
    V = 32 ** 4
    a, b = gen.lattice(gen.DEFAULT_SEED, V)
    got = run_form(h, a, b, su3.F64)
    mx, rms = oracle.error(got, oracle.mult(a, b))
    assert mx <= 1e-13, (mx, rms)


@pytest.mark.parametrize("form", [(su3.F64, su3.FULL18, su3.AOS), (su3.F32, su3.FULL18, su3.AOS),
                                  (su3.F64, su3.TWOROW12, su3.AOS), (su3.F32, su3.TWOROW12, su3.AOS),
                                  (su3.F64, su3.FULL18, su3.SOA), (su3.F32, su3.FULL18, su3.SOA),
                                  (su3.F64, su3.FULL18, su3.AOSOA32)],
                         ids=["f64-aos", "f32-aos", "f64-2row-aos", "f32-2row-aos", "f64-soa", "f32-soa",
                              "f64-aosoa32"])
def test_L48_forms_full_compare(h, form, L48):
    dt, rep, lay = form
    a, b, ref = L48
    got = run_form(h, a, b, dt, rep, rep, lay)
    mx, rms = oracle.error(got, ref)
    assert mx <= tol(dt, rep), (mx, rms)


@pytest.fixture(scope="module")
def L48():
    V = 48 ** 4
    a, b = gen.lattice(gen.DEFAULT_SEED, V)
    return a, b, oracle.mult(a, b)


F64, F32, F16, BF16 = su3.F64, su3.F32, su3.F16, su3.BF16
NAT, PAIR, FULL, TWO = su3.NATIVE, su3.F32PAIR, su3.FULL18, su3.TWOROW12
AOS, SOA, AOSOA = su3.AOS, su3.SOA, su3.AOSOA32


@pytest.mark.parametrize("dtype,arith,rep,rep_out,layout,stride", [
    (F64, NAT, FULL, FULL, AOS, 0), (F64, PAIR, FULL, FULL, AOS, 0), (F16, NAT, FULL, FULL, AOS, 0),
    (BF16, NAT, FULL, FULL, AOS, 0), (F32, NAT, FULL, FULL, AOS, 0), (F64, NAT, FULL, FULL, SOA, 0),
    (F16, NAT, FULL, FULL, SOA, 0), (F32, NAT, FULL, FULL, SOA, 0),
    (F64, PAIR, FULL, FULL, AOSOA, 0), (F16, NAT, FULL, FULL, AOSOA, 0), (F64, PAIR, TWO, TWO, AOS, 0),
    (F32, NAT, TWO, TWO, AOS, 0), (F64, PAIR, TWO, FULL, AOS, 0), (F64, NAT, TWO, FULL, AOS, 0),
    (F64, NAT, FULL, FULL, AOS, 640), (F64, PAIR, FULL, FULL, AOS, 640)],
    ids=["f64", "f64-f32pair", "f16", "bf16", "f32", "f64-soa", "f16-soa", "f32-soa", "f64-f32pair-aosoa32",
         "f16-aosoa32", "f64-f32pair-2row", "f32-2row", "f64-f32pair-2row-to-full", "f64-2row-to-full",
         "f64-site640", "f64-f32pair-site640"])
def test_L64_sampled(h, dtype, arith, rep, rep_out, layout, stride):
    """L=64 (16.7M sites, every array past 2^32 bytes for FP64): the whole lattice runs on the GPU
    in the tuned launch configuration (SoA tiles through tensor copies, two-row in / full out
    through per-warp output copies, the paper's 640-byte sites through the padded kernel); 65,536
    random sites are recomputed by the oracle from the same generator and compared element by
    element."""
    import torch
    V = 64 ** 4
    a = gen.sites(gen.DEFAULT_SEED, 0, V)
    b = gen.bmat(gen.DEFAULT_SEED, 0, V)
    a_dev = torch.from_numpy(a).cuda()
    del a
    d = su3.Desc(dtype, rep, layout, V, stride, arith)
    dc = su3.Desc(dtype, rep_out, layout, V, stride, arith)
    if dtype == su3.F64 and rep == su3.FULL18 and layout == su3.AOS and not stride:
        abuf = a_dev
    else:
        abuf = torch.empty(su3.array_bytes(d), dtype=torch.uint8, device="cuda")
        h.pack(a_dev, d, abuf)
    cbuf = torch.empty(su3.array_bytes(dc), dtype=torch.uint8, device="cuda")
    h.mult(d, abuf, b, dc, cbuf)
    out = a_dev if abuf is not a_dev else torch.empty_like(a_dev)
    h.unpack(dc, cbuf, out)
    h.sync()
    del abuf, cbuf
    idx = np.sort(np.random.default_rng(64).choice(V, 65536, replace=False))
    idx[0], idx[-1] = 0, V - 1  # both ends of the lattice
    got = out.view(V, 72)[torch.from_numpy(idx).cuda()].cpu().numpy()
    ref = oracle.mult_sites(gen.sites_at(gen.DEFAULT_SEED, 0, idx), b)
    mx, rms = oracle.error(got, ref)
    assert mx <= tol(dtype, rep, rep_out), (mx, rms)


@pytest.mark.parametrize("arith", [su3.NATIVE, su3.F32PAIR], ids=["native", "f32pair"])
def test_L64_f64_aos_full_compare(h, arith):
    """The bench step itself: the whole L=64 lattice (16,777,216 sites, 1.2 G reals) against the
    oracle element by element, from a and c in the same device buffers bench.py uses."""
    import torch
    V = 64 ** 4
    a = torch.empty(V * 72, dtype=torch.float64, pin_memory=True)
    gen.sites(gen.DEFAULT_SEED, 0, V, out=a.numpy())
    b = gen.bmat(gen.DEFAULT_SEED, 0, V)
    a_dev = a.cuda()
    c_dev = torch.empty_like(a_dev)
    d = su3.Desc(su3.F64, su3.FULL18, su3.AOS, V, 0, arith)
    h.mult(d, a_dev, b, d, c_dev)
    h.sync()
    got = c_dev.cpu().numpy()
    del a_dev, c_dev
    ref = oracle.mult(a.numpy(), b)
    mx, rms = oracle.error(got, ref)
    assert mx <= 1e-13, (mx, rms)


def test_every_bench_form_under_tuned_configs(h):
    """Each form bench.py times, with the tuned launch configurations installed (the same handle
    set-up bench.py uses), on a lattice spanning many tiles: within its tolerance of the oracle."""
    import bench
    V = 6 * 8 ** 3 + 11
    a, b = gen.lattice(5, V)
    ref = oracle.mult(a, b)
    for name, dt, ri, ro, lay, *ar in bench.FORMS:
        got = run_form(h, a, b, dt, ri, ro, lay, arith=ar[0] if ar else su3.NATIVE)
        mx, _ = oracle.error(got, ref)
        assert mx <= tol(dt, ri, ro), (name, mx)
    for arith in (su3.NATIVE, su3.F32PAIR):  # the paper's 640-byte Site (bench.py's paper_site640 leg)
        got = run_form(h, a, b, su3.F64, stride=640, arith=arith)
        mx, _ = oracle.error(got, ref)
        assert mx <= 1e-13, ("site640", arith, mx)


@pytest.mark.parametrize("arith", [su3.NATIVE, su3.F32PAIR], ids=["native", "f32pair"])
def test_L64_adjacent_sampled(h, arith):
    """The adjacent products bench.py times at L=64 (a b^dagger, a^dagger b, a v, a^dagger v) on the
    whole FP64 lattice in HBM, compared with the oracle on 65,536 sampled sites."""
    import torch
    V = 64 ** 4
    a = gen.sites(gen.DEFAULT_SEED, 0, V)
    b = gen.bmat(gen.DEFAULT_SEED, 0, V)
    a_dev = torch.from_numpy(a).cuda()
    del a
    d = su3.Desc(su3.F64, su3.FULL18, su3.AOS, V, 0, arith)
    idx = np.sort(np.random.default_rng(65).choice(V, 65536, replace=False))
    idx[0], idx[-1] = 0, V - 1
    sel = torch.from_numpy(idx).cuda()
    a_sel = gen.sites_at(gen.DEFAULT_SEED, 0, idx)
    c = torch.empty_like(a_dev)
    for op, ref in ((su3.OP_NA, oracle.mult_na), (su3.OP_AN, oracle.mult_an)):
        c.fill_(float("nan"))
        h.mult_op(op, d, a_dev, b, d, c)
        h.sync()
        got = c.view(V, 72)[sel].cpu().numpy()
        assert oracle.error(got, ref(a_sel, b))[0] <= 1e-13, op
    del c
    v = np.random.default_rng(64).standard_normal(24) / 2.0
    w = torch.empty(V * 24, dtype=torch.float64, device="cuda")
    for adjoint in (False, True):
        w.fill_(float("nan"))
        h.mat_vec(d, a_dev, v, w, adjoint=adjoint)
        h.sync()
        got = w.view(V, 24)[sel].cpu().numpy()
        assert oracle.error(got, oracle.mat_vec(a_sel, v, adjoint=adjoint))[0] <= 1e-13, adjoint
