"""The adjacent SU(3) products (a b^dagger, a^dagger b, a v, a^dagger v) against the oracle."""
import numpy as np
import pytest

import oracle
import paper_2103_00571_gb300 as su3
import su3_inputs as gen
from gpu_helpers import TOL, empty_bytes, to_dev

pytestmark = pytest.mark.gpu

SIZES = [1, 4096 + 13, 3 * 8 ** 3 + 5]
DTYPES = [su3.F64, su3.F32, su3.F16, su3.BF16]
IDS = ["f64", "f32", "f16", "bf16"]


@pytest.fixture(scope="module")
def h():
    return su3.Handle(0)


def _packed(h, a64, dtype, stride=0):
    V = a64.size // 72
    d = su3.Desc(dtype, su3.FULL18, su3.AOS, V, stride)
    buf = empty_bytes(su3.array_bytes(d))
    h.pack(to_dev(a64), d, buf)
    return d, buf


def _unpack(h, d, buf):
    import torch
    out = torch.empty(d.n_sites * 72, dtype=torch.float64, device="cuda")
    h.unpack(su3.Desc(d.dtype, su3.FULL18, su3.AOS, d.n_sites, d.site_stride_bytes), buf, out)
    h.sync()
    return out.cpu().numpy()


def _vectors_to_f64(raw, dtype):
    if dtype == su3.F64:
        return raw.view(np.float64).astype(np.float64)
    if dtype == su3.F32:
        return raw.view(np.float32).astype(np.float64)
    if dtype == su3.F16:
        return raw.view(np.float16).astype(np.float64)
    return (raw.view(np.uint16).astype(np.uint32) << 16).view(np.float32).astype(np.float64)


@pytest.mark.parametrize("dtype", DTYPES, ids=IDS)
@pytest.mark.parametrize("op", [su3.OP_NA, su3.OP_AN], ids=["a_bdag", "adag_b"])
@pytest.mark.parametrize("V", SIZES)
def test_adjoint_products(h, dtype, op, V):
    a, b = gen.lattice(12, V)
    d, abuf = _packed(h, a, dtype)
    cbuf = empty_bytes(su3.array_bytes(d))
    h.mult_op(op, d, abuf, b, d, cbuf)
    got = _unpack(h, d, cbuf)
    ref = oracle.mult_na(a, b) if op == su3.OP_NA else oracle.mult_an(a, b)
    assert oracle.error(got, ref)[0] <= TOL[(dtype, su3.FULL18)]


@pytest.mark.parametrize("dtype", DTYPES, ids=IDS)
@pytest.mark.parametrize("adjoint", [False, True], ids=["a_v", "adag_v"])
@pytest.mark.parametrize("V", SIZES)
def test_mat_vec(h, dtype, adjoint, V):
    a, _ = gen.lattice(13, V)
    v = np.random.default_rng(V).standard_normal(24) / 2.0
    d, abuf = _packed(h, a, dtype)
    rb = {su3.F64: 8, su3.F32: 4, su3.F16: 2, su3.BF16: 2}[dtype]
    w = empty_bytes(V * 24 * rb + 4096, fill=0x33)
    h.mat_vec(d, abuf, v, w, adjoint=adjoint)
    h.sync()
    raw = w.cpu().numpy()
    assert np.all(raw[V * 24 * rb:] == 0x33)  # nothing written past the output
    got = _vectors_to_f64(raw[: V * 24 * rb], dtype)
    ref = oracle.mat_vec(a, v, adjoint=adjoint)
    assert oracle.error(got, ref)[0] <= TOL[(dtype, su3.FULL18)]


def test_adjacent_on_padded_sites_and_in_place(h):
    """The paper's 640-byte FP64 Site for a^dagger b and a v; a^dagger b in place."""
    V = 1500
    a, b = gen.lattice(14, V)
    a640 = np.zeros((V, 80))
    a640[:, :72] = a.reshape(V, 72)
    d = su3.Desc(su3.F64, su3.FULL18, su3.AOS, V, 640)
    abuf = to_dev(a640.reshape(-1))
    c = to_dev(np.full(V * 80, 5.5))
    h.mult_op(su3.OP_AN, d, abuf, b, d, c)
    v = np.linspace(-1, 1, 24)
    w = to_dev(np.zeros(V * 24))
    h.mat_vec(d, abuf, v, w)
    h.sync()
    cc = c.cpu().numpy().reshape(V, 80)
    assert np.all(cc[:, 72:] == 5.5)
    assert oracle.error(cc[:, :72].reshape(-1), oracle.mult_an(a, b))[0] <= 1e-13
    assert oracle.error(w.cpu().numpy(), oracle.mat_vec(a, v))[0] <= 1e-13
    # in place
    h.mult_op(su3.OP_AN, d, abuf, b, d, abuf)
    h.sync()
    assert oracle.error(abuf.cpu().numpy().reshape(V, 80)[:, :72].reshape(-1), oracle.mult_an(a, b))[0] <= 1e-13


def test_adjacent_rejects(h):
    V = 10
    d = su3.Desc(su3.F64, su3.FULL18, su3.SOA, V)
    buf = empty_bytes(su3.array_bytes(d))
    with pytest.raises(su3.Su3Error) as e:
        h.mult_op(su3.OP_AN, d, buf, np.zeros(72), d, buf)
    assert e.value.status == 2
    with pytest.raises(su3.Su3Error) as e:
        h.mult_op(7, d, buf, np.zeros(72), d, buf)
    assert e.value.status == 1
    da = su3.Desc(su3.F64, su3.FULL18, su3.AOS, V)
    with pytest.raises(su3.Su3Error) as e:
        h.mat_vec(da, buf, np.zeros(24), buf.data_ptr() + 16)  # overlapping output
    assert e.value.status == 1
    h.sync()


@pytest.mark.parametrize("V", SIZES)
def test_adjacent_in_fp32_pairs(h, V):
    """a b^dagger, a^dagger b, a v and a^dagger v with FP64 storage and FP32-pair arithmetic: within
    the FP64 tolerance of the oracle, also on padded 640-byte sites and in place (a^dagger b)."""
    a, b = gen.lattice(15, V)
    d = su3.Desc(su3.F64, su3.FULL18, su3.AOS, V, 0, su3.F32PAIR)
    abuf = to_dev(a)
    for op, ref in ((su3.OP_NA, oracle.mult_na(a, b)), (su3.OP_AN, oracle.mult_an(a, b))):
        cbuf = to_dev(np.zeros_like(a))
        h.mult_op(op, d, abuf, b, d, cbuf)
        h.sync()
        assert oracle.error(cbuf.cpu().numpy(), ref)[0] <= 1e-13, op
    v = np.random.default_rng(V + 1).standard_normal(24) / 2.0
    for adjoint in (False, True):
        w = empty_bytes(V * 24 * 8 + 4096, fill=0x33)
        h.mat_vec(d, abuf, v, w, adjoint=adjoint)
        h.sync()
        raw = w.cpu().numpy()
        assert np.all(raw[V * 24 * 8:] == 0x33)
        assert oracle.error(raw[: V * 24 * 8].view(np.float64), oracle.mat_vec(a, v, adjoint=adjoint))[0] <= 1e-13
    # padded sites, and a^dagger b in place
    a640 = np.zeros((V, 80))
    a640[:, :72] = a.reshape(V, 72)
    d640 = su3.Desc(su3.F64, su3.FULL18, su3.AOS, V, 640, su3.F32PAIR)
    buf = to_dev(a640.reshape(-1))
    h.mult_op(su3.OP_AN, d640, buf, b, d640, buf)
    h.sync()
    got = buf.cpu().numpy().reshape(V, 80)
    assert np.all(got[:, 72:] == 0.0)
    assert oracle.error(got[:, :72].reshape(-1), oracle.mult_an(a, b))[0] <= 1e-13


def test_adjacent_pairs_generic_magnitudes(h):
    """a^dagger b and a v in FP32 pairs on entries of mixed magnitude: within 2^-42 of the sum of
    |x||y| over each output's six real terms (the same relative bound as the product)."""
    rng = np.random.default_rng(16)
    V = 2000
    a = rng.standard_normal(V * 72) * np.exp(rng.uniform(-15, 15, V * 72))
    _, b = gen.lattice(16, V)
    d = su3.Desc(su3.F64, su3.FULL18, su3.AOS, V, 0, su3.F32PAIR)
    abuf = to_dev(a)
    c = to_dev(np.zeros_like(a))
    h.mult_op(su3.OP_AN, d, abuf, b, d, c)
    v = rng.standard_normal(24)
    w = to_dev(np.zeros(V * 24))
    h.mat_vec(d, abuf, v, w)
    h.sync()
    A = np.abs(a).reshape(V, 4, 3, 3, 2).sum(-1)
    B = np.abs(b).reshape(4, 3, 3, 2).sum(-1)
    bound_an = np.einsum("sjmk,jml->sjkl", A, B).repeat(2, axis=-1).reshape(-1)
    assert np.all(np.abs(c.cpu().numpy() - oracle.mult_an(a, b)) <= 2.0 ** -42 * bound_an + 1e-30)
    Vv = np.abs(v).reshape(4, 3, 2).sum(-1)
    bound_mv = np.einsum("sjkm,jm->sjk", A, Vv).repeat(2, axis=-1).reshape(-1)
    assert np.all(np.abs(w.cpu().numpy() - oracle.mat_vec(a, v)) <= 2.0 ** -42 * bound_mv + 1e-30)
