"""CUDA path vs the CPU FP64 oracle, element by element, for every form the library computes.

Sizes span several tiles with ragged tails (tile = 32 sites for FP64 AoS, 64/128 for narrower
forms; the direct kernels stride over 256-thread CTAs), plus the degenerate single site."""
import numpy as np
import pytest

import oracle
import paper_2103_00571_gb300 as su3
import su3_inputs as gen
from gpu_helpers import run_form, tol

pytestmark = pytest.mark.gpu

SIZES = [1, 4096, 4096 + 13, 3 * 8 ** 3 + 5]
FORMS = [
    (su3.F64, su3.FULL18, su3.FULL18),
    (su3.F32, su3.FULL18, su3.FULL18),
    (su3.F16, su3.FULL18, su3.FULL18),
    (su3.BF16, su3.FULL18, su3.FULL18),
    (su3.F64, su3.TWOROW12, su3.TWOROW12),
    (su3.F32, su3.TWOROW12, su3.TWOROW12),
    (su3.F64, su3.TWOROW12, su3.FULL18),
    (su3.F32, su3.TWOROW12, su3.FULL18),
    (su3.F16, su3.TWOROW12, su3.TWOROW12),
    (su3.BF16, su3.TWOROW12, su3.FULL18),
]
LAYOUTS = [su3.AOS, su3.AOSOA32, su3.SOA]


@pytest.fixture(scope="module")
def h():
    return su3.Handle(0)


def _name(f):
    return "%s-%s-%s" % ({0: "f64", 1: "f32", 2: "f16", 3: "bf16"}[f[0]], f[1], f[2])


@pytest.mark.parametrize("layout", LAYOUTS, ids=["aos", "aosoa32", "soa"])
@pytest.mark.parametrize("form", FORMS, ids=[_name(f) for f in FORMS])
@pytest.mark.parametrize("V", SIZES)
def test_form_vs_oracle(h, form, layout, V):
    dtype, rin, rout = form
    a, b = gen.lattice(gen.DEFAULT_SEED, V)
    ref = oracle.mult(a, b)
    got = run_form(h, a, b, dtype, rin, rout, layout)
    mx, rms = oracle.error(got, ref)
    assert mx <= tol(dtype, rin, rout), (mx, rms)


@pytest.mark.parametrize("dtype", [su3.F64, su3.F32, su3.F16, su3.BF16])
def test_error_also_vs_dequantised_input(h, dtype):
    """Diagnostic split of the error: against the oracle run on the rounded (de-quantised) input the
    remaining error is the arithmetic and output rounding alone, and must be no larger."""
    V = 2000
    a, b = gen.lattice(5, V)
    got = run_form(h, a, b, dtype)
    if dtype == su3.F64:
        aq = a
    elif dtype == su3.F32:
        aq = oracle.round_float(a).astype(np.float64)
    elif dtype == su3.F16:
        aq = oracle.widen_half(oracle.round_half(a))
    else:
        aq = oracle.widen_bf16(oracle.round_bf16(a))
    e_orig, _ = oracle.error(got, oracle.mult(a, b))
    e_deq, _ = oracle.error(got, oracle.mult(aq, b))
    assert e_deq <= e_orig * 1.0001 + 1e-15


@pytest.mark.parametrize("dtype", [su3.F32, su3.F16, su3.BF16])
@pytest.mark.parametrize("layout", LAYOUTS, ids=["aos", "aosoa32", "soa"])
def test_pack_is_bit_exact(h, dtype, layout):
    """su3_pack rounds once from FP64 to nearest even: the same bits as the oracle's rounding."""
    import torch
    V = 777
    a, _ = gen.lattice(8, V)
    d = su3.Desc(dtype, su3.FULL18, layout, V)
    buf = torch.empty(su3.array_bytes(d), dtype=torch.uint8, device="cuda")
    h.pack(torch.from_numpy(a).cuda(), d, buf)
    back = torch.empty(V * 72, dtype=torch.float64, device="cuda")
    h.unpack(d, buf, back)
    h.sync()
    back = back.cpu().numpy()
    if dtype == su3.F32:
        want = oracle.round_float(a).astype(np.float64)
    elif dtype == su3.F16:
        want = oracle.widen_half(oracle.round_half(a))
    else:
        want = oracle.widen_bf16(oracle.round_bf16(a))
    assert np.array_equal(back, want)


@pytest.mark.parametrize("layout", LAYOUTS, ids=["aos", "aosoa32", "soa"])
def test_pack_unpack_roundtrip(h, layout):
    """FP64 FULL18 round trip is bitwise; FP64 TWOROW12 rebuilds row 2 within 1e-15 (SU(3) input)."""
    import torch
    V = 999
    a, _ = gen.lattice(9, V)
    for rep, tol_rt in ((su3.FULL18, 0.0), (su3.TWOROW12, 1e-15)):
        d = su3.Desc(su3.F64, rep, layout, V)
        buf = torch.empty(su3.array_bytes(d), dtype=torch.uint8, device="cuda")
        h.pack(torch.from_numpy(a).cuda(), d, buf)
        back = torch.empty(V * 72, dtype=torch.float64, device="cuda")
        h.unpack(d, buf, back)
        h.sync()
        err = np.max(np.abs(back.cpu().numpy() - a))
        assert err <= tol_rt, (rep, err)


@pytest.mark.parametrize("layout", LAYOUTS, ids=["aos", "aosoa32", "soa"])
@pytest.mark.parametrize("reps", [(su3.FULL18, su3.FULL18), (su3.TWOROW12, su3.TWOROW12), (su3.TWOROW12, su3.FULL18)],
                         ids=["full", "2row", "2row-to-full"])
@pytest.mark.parametrize("V", SIZES)
def test_f32pair_vs_oracle(h, layout, reps, V):
    """FP64 storage with FP32-pair arithmetic: within the FP64 tolerance of the oracle (two-row to
    full rebuilds row 2 of a in FP64 first)."""
    ri, ro = reps
    a, b = gen.lattice(gen.DEFAULT_SEED, V)
    ref = oracle.mult(a, b)
    got = run_form(h, a, b, su3.F64, ri, ro, layout, arith=su3.F32PAIR)
    mx, rms = oracle.error(got, ref)
    assert mx <= tol(su3.F64, ri, ro), (mx, rms)


def test_f32pair_generic_and_constant_inputs(h):
    """Non-SU(3) inputs of mixed magnitude (the relative bound scales with sum |a||b|) and the
    paper's constant case, whose exact zeros the split replaces by values below 2^-73."""
    rng = np.random.default_rng(4)
    V = 3000
    a = rng.standard_normal(V * 72) * np.exp(rng.uniform(-20, 20, V * 72))
    _, b = gen.lattice(4, V)
    got = run_form(h, a, b, su3.F64, arith=su3.F32PAIR)
    ref = oracle.mult(a, b)
    # sum over the six real terms of |x||y| <= sum_m (|re a|+|im a|)(|re b|+|im b|)
    A = np.abs(a).reshape(V, 4, 3, 3, 2).sum(-1)
    B = np.abs(b).reshape(4, 3, 3, 2).sum(-1)
    bound = np.einsum("sjkm,jml->sjkl", A, B).repeat(2, axis=-1).reshape(-1)
    assert np.all(np.abs(got - ref) <= 2.0 ** -42 * bound + 1e-30)
    ac, bc = gen.paper_constant(4096)
    got = run_form(h, ac, bc, su3.F64, arith=su3.F32PAIR).reshape(-1, 72)
    assert np.max(np.abs(got[:, 0::2] - 1.0)) <= 1e-15 and np.max(np.abs(got[:, 1::2])) <= 1e-20


@pytest.mark.parametrize("tpl", [1, 3])
def test_f32pair_tworow_to_full_rebuild(h, tpl):
    """Two-row in, full out, in FP32-pair arithmetic: row 2 of a is rebuilt as conj(row0 x row1)
    from the pair splits of rows 0 and 1. On SU(3) input: within the FP64 form's 1e-13 of the
    oracle. On rows of mixed magnitude (not SU(3)): against the oracle's FP64 expansion of the same
    two rows, rows 0-1 within the product's 2^-42 sum_m |a_km||b_ml| and row 2 within
    2^-40 sum_m S_m |b_ml|, S_m the moduli of the four products behind element m of row 2."""
    cfg = {"tile_sites": 32, "stages": 3, "block": 128, "threads_per_link": tpl}
    V = 3 * 8 ** 3 + 5
    a, b = gen.lattice(17, V)
    got = run_form(h, a, b, su3.F64, su3.TWOROW12, su3.FULL18, arith=su3.F32PAIR, cfg=cfg)
    assert oracle.error(got, oracle.mult(a, b))[0] <= 1e-13
    rng = np.random.default_rng(18)
    V = 2000
    a = rng.standard_normal(V * 72) * np.exp(rng.uniform(-10, 10, V * 72))
    a = oracle.tworow_expand(oracle.tworow_compress(a))  # row 2 = conj(row0 x row1) in FP64
    got = run_form(h, a, b, su3.F64, su3.TWOROW12, su3.FULL18, arith=su3.F32PAIR, cfg=cfg)
    ref = oracle.mult(a, b)
    A1 = np.abs(a).reshape(V, 4, 3, 3, 2).sum(-1)  # |re| + |im| of every element
    B1 = np.abs(b).reshape(4, 3, 3, 2).sum(-1)
    S = np.empty((V, 4, 3))
    for m in range(3):
        p, q = (m + 1) % 3, (m + 2) % 3
        S[:, :, m] = A1[:, :, 0, p] * A1[:, :, 1, q] + A1[:, :, 0, q] * A1[:, :, 1, p]
    bound = 2.0 ** -42 * np.einsum("sjkm,jml->sjkl", A1, B1)
    bound[:, :, 2, :] = 2.0 ** -40 * np.einsum("sjm,jml->sjl", S, B1)
    err = np.abs(got - ref).reshape(V, 4, 3, 3, 2)
    assert np.all(err <= bound[..., None] + 1e-30)


@pytest.mark.parametrize("layout", LAYOUTS, ids=["aos", "aosoa32", "soa"])
@pytest.mark.parametrize("rep", [su3.FULL18, su3.TWOROW12], ids=["full", "2row"])
def test_hybrid_is_native_or_pair_per_site(layout, rep):
    """HYBRID splits the lattice between FP64-pipe CTAs and FP32-pair CTAs: every site's result is
    bit for bit the NATIVE or the F32PAIR result, about the configured share is native, and the
    whole is within the FP64 tolerance of the oracle."""
    hh = su3.Handle(0)
    V = 9 * 8 ** 3 + 7
    a, b = gen.lattice(11, V)
    # 2 of 8 warps: every 4th warp-tile runs natively; AOS tiles of 64 sites keep all 8 warps busy
    cfg = {"native_permille": 250, "block": 256}
    if layout == su3.AOS:
        cfg.update(tile_sites=64, stages=3, ctas_per_sm=2)
    got = run_form(hh, a, b, su3.F64, rep, rep, layout, arith=su3.HYBRID, cfg=cfg).reshape(V, 72)
    nat = run_form(hh, a, b, su3.F64, rep, rep, layout, arith=su3.NATIVE).reshape(V, 72)
    pair = run_form(hh, a, b, su3.F64, rep, rep, layout, arith=su3.F32PAIR).reshape(V, 72)
    is_nat = np.all(got == nat, axis=1)
    is_pair = np.all(got == pair, axis=1)
    assert np.all(is_nat | is_pair)
    share = np.mean(is_nat & ~is_pair)
    assert 0.18 < share < 0.32, share
    mx, _ = oracle.error(got.reshape(-1), oracle.mult(a, b))
    assert mx <= tol(su3.F64, rep)
    hh.close()


@pytest.mark.parametrize("arith", [su3.NATIVE, su3.F32PAIR], ids=["native", "f32pair"])
@pytest.mark.parametrize("rep", [su3.FULL18, su3.TWOROW12], ids=["full", "2row-to-full"])
def test_total_cancellation_gives_identity(h, arith, rep):
    """a[i][j] = b[j]^dagger for every site: c = b^dagger b = I exactly. Each off-diagonal output is a
    sum of O(1) terms that cancels to zero and each diagonal output is exactly 1, the case in which
    a lost or doubly counted error term of the FP32-pair sums would show. Against the exact I,
    within the FP64 tolerance."""
    V = 777
    _, b = gen.lattice(61, V)
    bj = b.reshape(4, 3, 3, 2)
    bdag = np.empty_like(bj)
    bdag[..., 0] = np.transpose(bj[..., 0], (0, 2, 1))
    bdag[..., 1] = -np.transpose(bj[..., 1], (0, 2, 1))
    a = np.tile(bdag.reshape(-1), V)
    ident = np.zeros((4, 3, 3, 2))
    for k in range(3):
        ident[:, k, k, 0] = 1.0
    want = np.tile(ident.reshape(-1), V)
    assert oracle.error(oracle.mult(a, b), want)[0] <= 1e-14  # the oracle agrees: b is unitary
    got = run_form(h, a, b, su3.F64, rep, su3.FULL18, arith=arith)
    assert oracle.error(got, want)[0] <= 1e-13
