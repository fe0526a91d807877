"""Pins of the CPU oracle to facts fixed by the paper and by mathematics (not by the oracle itself).

Each pin is chosen so that a plausible slip in the oracle (a transposed or swapped operand, a sign,
a dropped term, a wrong link index) fails at least one of them.
"""
import json
import os
from fractions import Fraction

import numpy as np
import pytest

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _cplx(x18):
    """[..., 18] interleaved doubles -> complex [..., 3, 3]."""
    x = np.asarray(x18).reshape(-1, 18)
    return (x[:, 0::2] + 1j * x[:, 1::2]).reshape(-1, 3, 3)


def _real18(z):
    z = np.asarray(z).reshape(-1, 9)
    out = np.empty((z.shape[0], 18))
    out[:, 0::2] = z.real
    out[:, 1::2] = z.imag
    return out


@pytest.mark.parametrize("L", [1, 2])
def test_matches_numpy_einsum(oracle_lib, gen, L):
    """Brute force on tiny lattices against numpy.einsum over complex128 (a library contraction):
    c[s, j, k, l] = sum_m a[s, j, k, m] b[j, m, l]."""
    V = L ** 4
    a, b = gen.lattice(7, V)
    c = oracle_lib.mult(a, b)
    A = _cplx(a).reshape(V, 4, 3, 3)
    B = _cplx(b).reshape(4, 3, 3)
    ref = np.einsum("sjkm,jml->sjkl", A, B)
    got = _cplx(c).reshape(V, 4, 3, 3)
    assert np.max(np.abs(got - ref)) < 1e-15


def test_identity_b_gives_a_bitwise(oracle_lib, gen):
    """b = I for every direction: c == a bit for bit (each output is x*1 plus exact zeros)."""
    a, _ = gen.lattice(11, 81)
    eye = _real18(np.eye(3, dtype=complex)[None].repeat(4, 0)).reshape(72)
    c = oracle_lib.mult(a, eye)
    assert np.array_equal(c.view(np.uint64), a.view(np.uint64))


def test_paper_constant_initialisation(oracle_lib):
    """The paper's own initialisation: a = 1+0i everywhere, b = 1/3+0i everywhere => c = 1+0i."""
    g = json.load(open(os.path.join(GOLDEN, "paper_numbers.json")))["constant_init"]
    V = 4 ** 4
    a = np.zeros((V, 72))
    a[:, 0::2] = g["a_element"][0]
    a[:, 1::2] = g["a_element"][1]
    b = np.zeros(72)
    b[0::2] = g["b_element"][0]
    b[1::2] = g["b_element"][1]
    c = oracle_lib.mult(a.reshape(-1), b).reshape(V, 72)
    assert np.max(np.abs(c[:, 0::2] - g["c_element"][0])) <= 1e-15
    assert np.max(np.abs(c[:, 1::2] - g["c_element"][1])) <= 1e-15


def test_rotation_closed_form(oracle_lib):
    """Real rotations in the (0,1) plane: R(t) R(p) = R(t + p). A transposed b gives R(t - p)."""
    def rot(t):
        m = np.eye(3, dtype=complex)
        m[0, 0], m[0, 1], m[1, 0], m[1, 1] = np.cos(t), -np.sin(t), np.sin(t), np.cos(t)
        return m
    ts = [0.3, 1.1, -0.7, 2.9]
    ps = [0.5, -1.3, 0.25, 0.9]
    a = _real18(np.stack([rot(t) for t in ts])).reshape(72)
    b = _real18(np.stack([rot(p) for p in ps])).reshape(72)
    c = _cplx(oracle_lib.mult(a, b))
    for j in range(4):
        assert np.max(np.abs(c[j] - rot(ts[j] + ps[j]))) < 1e-15


def test_order_closed_form(oracle_lib):
    """a = cyclic permutation P, b = diag(d): (a b)[k][l] = P[k][l] d[l], whereas the swapped
    product b a would give d[k] P[k][l]. Pins the operand order and the per-link b index."""
    P = np.zeros((3, 3), dtype=complex)
    P[0, 1] = P[1, 2] = P[2, 0] = 1.0
    ds = [np.exp(1j * np.array([0.1, 0.7, -0.8]) * (j + 1)) for j in range(4)]
    a = _real18(np.stack([P] * 4)).reshape(72)
    b = _real18(np.stack([np.diag(d) for d in ds])).reshape(72)
    c = _cplx(oracle_lib.mult(a, b))
    for j in range(4):
        want = P * ds[j][None, :]
        assert np.max(np.abs(c[j] - want)) < 1e-15
        assert np.max(np.abs(c[j] - ds[j][:, None] * P)) > 0.1


def test_linearity_in_a(oracle_lib, gen):
    """c(x a1 + y a2) = x c(a1) + y c(a2) for generic (non-SU(3)) a, within rounding."""
    rng = np.random.default_rng(5)
    V = 50
    a1 = rng.standard_normal(V * 72)
    a2 = rng.standard_normal(V * 72)
    _, b = gen.lattice(3, V)
    x, y = 0.37, -2.5
    lhs = oracle_lib.mult(x * a1 + y * a2, b)
    rhs = x * oracle_lib.mult(a1, b) + y * oracle_lib.mult(a2, b)
    assert np.max(np.abs(lhs - rhs)) < 1e-13


def test_associativity(oracle_lib, gen):
    """(a b1) b2 = a (b1 b2), with b1 b2 formed by numpy's complex matmul."""
    V = 30
    a, b1 = gen.lattice(21, V)
    b2 = gen.bmat(22, 0, V)
    B12 = np.matmul(_cplx(b1), _cplx(b2))
    lhs = oracle_lib.mult(oracle_lib.mult(a, b1), b2)
    rhs = oracle_lib.mult(a, _real18(B12).reshape(72))
    assert np.max(np.abs(lhs - rhs)) < 1e-14


def test_sites_are_independent(oracle_lib, gen):
    """Permuting the sites permutes the output bit for bit (no site reads another site)."""
    V = 64
    a, b = gen.lattice(9, V)
    perm = np.random.default_rng(1).permutation(V)
    c = oracle_lib.mult(a, b).reshape(V, 72)
    cp = oracle_lib.mult(a.reshape(V, 72)[perm].reshape(-1), b).reshape(V, 72)
    assert np.array_equal(cp, c[perm])


def test_stride_640_leaves_tail_alone(oracle_lib, gen):
    """The paper's padded 640-byte FP64 site (80 doubles): links at offset 0, tail never written;
    the link products equal the packed-site products."""
    V = 40
    a72, b = gen.lattice(13, V)
    a80 = np.full((V, 80), 7.5)
    a80[:, :72] = a72.reshape(V, 72)
    c80 = oracle_lib.mult(a80.reshape(-1), b, site_stride=80).reshape(V, 80)
    c72 = oracle_lib.mult(a72, b).reshape(V, 72)
    assert np.array_equal(c80[:, :72], c72)
    assert np.all(c80[:, 72:] == 0.0)


def test_su3_closure(oracle_lib, gen):
    """The product of SU(3) matrices is SU(3): unitarity and det = 1 within 1e-12."""
    a, b = gen.lattice(2103, 1024)
    c = oracle_lib.mult(a, b)
    u, d = oracle_lib.unitarity(c.reshape(-1, 18))
    assert u < 1e-12 and d < 1e-12


def test_unitarity_check_detects_violations(oracle_lib):
    """The unitarity/det checker itself: exact values on hand-made matrices."""
    eye = _real18(np.eye(3, dtype=complex)[None]).reshape(18)
    assert oracle_lib.unitarity(eye) == (0.0, 0.0)
    m = np.eye(3, dtype=complex) * 2.0  # M M^+ = 4 I, det = 8
    u, d = oracle_lib.unitarity(_real18(m[None]).reshape(18))
    assert u == pytest.approx(3.0) and d == pytest.approx(7.0)
    ph = np.diag(np.exp(1j * np.array([0.4, 0.4, 0.4])))  # unitary, det = e^{1.2 i}
    u, d = oracle_lib.unitarity(_real18(ph[None]).reshape(18))
    assert u < 1e-15 and d == pytest.approx(abs(np.exp(1.2j) - 1.0), abs=1e-15)


def _random_su3_expm(rng, n):
    """SU(3) from a library route independent of the generator: expm(i H), H Hermitian traceless."""
    from scipy.linalg import expm
    out = []
    for _ in range(n):
        X = rng.standard_normal((3, 3)) + 1j * rng.standard_normal((3, 3))
        H = (X + X.conj().T) / 2
        H -= np.trace(H) / 3 * np.eye(3)
        out.append(expm(1j * H))
    return np.stack(out)


def test_tworow_expand_rebuilds_su3(oracle_lib):
    """Row 2 of any SU(3) matrix equals conj(row0 x row1): checked on matrices built by scipy's
    matrix exponential, so neither the generator nor the oracle's formula is its own witness."""
    rng = np.random.default_rng(17)
    U = _random_su3_expm(rng, 200)
    full = _real18(U)
    back = oracle_lib.tworow_expand(oracle_lib.tworow_compress(full))
    assert np.max(np.abs(back - full)) < 1e-14
    # a plain (not special) unitary matrix, det = e^{i phi} != 1, does NOT round-trip
    V = U[0] * np.exp(0.3j)
    bad = oracle_lib.tworow_expand(oracle_lib.tworow_compress(_real18(V[None])))
    assert np.max(np.abs(bad - _real18(V[None]))) > 1e-2


def _all_values(kind):
    pats = np.arange(65536, dtype=np.uint32)
    if kind == "half":
        vals = pats.astype(np.uint16).view(np.float16).astype(np.float64)
    else:
        vals = (pats << 16).view(np.float32).astype(np.float64)
    ok = np.isfinite(vals)
    return pats[ok].astype(np.uint16), vals[ok]


def _nearest_even(x, pats, vals):
    """Brute force: among all finite patterns, the nearest value to x by exact rational distance,
    ties to the pattern with an even last bit."""
    best = None
    fx = Fraction(x)
    same_sign = (pats >> 15) == (1 if x < 0 else 0)  # a zero result keeps the sign of x
    cand = np.nonzero(same_sign)[0]
    order = cand[np.argsort(np.abs(vals[cand] - x))[:4]]
    for i in order:
        d = abs(Fraction(float(vals[i])) - fx)
        key = (d, int(pats[i]) & 1)
        if best is None or key < best[0]:
            best = (key, int(pats[i]))
    return best[1]


@pytest.mark.parametrize("kind", ["half", "bf16"])
def test_rounding_brute_force(oracle_lib, kind):
    """FP64 -> binary16 / bfloat16 round to nearest even, against brute force over every finite
    pattern (including ties, subnormals and signed values)."""
    pats, vals = _all_values(kind)
    pos = vals > 0
    rng = np.random.default_rng(3)
    xs = list(rng.standard_normal(300))
    xs += list(rng.uniform(-1, 1, 300) * 1e-6)
    # exact ties between neighbours, and neighbours of ties
    pv = np.sort(vals[pos])
    idx = rng.integers(0, pv.size - 1, 200)
    mids = (pv[idx] + pv[idx + 1]) / 2
    xs += list(mids) + list(np.nextafter(mids, 0)) + list(np.nextafter(mids, 1e9))
    xs = [x for x in xs if x != 0.0 and abs(x) < pv[-1]]
    fn = oracle_lib.round_half if kind == "half" else oracle_lib.round_bf16
    got = fn(np.array(xs))
    for x, g in zip(xs, got):
        assert int(g) == _nearest_even(x, pats, vals), (x, hex(int(g)))


def test_round_half_matches_numpy(oracle_lib):
    """numpy's float64 -> float16 conversion is a direct round-to-nearest-even: same bits."""
    rng = np.random.default_rng(8)
    x = np.concatenate([rng.standard_normal(20000), rng.standard_normal(2000) * 1e-5,
                        rng.standard_normal(200) * 7e4, [0.0, -0.0, 65504.0, 65519.99, 65520.0]])
    assert np.array_equal(oracle_lib.round_half(x), x.astype(np.float16).view(np.uint16))


def test_widen_is_exact(oracle_lib):
    pats, vals = _all_values("half")
    assert np.array_equal(oracle_lib.widen_half(pats), vals)
    pats, vals = _all_values("bf16")
    assert np.array_equal(oracle_lib.widen_bf16(pats), vals)


def test_round_float_is_c_cast(oracle_lib):
    x = np.random.default_rng(2).standard_normal(1000)
    assert np.array_equal(oracle_lib.round_float(x), x.astype(np.float32))


def test_error_metric(oracle_lib):
    x = np.array([1.0, 2.0, 3.0, 4.0])
    r = np.array([1.0, 2.5, 3.0, 3.0])
    mx, rms = oracle_lib.error(x, r)
    assert mx == 1.0 and rms == pytest.approx(np.sqrt((0.25 + 1.0) / 4))
    mx, _ = oracle_lib.error(np.array([np.nan]), np.array([0.0]))
    assert mx == np.inf


MUTANTS = [
    ("sign of the a_im*b_im term", "re = re - ai * bi;", "re = re + ai * bi;"),
    ("b transposed", "double br = B[6 * m + 2 * l], bi = B[6 * m + 2 * l + 1];",
     "double br = B[6 * l + 2 * m], bi = B[6 * l + 2 * m + 1];"),
    ("a transposed", "double ar = A[6 * k + 2 * m], ai = A[6 * k + 2 * m + 1];",
     "double ar = A[6 * m + 2 * k], ai = A[6 * m + 2 * k + 1];"),
    ("wrong link of b", "const double* B = b + 18 * j;", "const double* B = b + 18 * ((j + 1) % 4);"),
    ("dropped term", "im = im + ai * br;", "im = im + 0.0 * br;"),
    ("conjugated b", "re = re + ar * br;\n            re = re - ai * bi;\n            im = im + ar * bi;",
     "re = re + ar * br;\n            re = re + ai * bi;\n            im = im - ar * bi;"),
]


@pytest.mark.parametrize("name,old,new", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_pins_catch_planted_mistakes(tmp_path, gen, name, old, new):
    """Plant a plausible mistake in a copy of the oracle (on the CPU) and check that the pins
    above reject it: the einsum brute force and the order closed form."""
    import ctypes
    import subprocess
    import oracle as O
    src = open(O._SRC).read()
    assert old in src, name
    mpath = tmp_path / "mutant.c"
    mpath.write_text(src.replace(old, new))
    so = tmp_path / "mutant.so"
    subprocess.run(["gcc", "-O1", "-fopenmp", "-ffp-contract=off", "-fPIC", "-shared",
                    str(mpath), "-o", str(so), "-lm"], check=True)
    L = ctypes.CDLL(str(so))
    L.su3o_mult.argtypes = [ctypes.c_int64, ctypes.c_int64] + [ctypes.c_void_p] * 3
    V = 16
    a, b = gen.lattice(7, V)
    c = np.zeros_like(a)
    L.su3o_mult(V, 72, a.ctypes.data, b.ctypes.data, c.ctypes.data)
    ref = np.einsum("sjkm,jml->sjkl", _cplx(a).reshape(V, 4, 3, 3), _cplx(b).reshape(4, 3, 3))
    assert np.max(np.abs(_cplx(c).reshape(V, 4, 3, 3) - ref)) > 1e-3, name


def test_adjoint_products_match_einsum(oracle_lib, gen):
    """a^dagger b and a b^dagger against numpy einsum with explicit conjugates/transposes."""
    V = 16
    a, b = gen.lattice(3, V)
    A = _cplx(a).reshape(V, 4, 3, 3)
    B = _cplx(b).reshape(4, 3, 3)
    an = np.einsum("sjmk,jml->sjkl", A.conj(), B)
    na = np.einsum("sjkm,jlm->sjkl", A, B.conj())
    assert np.max(np.abs(_cplx(oracle_lib.mult_an(a, b)).reshape(V, 4, 3, 3) - an)) < 1e-15
    assert np.max(np.abs(_cplx(oracle_lib.mult_na(a, b)).reshape(V, 4, 3, 3) - na)) < 1e-15


def test_adjoint_products_of_a_matrix_with_itself_give_identity(oracle_lib, gen):
    """For SU(3) U: U^dagger U = U U^dagger = I (every link of a set to its direction's b)."""
    _, b = gen.lattice(8, 1)
    a = np.tile(b, 5)  # 5 sites, link j = b[j]
    eye = _real18(np.eye(3, dtype=complex)[None].repeat(20, 0)).reshape(-1)
    assert np.max(np.abs(oracle_lib.mult_an(a, b) - eye)) < 1e-14
    assert np.max(np.abs(oracle_lib.mult_na(a, b) - eye)) < 1e-14
    # and the two differ for a generic a (catches a swapped conjugation)
    a2, _ = gen.lattice(9, 5)
    assert np.max(np.abs(oracle_lib.mult_an(a2, b) - oracle_lib.mult_na(a2, b))) > 0.1


def test_mat_vec_matches_einsum_and_closed_forms(oracle_lib, gen):
    V = 16
    a, _ = gen.lattice(4, V)
    rng = np.random.default_rng(6)
    v = rng.standard_normal(24)
    A = _cplx(a).reshape(V, 4, 3, 3)
    X = (v[0::2] + 1j * v[1::2]).reshape(4, 3)
    w = oracle_lib.mat_vec(a, v)
    wa = oracle_lib.mat_vec(a, v, adjoint=True)
    W = (w[0::2] + 1j * w[1::2]).reshape(V, 4, 3)
    WA = (wa[0::2] + 1j * wa[1::2]).reshape(V, 4, 3)
    assert np.max(np.abs(W - np.einsum("sjkm,jm->sjk", A, X))) < 1e-15
    assert np.max(np.abs(WA - np.einsum("sjmk,jm->sjk", A.conj(), X))) < 1e-15
    # closed forms: identity links return v; U^dagger applied to U's column k gives e_k
    eye = _real18(np.eye(3, dtype=complex)[None].repeat(4, 0)).reshape(72)
    assert np.array_equal(oracle_lib.mat_vec(eye, v), v)
    U = A[0]  # 4 SU(3) matrices
    col = np.stack([U[j][:, j % 3] for j in range(4)])
    vv = np.empty(24)
    vv[0::2] = col.real.reshape(-1)
    vv[1::2] = col.imag.reshape(-1)
    got = oracle_lib.mat_vec(a[:72], vv, adjoint=True)
    G = (got[0::2] + 1j * got[1::2]).reshape(4, 3)
    for j in range(4):
        assert np.max(np.abs(G[j] - np.eye(3)[j % 3])) < 1e-15
