"""The seeded input generator: Philox known answers, SU(3)-ness, statistics, determinism."""
import json
import os
import subprocess
import sys

import numpy as np

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_philox_known_answers(gen):
    kat = json.load(open(os.path.join(GOLDEN, "philox4x32_10_kat.json")))
    for v in kat["vectors"]:
        ctr = [int(x, 16) for x in v["ctr"]]
        key = [int(x, 16) for x in v["key"]]
        out = [int(x, 16) for x in v["out"]]
        assert list(gen.philox4x32_10(ctr, key)) == out


def test_matrices_are_su3(gen, oracle_lib):
    m = gen.matrices(2103, 0, 0, 20000)
    u, d = oracle_lib.unitarity(m)
    assert u < 1e-14 and d < 1e-14


def test_normals_statistics(gen):
    z = np.concatenate([gen.normals(99, 0, i) for i in range(20000)])
    assert abs(z.mean()) < 0.02
    assert abs(z.var() - 1.0) < 0.02
    # fourth moment of N(0,1) is 3
    assert abs(np.mean(z ** 4) - 3.0) < 0.1


def test_sites_layout_and_b(gen):
    V = 10
    a = gen.sites(5, 0, V)
    m = gen.matrices(5, 0, 0, 4 * V)
    assert np.array_equal(a.reshape(V * 4, 18), m)
    b = gen.bmat(5, 0, V)
    assert np.array_equal(b.reshape(4, 18), gen.matrices(5, 0, 4 * V, 4))
    # chunked generation equals whole generation
    part = gen.sites(5, 0, V, first_site=3, count=4)
    assert np.array_equal(part, a[3 * 72: 7 * 72])
    at = gen.sites_at(5, 0, [7, 2])
    assert np.array_equal(at[0], a[7 * 72: 8 * 72]) and np.array_equal(at[1], a[2 * 72: 3 * 72])


def test_stride_leaves_pads(gen):
    out = np.full(3 * 80, -1.0)
    gen.sites(5, 0, 3, stride=80, out=out)
    out = out.reshape(3, 80)
    assert np.all(out[:, 72:] == -1.0)
    assert np.array_equal(out[:, :72].reshape(-1), gen.sites(5, 0, 3))


def test_lattices_differ(gen):
    a0 = gen.sites(5, 0, 4)
    a1 = gen.sites(5, 1, 4)
    a2 = gen.sites(6, 0, 4)
    assert not np.array_equal(a0, a1) and not np.array_equal(a0, a2)


def test_thread_count_invariance(gen):
    code = ("import sys; sys.path.insert(0, %r); import su3_inputs as g, hashlib;"
            "print(hashlib.sha256(g.sites(2103, 0, 4096).tobytes()).hexdigest())" % ROOT)
    outs = []
    for nt in ("1", "7"):
        env = dict(os.environ, OMP_NUM_THREADS=nt)
        outs.append(subprocess.run([sys.executable, "-c", code], env=env, check=True,
                                   capture_output=True, text=True).stdout.strip())
    assert outs[0] == outs[1]


def test_extents(gen):
    e = gen.extents(2103, 96)
    assert e.shape == (96, 4)
    assert set(np.unique(e)) <= set(range(4, 25, 2))
    assert len(set(np.unique(e))) == 11  # all values occur across 384 draws
    assert np.array_equal(e, gen.extents(2103, 96))


def test_paper_constant(gen):
    a, b = gen.paper_constant(3)
    a = a.reshape(3, 72)
    assert np.all(a[:, 0::2] == 1.0) and np.all(a[:, 1::2] == 0.0)
    assert np.all(b[0::2] == 1.0 / 3.0) and np.all(b[1::2] == 0.0)
