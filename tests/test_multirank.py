"""The N > 1 host logic of bench.py on CPU, with gloo ranks: replicas (each rank times its own
lattice) agree on the job time as the max over ranks, and slab shards (--shard: the ranks split
one lattice into contiguous slabs of sites) compute, together, exactly the single-rank result.
No data-path collective exists: sites are independent."""
import os
import socket

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    import sys
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    bench.barrier(world)
    t = bench.max_over_ranks(10.0 + rank * 5.0, world)
    # each rank's replica: its own lattice id (= rank), independent inputs
    import su3_inputs as gen
    a = gen.sites(bench.SEED, rank, 16, count=2)
    q.put((rank, t, float(a[0])))
    dist.destroy_process_group()


@pytest.mark.timeout(120)
def test_two_rank_max_and_replicas():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=90) for _ in procs)
    for p in procs:
        p.join(30)
        assert p.exitcode == 0
    assert [r[1] for r in res] == [15.0, 15.0]
    assert res[0][2] != res[1][2]  # different replica inputs per rank


@pytest.mark.timeout(240)
def test_reference_arm_under_torchrun_prints_once():
    """`torchrun --nproc-per-node 2 bench.py --impl reference`: the launch the driver uses for N > 1.
    Rank 0 alone times the oracle and prints the one JSON line; the other rank exits 0 without
    work (gloo rendezvous on 127.0.0.1, CPU only)."""
    import json
    import subprocess
    import sys
    port = _free_port()
    out = subprocess.run([sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
                          "--master-addr", "127.0.0.1", "--master-port", str(port),
                          os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2", "--L", "8",
                          "--steps", "2", "--warmup", "1"],
                         capture_output=True, text=True, timeout=200, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1, out.stdout
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["value"] > 0 and d["n_gpus"] == 2  # the launch's N


def test_slab_partition_covers_lattice():
    import bench
    for n in (0, 1, 7, 4096, 16777216, 1000003):
        for world in (1, 2, 3, 4, 8):
            spans = [bench.slab(n, world, r) for r in range(world)]
            assert spans[0][0] == 0 and sum(c for _, c in spans) == n
            for (f0, c0), (f1, _) in zip(spans, spans[1:]):
                assert f0 + c0 == f1  # contiguous, disjoint, in rank order
            assert max(c for _, c in spans) - min(c for _, c in spans) <= 1


def _slab_worker(rank, world, port, q):
    import sys
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    import oracle
    import su3_inputs as gen
    V = 6 ** 4 + 3  # ragged: the slabs differ by one site
    first, count = bench.slab(V, world, rank)
    a = gen.sites(bench.SEED, 0, V, first_site=first, count=count)  # this rank's sites only
    b = gen.bmat(bench.SEED, 0, V)  # the one lattice's b, the same on every rank
    c = oracle.mult(a, b)
    bench.barrier(world)
    q.put((rank, first, c.tobytes()))
    dist.destroy_process_group()


@pytest.mark.timeout(120)
def test_two_rank_slabs_equal_single_rank():
    """Two gloo ranks each compute their slab of one lattice (inputs generated for their own sites
    only); the slabs' outputs, concatenated in rank order, equal the one-rank output bit for bit."""
    import numpy as np
    import sys
    sys.path.insert(0, ROOT)
    import bench
    import oracle
    import su3_inputs as gen
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_slab_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=90) for _ in procs)
    for p in procs:
        p.join(30)
        assert p.exitcode == 0
    V = 6 ** 4 + 3
    whole = oracle.mult(gen.sites(bench.SEED, 0, V), gen.bmat(bench.SEED, 0, V))
    joined = np.concatenate([np.frombuffer(c, dtype=np.float64) for _, _, c in res])
    assert [f for _, f, _ in res] == [0, bench.slab(V, 2, 1)[0]]
    assert np.array_equal(joined, whole)
