"""The N > 1 replica path of bench.py on CPU: two gloo ranks get the same
seeds and disjoint targets of the same shape (weak scaling, no data exchange),
the job time is the maximum over ranks, and each rank's march of its own shard
(the oracle standing in for the GPU path) equals a single-process march of
those targets."""
import hashlib
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")


def _port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _digest(a):
    return hashlib.sha1(np.ascontiguousarray(a).tobytes()).hexdigest()


def _worker(rank, world, port, q, argv):
    import sys
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    args = bench.parse(argv)
    wl = bench.workload(args, rank)
    seeds = [_digest(g.seeds) for g in wl.groups]
    tgts = [_digest(g.targets) for g in wl.groups]
    shapes = [g.targets.shape for g in wl.groups]
    t = bench.max_over_ranks(1.5 + rank, dist, torch.device("cpu"))
    q.put((rank, seeds, tgts, shapes, t))
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("argv", [["--config", "2", "--ntargets", "8", "--T", "10"],
                                  ["--config", "3", "--ntargets", "6", "--T", "10"]])
def test_two_ranks_shard_targets_and_take_max_time(argv):
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q, argv)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (_, s0, t0, sh0, m0), (_, s1, t1, sh1, m1) = out
    assert s0 == s1                                   # same seeds on every rank
    assert all(a != b for a, b in zip(t0, t1))        # each rank its own targets
    assert sh0 == sh1                                 # of the same shape
    assert m0 == m1 == 2.5                            # the slowest rank's time


def _march_worker(rank, world, port, q, argv, steps):
    # each replica marches its own shard (the oracle stands in for the GPU
    # path on CPU) and reports its final target states; nothing is exchanged
    import sys
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    from oracle import oracle as O
    try:
        args = bench.parse(argv)
        wl = bench.workload(args, rank)
        g = wl.groups[0]
        _, mt, _ = O.march(g.H, g.W, wl.T, wl.g2, g.seeds, g.targets, g.target_seed, steps=steps,
                           tol_ref=wl.tol, m_ref=wl.m, m_seed=wl.m_seed, a=wl.a)
        q.put((rank, mt, None))
    except Exception as e:                          # report instead of leaving the parent waiting
        q.put((rank, None, repr(e)))
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_march_their_own_shards():
    # config 1 (28x28, 4 targets per rank), two timesteps: each rank's final
    # states are those of a single-process march of that rank's targets, and
    # the two shards are different systems
    import sys
    import torch.multiprocessing as mp
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    from oracle import oracle as O
    O.build()
    argv = ["--config", "1", "--T", "10"]
    steps = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _port()
    procs = [ctx.Process(target=_march_worker, args=(r, 2, port, q, argv, steps)) for r in range(2)]
    for p in procs:
        p.start()
    out = dict((r, (mt, err)) for r, mt, err in (q.get(timeout=120) for _ in procs))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert all(err is None for _, err in out.values()), out
    args = bench.parse(argv)
    for r in (0, 1):
        wl = bench.workload(args, r)
        g = wl.groups[0]
        _, mt, _ = O.march(g.H, g.W, wl.T, wl.g2, g.seeds, g.targets, g.target_seed, steps=steps,
                           tol_ref=wl.tol, m_ref=wl.m, m_seed=wl.m_seed, a=wl.a)
        assert np.array_equal(out[r][0], mt)
    assert not np.allclose(out[0][0], out[1][0])
