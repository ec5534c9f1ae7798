"""The multi-GPU harness of bench.py on CPU: world_size-2 gloo ranks (one process each,
127.0.0.1 rendezvous).  Streams are independent, so the path shards by stream with no
collective on the data path: each rank times its own frames and the whole-job value is the
frames of all ranks over the slowest rank's time."""
import os
import socket

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank_main(rank, world, port, q):
    import sys
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE=str(world), RANK=str(rank),
                      LOCAL_RANK=str(rank))
    import bench
    import torch.distributed as dist
    r, w, local = bench.dist_setup(backend="gloo")
    assert (r, w, local) == (rank, world, rank)
    # rank k "took" (k + 1) seconds for 10 frames: the slowest rank sets the job's time
    bench.barrier(w)
    v = bench.weak_scaling_value(10, float(rank + 1), w)
    m = bench.max_over_ranks(float(rank + 1), w)
    # each rank draws its own sequence (independent streams, no shared data)
    frames, _ = bench.make_frames(seed=rank, n=2, width=64, height=48)
    q.put((rank, v, m, float(frames[0].mean())))
    dist.destroy_process_group()


def test_two_gloo_ranks_weak_scaling():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(k, world, port, q)) for k in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    got = sorted(q.get() for _ in range(world))
    for rank, v, m, _ in got:
        assert m == 2.0                        # max over ranks of the timed region
        assert v == pytest.approx(2 * 10 / 2.0)  # all ranks' frames / the slowest time
    assert got[0][3] != got[1][3]              # the ranks' inputs differ (seeded by rank)
