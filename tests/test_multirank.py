"""Host-side multi-rank logic of bench.py on CPU with the gloo backend (world size 2).

The method's units (channels, whole problems) are independent, so N GPUs run N replicas with
no collective on the data path; the ranks meet only at a barrier around the timed region and
for the maximum of their step times. Those two collectives are what this test exercises."""
import os
import socket

import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    os.environ.update({"RANK": str(rank), "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank),
                       "MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port)})
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    r, w = bench.dist_init()
    assert (r, w) == (rank, world)
    bench.barrier(w)
    t = bench.allreduce_max(1.0 + rank, w)  # each rank's step time; the job's time is the max
    # weak scaling: every rank builds its own independent problem of the same size
    prob = bench.make_problem("c1", seed_offset=rank)
    fp = float(sum(abs(p.uvw.astype("float64")).sum() for p in prob.pairs))
    # the reference arm runs on rank 0 alone; the other ranks return without work
    ref = bench.run_reference(None, rank, w) if rank != 0 else None
    q.put((rank, t, prob.total_vis, fp, ref))
    import torch.distributed as dist
    dist.destroy_process_group()


def test_two_gloo_ranks_barrier_and_max_time():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    out = sorted((q.get(timeout=10) for _ in range(2)), key=lambda o: o[0])
    assert [o[1] for o in out] == [2.0, 2.0]
    assert out[0][2] == out[1][2] == 8190       # same units per rank
    assert out[0][3] != out[1][3]               # but different (independently seeded) problems
    assert out[1][4] is None
