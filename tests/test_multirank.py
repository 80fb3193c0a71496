"""The multi-GPU path of bench.py is replicas only: every rank solves its own problems and the ranks
exchange two numbers after the timed region (the slowest rank's seconds, the sum of the units processed).
These tests run that exchange on two CPU processes with the gloo backend (no GPU)."""
import os
import socket
import sys


ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    secs, units = bench.replica_totals(1.5 + rank, 100.0 * (rank + 1), "cpu")
    sizes, ppws, orders = bench.problem_table(8, rank)
    dist.barrier()
    q.put((rank, secs, units, sizes.tolist(), [round(v, 6) for v in ppws.tolist()]))
    dist.destroy_process_group()


def test_replica_totals_over_two_gloo_ranks():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = {}
    for _ in range(2):
        r, secs, units, sizes, ppws = q.get(timeout=120)
        out[r] = (secs, units, sizes, ppws)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r in range(2):
        assert out[r][0] == 2.5            # the slowest rank's time
        assert out[r][1] == 300.0          # units of both ranks
    assert out[0][3] != out[1][3]          # ranks draw different problems
    assert all(s in (48, 64, 96, 128, 160) for s in out[0][2] + out[1][2])


def test_replica_totals_single_process_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.replica_totals(0.25, 1234.0, "cpu") == (0.25, 1234.0)
    s0 = bench.problem_table(64, 0)[0]
    assert len(s0) == 64 and (bench.problem_table(64, 0)[0] == s0).all()   # seeded
