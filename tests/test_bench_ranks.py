"""Host logic of bench.py under several ranks, as gloo processes on the CPU.

Under torchrun every rank runs an independent replica (events are independent
and every random draw is keyed by the event index, so the path shards without a
data-path collective).  What the ranks share is host logic: the process group,
the max-over-ranks time, disjoint event indices per replica, the whole-job rate,
and the reference arm's rule that only rank 0 works and prints.  Two ranks
check each of these here.
"""
import io
import multiprocessing as mp
import os
import socket
import sys
from contextlib import redirect_stdout

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, ws, port, q):
    try:
        os.environ.update(RANK=str(rank), WORLD_SIZE=str(ws), LOCAL_RANK=str(rank),
                          MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), PDR_DIST_BACKEND="gloo")
        sys.path.insert(0, ROOT)
        import bench
        dist, r, w = bench._dist()
        assert (r, w) == (rank, ws)
        # slowest rank's time: rank k reports 10 + 7k ms
        got = bench.max_over_ranks(dist, 10.0 + 7.0 * rank)
        # replicas take disjoint event ranges
        n_ev = 1000
        base = bench.replica_event_base(rank, n_ev)
        bases = [None] * ws
        dist.all_gather_object(bases, (base, base + n_ev))
        # the reference arm: ranks other than 0 return without work or output
        out = io.StringIO()
        if rank != 0:
            with redirect_stdout(out):
                bench.main(["--impl", "reference", "--workload", "tiny", "--steps", "1", "--warmup", "0"])
        dist.barrier()
        dist.destroy_process_group()
        q.put((rank, got, bases, out.getvalue()))
    except BaseException as e:  # report to the parent instead of hanging it
        q.put((rank, "error", repr(e), ""))


def test_two_gloo_ranks():
    ws = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank_main, args=(r, ws, port, q)) for r in range(ws)]
    for p in procs:
        p.start()
    res = {}
    try:
        for _ in range(ws):
            rank, got, bases, printed = q.get(timeout=120)
            res[rank] = (got, bases, printed)
    finally:
        for p in procs:
            p.join(timeout=30)
            if p.is_alive():
                p.kill()
    for rank, (got, bases, printed) in res.items():
        assert got != "error", bases
        assert got == 10.0 + 7.0 * (ws - 1)  # every rank sees the max
        ranges = sorted(bases)
        assert all(a1 <= b0 for (_, a1), (b0, _) in zip(ranges, ranges[1:]))  # disjoint
        assert ranges[0][0] == 0
        if rank != 0:
            assert printed == ""
    assert all(p.exitcode == 0 for p in procs)


def test_job_rate_counts_all_ranks_over_slowest_time():
    sys.path.insert(0, ROOT)
    import bench
    # 2 ranks x 1e6 particles x 10 steps in 20 ms (the slowest rank) = 1e9 / s
    assert abs(bench.job_rate(1_000_000, 2, 10, 20.0) - 1.0e9) < 1e-3
    assert bench.max_over_ranks(None, 3.5) == 3.5
