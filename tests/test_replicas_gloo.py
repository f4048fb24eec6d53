"""Host logic of the multi-GPU path (replicas, Sec. 7 of the design: pixels
and frames are independent, so ranks share no data), run as two gloo ranks on
the CPU: rendezvous, barrier, max-over-ranks timing, per-rank frame seeds and
the whole-job throughput; the reference arm runs on rank 0 only."""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    os.environ.update(RANK=str(rank), LOCAL_RANK=str(rank), WORLD_SIZE=str(world),
                      MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import bench
    import torch.distributed as dist
    try:
        w, r, _ = bench.dist_setup(world)
        assert dist.get_backend() == "gloo"
        bench.barrier(w)
        # rank r "took" 10 + r ms: every rank must see the slowest one's time
        mx = bench.allreduce_max(w, 10.0 + r)
        seeds = bench.rank_frame_seeds(r, 4)
        q.put((r, w, mx, seeds, bench.job_mpx_per_s(w, 512 * 512, 20, mx)))
    finally:
        dist.destroy_process_group()


def test_two_gloo_replicas():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
    codes = [p.exitcode for p in procs]
    for p in procs:
        if p.is_alive():
            p.kill()
    assert codes == [0, 0], codes
    got = sorted(q.get(timeout=5) for _ in range(world))
    assert [g[0] for g in got] == [0, 1] and all(g[1] == 2 for g in got)
    assert all(g[2] == 11.0 for g in got)  # the max over ranks, on every rank
    s0, s1 = set(got[0][3]), set(got[1][3])
    assert len(s0) == 4 and len(s1) == 4 and not (s0 & s1)  # disjoint frames per rank
    # two ranks' pixels over the slowest rank's 11 ms
    assert got[0][4] == pytest.approx(2 * 512 * 512 * 20 / 11e-3 / 1e6, rel=1e-12)
    assert got[0][4] == got[1][4]


def test_reference_arm_rank1_does_no_work(monkeypatch):
    """Under torchrun only rank 0 times the oracle; rank 1 returns at once."""
    sys.path.insert(0, ROOT)
    import bench
    calls = []
    monkeypatch.setitem(sys.modules, "oracle", type(sys)("oracle_stub"))
    monkeypatch.setattr("builtins.print", lambda *a, **k: calls.append(a))
    assert bench.run_reference(None, 2, 1) is None
    assert calls == []
