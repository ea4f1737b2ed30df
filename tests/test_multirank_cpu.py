"""The N > 1 path of bench.py on CPU: two gloo ranks (no GPU).

Each GPU of a multi-GPU run solves its own replica (weak scaling, no collective on the
data path); the only cross-rank steps are the barrier around the timed region and the
maximum of the ranks' times, from which the whole-job rate is computed.  Replicas draw
different seeded inputs per rank.
"""
import os
import socket

import pytest

torch = pytest.importorskip("torch")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, times, out):
    import torch.distributed as tdist
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    tdist.init_process_group("gloo", rank=rank, world_size=world)
    tdist.barrier()
    t = bench.max_over_ranks(times[rank], "cpu")
    w, _ = bench.inputs(rank)
    out[rank] = (t, bench.whole_job_rate(world, 5, t), float(w.p0_true.sum()))
    tdist.barrier()
    tdist.destroy_process_group()


def test_two_gloo_ranks_agree_on_the_slowest_time():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    times = [812.5, 1033.0]
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, times, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    t0, rate0, s0 = out[0]
    t1, rate1, s1 = out[1]
    assert t0 == t1 == max(times)
    assert rate0 == rate1 == pytest.approx(2 * 5 / (max(times) / 1000.0))
    assert s0 != s1          # each replica solves its own seeded problem


def test_reference_arm_runs_on_rank_zero_only(monkeypatch, capsys):
    import bench
    monkeypatch.setattr("sys.argv", ["bench.py", "--impl", "reference", "--gpus", "2"])
    args = bench.parse()
    bench.run_reference(args, 1)       # a non-zero rank exits without work or output
    assert capsys.readouterr().out == ""
