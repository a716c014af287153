"""Multi-rank host logic of bench.py on CPU: two gloo ranks.

Each rank runs an independent replica (its own seed); the job's time is the
maximum over ranks and its throughput counts the units of every rank.  No
collective touches the data path, so the reduction of timings is the only
exchange to check.
"""
import os
import socket

import pytest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _inputs():
    """The input generators, loaded by path (no native library needed)."""
    import importlib.util
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    spec = importlib.util.spec_from_file_location("kmc_inputs", os.path.join(root, "paper_1210_8084_gb300", "inputs.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import torch.distributed as dist
    import bench
    inputs = _inputs()
    r, w, local = bench.dist_env()
    dist.init_process_group("gloo", rank=r, world_size=w)
    try:
        times = bench.max_over_ranks([1.0 + r, 10.0 - r, 0.5 * r], w, "cpu")
        wl = dict(inputs.WORKLOADS["sod1d_fp64_200k"])
        pos, vel = inputs.make_state(wl, n=1000, seed=bench.replica_seed(wl["seed"], r))
        out[r] = dict(rank=r, world=w, local=local, times=times, first=float(pos[0, 0]),
                      rate=bench.job_rate(1000, w, 5, times[0]))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_reduce_timings_and_keep_replicas_independent():
    mp = pytest.importorskip("torch.multiprocessing")
    ctx = mp.get_context("spawn")
    port = _free_port()
    with ctx.Manager() as m:
        out = m.dict()
        procs = [ctx.Process(target=_rank_main, args=(r, 2, port, out)) for r in range(2)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(120)
        assert all(p.exitcode == 0 for p in procs), [p.exitcode for p in procs]
        res = [dict(out[r]) for r in range(2)]
    for r in range(2):
        assert res[r]["rank"] == r and res[r]["world"] == 2 and res[r]["local"] == r
        assert res[r]["times"] == [2.0, 10.0, 0.5]          # maximum over ranks, elementwise
        assert res[r]["rate"] == pytest.approx(1000 * 2 * 5 / 2.0)
    assert res[0]["first"] != res[1]["first"]               # replicas draw different states


def test_single_rank_is_identity():
    import bench
    assert bench.max_over_ranks([3.0, 4.0], 1, "cpu") == [3.0, 4.0]
    assert bench.replica_seed(7, 0) == 7
    assert bench.job_rate(10, 1, 2, 4.0) == 5.0
