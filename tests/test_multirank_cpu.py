"""The N > 1 path of the benchmark on CPU: two gloo ranks shard the global batch into disjoint consecutive
pieces that cover it, take the slowest rank's time by an all-reduce MAX, and report the whole job's units
over that time; the reference arm under several ranks runs on rank 0 only.  No GPU and no solver involved:
this is the host logic around the per-rank solves."""
import os
import socket
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as tmp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import bench
    import inputs
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        B = 5
        mine = bench.shard(inputs.mu_batch(B * world), rank, world)
        seconds = 1.0 + 0.5 * rank                      # a slower rank 1
        t = bench.max_over_ranks(seconds, dist, torch.device("cpu"))
        value = bench.job_throughput(B, world, 3, t)
        dist.barrier()
        q.put((rank, mine, t, value))
    finally:
        dist.destroy_process_group()


def test_two_rank_sharding_and_timing():
    world, port = 2, _free_port()
    ctx = tmp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    import inputs
    full = inputs.mu_batch(10)
    assert np.array_equal(np.concatenate([o[1] for o in out]), full)      # disjoint, consecutive, covering
    for rank, mine, t, value in out:
        assert mine.shape == (5, 2)
        assert t == 1.5                                                   # the slowest rank's time
        assert value == pytest.approx(5 * 2 * 3 / 1.5)                    # whole-job units / that time


def _reference_rank(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import io
    import contextlib
    import bench
    called = []
    bench.reference_sample = lambda *a, **k: called.append(1) or ([1.0], [1.0], dict(
        value=1.0, unit="solves/s", cores=1, kind="oracle", sample="stub"))
    buf = io.StringIO()
    with contextlib.redirect_stdout(buf):
        bench.run_reference(type("A", (), dict(config="c1", steps=1, warmup=0, gpus=world))())
    q.put((rank, len(called), buf.getvalue()))


def test_reference_arm_runs_on_rank_zero_only():
    world, port = 2, _free_port()
    ctx = tmp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_reference_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, n0, text0), (r1, n1, text1) = out
    assert n0 == 1 and '"impl": "reference"' in text0
    assert n1 == 0 and text1 == ""
