"""Multi-process host logic on CPU ranks (torch.distributed, gloo,
world_size 2): the benchmark's max-over-ranks timing and whole-job value, and
the one exchange a measurement-sharded image needs -- the weighted sum of
partial images -- checked against the FP64 oracle's image of all
measurements."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _init(rank, world, port):
    import sys
    if ROOT not in sys.path:
        sys.path.insert(0, ROOT)
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)


def _bench_worker(rank, world, port, out):
    _init(rank, world, port)
    import bench
    ms, value = bench.aggregate(10.0 * (rank + 1), 1000, 5, world, torch.device("cpu"))
    out[rank] = (ms, value)
    dist.destroy_process_group()


def _sharded_worker(rank, world, port, out):
    _init(rank, world, port)
    import oracle
    import synth
    from paper_2504_00959_gb300.sharded import combine_images
    prob = synth.to_numpy(synth.disk_problem(64, 4, 3000, synth.KERNEL_KB, 7, 4.0, 60.0, 91, weights="random"))
    q = prob["params"]
    m = prob["u"].shape[0]
    sl = slice(rank * m // world, (rank + 1) * m // world)
    img, sw, _ = oracle.dirty_image(q, prob["u"][sl], prob["v"][sl], prob["w"][sl], prob["wt"][sl],
                                    prob["vis"][sl], flags=synth.FLAG_CORRECT)
    full = combine_images(torch.from_numpy(img), sw)
    if rank == 0:
        ref, _, _ = oracle.dirty_image(q, prob["u"], prob["v"], prob["w"], prob["wt"], prob["vis"],
                                       flags=synth.FLAG_CORRECT)
        out[0] = float(np.max(np.abs(full.numpy() - ref)) / np.max(np.abs(ref)))
    dist.destroy_process_group()


def _run(fn, world=2):
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    procs = [ctx.Process(target=fn, args=(r, world, port, out)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=300)
    assert all(p.exitcode == 0 for p in procs), [p.exitcode for p in procs]
    return dict(out)


def test_bench_takes_the_slowest_rank():
    out = _run(_bench_worker)
    for rank in (0, 1):
        ms, value = out[rank]
        assert ms == 20.0
        assert value == pytest.approx(2 * 1000 * 5 / 0.020)


def test_sharded_image_equals_whole_image():
    out = _run(_sharded_worker)
    assert out[0] < 1e-12
