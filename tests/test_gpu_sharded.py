"""One image shared by two ranks through librick (ShardedImager): two
processes on the one GPU, a gloo group for the all-reduce (the library's
kernels of the two ranks never wait on each other).  Each rank images its
share -- half of the w-planes of all measurements (rick_set_plane_range), or
half of the measurements normalised by the summed weight sum
(rick_set_weight_sum) -- and the sum of the two images must equal the
single-rank image (1e-5 of the peak) and the FP64 oracle (1e-4)."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import synth

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CORRECT, REAL, UNIFORM = synth.FLAG_CORRECT, synth.FLAG_REAL, synth.FLAG_UNIFORM


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _problem():
    return synth.disk_problem(256, 8, 40000, synth.KERNEL_KB, 7, 3.0, 80.0, 4321, weights="random")


def _worker(rank, world, port, out, mode, flags):
    import sys
    if ROOT not in sys.path:
        sys.path.insert(0, ROOT)
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    torch.cuda.set_device(0)
    from paper_2504_00959_gb300.sharded import ShardedImager
    prob = _problem()
    q = dict(prob["params"], flags=flags)
    g = {k: prob[k].cuda() for k in ("vis", "u", "v", "w", "wt")}
    m = prob["u"].numel()
    sl = slice(rank * m // world, (rank + 1) * m // world) if mode == "measurements" else slice(0, m)
    sh = ShardedImager(q, device=torch.device("cuda", 0), mode=mode)
    for _ in range(2):  # twice: reset keeps the share
        sh.reset()
        sh.grid(g["vis"][sl], g["u"][sl], g["v"][sl], g["w"][sl], g["wt"][sl])
        img = sh.image()
    torch.cuda.synchronize()
    out[rank] = img.cpu().numpy()
    sh.close()
    dist.destroy_process_group()


@pytest.fixture(scope="module")
def rick():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2504_00959_gb300 import build
    build.build()
    import paper_2504_00959_gb300 as r
    r.load()
    return r


@pytest.mark.parametrize("mode,flags", [("planes", CORRECT | REAL), ("planes", CORRECT | REAL | UNIFORM),
                                        ("measurements", CORRECT | REAL), ("measurements", CORRECT)])
def test_two_ranks_sum_to_the_image(rick, oracle_mod, mode, flags):
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, out, mode, flags)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=600)
    assert all(p.exitcode == 0 for p in procs), [p.exitcode for p in procs]
    a, b = out[0], out[1]
    assert np.array_equal(a, b)  # every rank holds the summed image
    prob = _problem()
    q = dict(prob["params"], flags=flags)
    g = {k: prob[k].cuda() for k in ("vis", "u", "v", "w", "wt")}
    im = rick.Imager(q)
    im.grid(g["vis"], g["u"], g["v"], g["w"], g["wt"])
    one = im.image().cpu().numpy()
    im.close()
    assert np.max(np.abs(a - one)) <= 1e-5 * np.max(np.abs(one))
    p = synth.to_numpy(prob)
    ref, _, _ = oracle_mod.dirty_image(q, p["u"], p["v"], p["w"], p["wt"], p["vis"], flags=flags & ~REAL & ~CORRECT)
    n = q["n"]
    c = oracle_mod.taper(n, synth.KERNEL_KB, 7, 0.0)
    cc = np.outer(c, c) if flags & CORRECT else np.ones((n, n))
    ref = ref.real if flags & REAL else ref
    assert np.max(np.abs(a * cc - ref)) <= 1e-4 * np.max(np.abs(ref))
