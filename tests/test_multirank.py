"""Multi-process host logic on CPU ranks (torch.distributed, gloo,
world_size 2): the benchmark's max-over-ranks timing and whole-job value, and
the one exchange a sharded image needs -- the sum of the partial images,
each normalised by the common weight sum, over shares of the w-planes or of
the measurements -- checked against the FP64 oracle's image of everything."""
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


class _OracleImager:
    """The per-rank imager interface of ShardedImager backed by the FP64
    oracle on the CPU (the host logic of sharding, without a GPU)."""

    def __init__(self, params, device=None):
        self.q = dict(params)
        self.lo, self.hi = 0, int(params["nw"])
        self.sw_given = None
        self.data = None

    def set_plane_range(self, k0, k1):
        self.lo, self.hi = k0, k1

    def set_weight_sum(self, s):
        self.sw_given = s

    def reset(self):
        self.data = None

    def grid(self, vis, u, v, w, wt=None):
        self.data = (vis, u, v, w, wt)

    def _args(self):
        vis, u, v, w, wt = self.data
        return u.numpy(), v.numpy(), w.numpy(), wt.numpy(), vis.numpy()

    def stats(self):
        import oracle
        _, sw, _ = oracle.grid(self.q, *self._args(), k0=0, k1=0)
        return {"sum_weights": sw}

    def image(self, out=None):
        import oracle
        img, sw, _ = oracle.dirty_image(self.q, *self._args(), k0=self.lo, k1=self.hi)
        if self.sw_given is not None:
            img = img * (sw / self.sw_given)
        return torch.from_numpy(img)

    def close(self):
        pass


def _sharded_worker(rank, world, port, out, mode, flags):
    _init(rank, world, port)
    import oracle
    import synth
    from paper_2504_00959_gb300.sharded import ShardedImager
    prob = synth.disk_problem(64, 5, 3000, synth.KERNEL_KB, 7, 4.0, 60.0, 91, weights="random")
    q = dict(prob["params"], flags=flags)
    m = prob["u"].numel()
    sh = ShardedImager(q, mode=mode, imager_factory=_OracleImager)
    sl = slice(rank * m // world, (rank + 1) * m // world) if mode == "measurements" else slice(0, m)
    sh.grid(prob["vis"][sl], prob["u"][sl], prob["v"][sl], prob["w"][sl], prob["wt"][sl])
    full = sh.image()
    out[rank] = (sh.k0, sh.k1)
    if rank == 0:
        p = synth.to_numpy(prob)
        ref, _, _ = oracle.dirty_image(q, p["u"], p["v"], p["w"], p["wt"], p["vis"])
        out["err"] = float(np.max(np.abs(full.numpy() - ref)) / np.max(np.abs(ref)))
    dist.destroy_process_group()


def _run(fn, world=2, *extra):
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    procs = [ctx.Process(target=fn, args=(r, world, port, out) + extra) for r in range(world)]
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
        assert value == pytest.approx(1000 * 5 / 0.020)


@pytest.mark.parametrize("mode,flags", [("planes", 1), ("planes", 1 | 8), ("measurements", 1)])
def test_sharded_image_equals_whole_image(mode, flags):
    """Two ranks, each imaging its share (half the w-planes with all
    measurements, or half the measurements normalised by the summed weight
    sum; uniform weighting with the plane shares), summed by one all-reduce:
    the FP64 oracle's image of everything."""
    out = _run(_sharded_worker, 2, mode, flags)
    assert out["err"] < 1e-12
    if mode == "planes":
        assert (out[0], out[1]) == ((0, 2), (2, 5))


def test_plane_share_covers_the_planes():
    from paper_2504_00959_gb300.sharded import plane_share
    for nw in (1, 5, 32, 128):
        for world in range(1, min(nw, 9) + 1):
            spans = [plane_share(nw, r, world) for r in range(world)]
            assert spans[0][0] == 0 and spans[-1][1] == nw
            assert all(a[1] == b[0] and a[0] < a[1] for a, b in zip(spans, spans[1:]))
    with pytest.raises(ValueError):
        plane_share(4, 0, 5)
