"""rick_grid_planes_static: gridding for callers that cannot allocate device
memory (a host framework that owns the whole device heap, a context where
cudaMalloc is not permitted, a real-time loop that forbids allocation after
start-up).  Its working memory is a fixed 64 MiB array in the library's
static device data.

Checked through the C ABI against the allocating path (rick_create +
rick_grid + rick_grid_planes) on two calls in a row, at the tolerance the
other plane comparisons use (1e-5 of the largest cell), plus the size limit.
This file is collected last so that a run stopping at the first failure has
run every other test; it passes alone in a fresh process too.
"""
import ctypes

import numpy as np
import pytest
import torch

import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rick():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2504_00959_gb300 import build
    build.build()
    import paper_2504_00959_gb300 as r
    r.load()
    return r


def _p(t):
    return ctypes.c_void_p(t.data_ptr() if t is not None else None)


def _call(rick, params, prob, planes, err):
    from paper_2504_00959_gb300 import _lib
    rp = rick._params_struct(params)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    return _lib.load().rick_grid_planes_static(
        ctypes.byref(rp), _p(prob["vis"]), _p(prob["u"]), _p(prob["v"]), _p(prob["w"]), _p(prob["wt"]),
        prob["u"].numel(), _p(planes), stream, err, len(err))


@pytest.mark.parametrize("flags", [synth.FLAG_CORRECT | synth.FLAG_REAL, synth.FLAG_UNIFORM])
def test_static_scratch_matches_allocating_path(rick, flags):
    prob = synth.config1(device="cuda")
    params = dict(prob["params"], flags=flags)
    im = rick.Imager(params)
    im.grid(prob["vis"], prob["u"], prob["v"], prob["w"], prob["wt"])
    ref = im.grid_planes()
    torch.cuda.synchronize()
    im.close()
    nw, n = params["nw"], params["n"]
    err = ctypes.create_string_buffer(512)
    for _ in range(2):
        out = torch.full((nw, n, n), float("nan"), dtype=torch.complex64, device="cuda")
        status = _call(rick, params, prob, out, err)
        assert status == 0, err.value.decode()
        torch.cuda.synchronize()
        assert torch.isfinite(out).all().item()  # every cell written
        diff = torch.max(torch.abs(out - ref)).item()
        assert diff <= 1e-5 * torch.max(torch.abs(ref)).item(), diff


def test_static_scratch_rejects_sizes_beyond_the_limit(rick):
    m = 2_000_000  # 4 * 16 bytes of entries per measurement: 128 MB > 64 MiB
    params = synth.make_params(4096, 32, 1e-5, -100.0, 100.0, synth.KERNEL_KB, 7)
    prob = dict(u=torch.zeros(m, device="cuda"), v=torch.zeros(m, device="cuda"), w=torch.zeros(m, device="cuda"),
                wt=torch.ones(m, device="cuda"), vis=torch.zeros(m, dtype=torch.complex64, device="cuda"))
    planes = torch.empty((1,), dtype=torch.complex64, device="cuda")  # never written: the call is refused first
    err = ctypes.create_string_buffer(512)
    status = _call(rick, params, prob, planes, err)
    assert status == 1  # RICK_ERR_ARG
    assert "limit" in err.value.decode()


def test_static_scratch_hot_tile(rick):
    """2e5 measurements inside one cell of a 128^2 x 4-plane grid: the static
    scratch lists the hot tiles in its cursor array (two counters, then one
    word per tile) for the heavy-tile CTAs; the planes must agree with
    the allocating path (1e-4 of the largest cell: the hot cell sums 2e5 FP32
    terms, in an order that depends on the scatter's slots)."""
    n = 128
    prob = synth.disk_problem(n, 4, 20000, synth.KERNEL_KB, 7, 3.0, 50.0, 11)
    du = 1 / (n * prob["params"]["pixel_rad"])
    g = torch.Generator().manual_seed(5)
    hot = 200000
    prob = dict(params=prob["params"],
                u=torch.cat([prob["u"], (3.2 + 0.3 * torch.rand(hot, generator=g)) * du]).cuda(),
                v=torch.cat([prob["v"], (-1.7 + 0.3 * torch.rand(hot, generator=g)) * du]).cuda(),
                w=torch.cat([prob["w"], torch.full((hot,), 1.0)]).cuda(),
                wt=torch.ones(20000 + hot, device="cuda"),
                vis=torch.cat([prob["vis"], torch.complex(torch.randn(hot, generator=g),
                                                          torch.randn(hot, generator=g))]).cuda())
    params = dict(prob["params"], flags=synth.FLAG_REAL)
    im = rick.Imager(params)
    im.grid(prob["vis"], prob["u"], prob["v"], prob["w"], prob["wt"])
    ref = im.grid_planes()
    torch.cuda.synchronize()
    im.close()
    out = torch.full((4, n, n), float("nan"), dtype=torch.complex64, device="cuda")
    err = ctypes.create_string_buffer(512)
    assert _call(rick, params, prob, out, err) == 0, err.value.decode()
    torch.cuda.synchronize()
    assert torch.isfinite(out).all().item()
    diff = torch.max(torch.abs(out - ref)).item()
    assert diff <= 1e-4 * torch.max(torch.abs(ref)).item(), diff
