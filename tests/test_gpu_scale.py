"""The 16384^2 / 128 w-plane / 2e8 measurement configuration with uniform
weighting on the GPU, in the plane-group launch configuration the library
picks for it (the planes do not all fit at once): sampled pixels against the
FP64 oracle's per-pixel evaluation at a 16 x 16 pixel lattice spanning the
image edge to edge (1e-4 of the image peak, compared before the taper
division), no drops, and the uniform-weighting weight sum equal to
the number of occupied cells."""
import numpy as np
import pytest
import torch

import synth

pytestmark = pytest.mark.gpu

CORRECT, REAL, UNIFORM = synth.FLAG_CORRECT, synth.FLAG_REAL, synth.FLAG_UNIFORM


@pytest.fixture(scope="module")
def rick():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2504_00959_gb300 import build
    build.build()
    import paper_2504_00959_gb300 as r
    r.load()
    return r


def test_config3_plane_groups_uniform_weighting(rick, oracle_mod):
    prob = synth.config3(device="cuda")
    q = prob["params"]
    n = q["n"]
    im = rick.Imager(dict(q, flags=CORRECT | REAL | UNIFORM))
    im.grid(prob["vis"], prob["u"], prob["v"], prob["w"], prob["wt"])
    img = im.image()
    torch.cuda.synchronize()
    st = im.stats()
    im.close()
    assert st["plane_group"] < q["nw"]  # several plane groups
    assert st["n_dropped"] == 0 and st["n_gridded"] == prob["u"].numel()
    # weight sum of uniform weighting = occupied nearest cells (binary32 decisions
    # rebuilt here with torch; rare half-cell ties may differ, hence the tolerance)
    s = torch.tensor(n * q["pixel_rad"], dtype=torch.float32).item()
    cu = torch.floor(prob["u"] * s + n / 2 + 0.5).to(torch.int64)
    cv = torch.floor(prob["v"] * s + n / 2 + 0.5).to(torch.int64)
    occupied = torch.unique(cv * n + cu).numel()
    assert abs(st["sum_weights"] - occupied) <= 1e-5 * occupied
    del cu, cv
    flat = int(torch.argmax(img.abs()).item())
    xs = np.unique(np.linspace(0, n - 1, 16).round().astype(np.int64))
    pix = {(int(x), int(y)) for y in xs for x in xs} | {(flat % n, flat // n), (n // 2, n // 2),
                                                       (n // 2 + 1234, n // 2 - 777)}
    pix = np.array(sorted(pix), np.int32)
    assert pix.shape[0] >= 256
    got = img.cpu().numpy()[pix[:, 1], pix[:, 0]]
    del img
    p = synth.to_numpy(prob)
    del prob
    # the oracle before the taper division; the GPU image times c(x) c(y)
    ref = oracle_mod.image_at(dict(q), p["u"], p["v"], p["w"], p["wt"], p["vis"], pix, flags=UNIFORM).real
    c = oracle_mod.taper(n, synth.KERNEL_KB, q["support"], 0.0)
    got = got * c[pix[:, 0]] * c[pix[:, 1]]
    assert np.max(np.abs(got - ref)) <= 1e-4 * np.max(np.abs(ref)), (np.max(np.abs(got - ref)), np.max(np.abs(ref)))


def test_maximum_grid_side(rick, oracle_mod):
    """The largest grid the library accepts, 32768^2 (n^2 > 2^30: the 64-bit
    index paths of the sort, the gridder's tile stores, cuFFT and the stack),
    2 w-planes (17 GB of planes), 2e5 measurements with uniform weighting:
    sampled pixels against the oracle's per-pixel evaluation at 1e-4 of the
    peak."""
    n = 32768
    prob = synth.disk_problem(n, 2, 200000, synth.KERNEL_KB, 7, 4.0, 300.0, 511, fill=0.45)
    q = dict(prob["params"], flags=REAL | CORRECT | UNIFORM)
    g = {k: prob[k].cuda() for k in ("vis", "u", "v", "w", "wt")}
    im = rick.Imager(q)
    im.grid(g["vis"], g["u"], g["v"], g["w"], g["wt"])
    img = im.image()
    torch.cuda.synchronize()
    st = im.stats()
    im.close()
    assert st["n_gridded"] + st["n_dropped"] == 200000
    rng = np.random.default_rng(29)
    flat = int(torch.argmax(img.abs()).item())
    pix = [(flat % n, flat // n), (n // 2, n // 2), (n - 1, n - 1), (0, n // 2 + 3)]
    pix += [tuple(rng.integers(0, n, 2)) for _ in range(4)]
    pix = np.array(pix, np.int32)
    got = img[torch.from_numpy(pix[:, 1]).long().cuda(), torch.from_numpy(pix[:, 0]).long().cuda()].cpu().numpy()
    del img
    p = synth.to_numpy(prob)
    ref = oracle_mod.image_at(q, p["u"], p["v"], p["w"], p["wt"], p["vis"], pix, flags=CORRECT | UNIFORM).real
    c = oracle_mod.taper(n, synth.KERNEL_KB, 7, 0.0)
    cc = c[pix[:, 0]] * c[pix[:, 1]]
    assert np.max(np.abs(got - ref) * cc) <= 1e-4 * np.max(np.abs(ref) * cc), (got, ref)
