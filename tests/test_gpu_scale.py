"""The 16384^2 / 128 w-plane / 2e8 measurement configuration with uniform
weighting on the GPU, in the plane-group launch configuration the library
picks for it (the planes do not all fit at once): sampled pixels against the
FP64 oracle's per-pixel evaluation (1e-4 of the image peak, before and after
grid correction), no drops, and the uniform-weighting weight sum equal to
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
    im = rick.Imager(dict(q, flags=REAL | UNIFORM))
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
    rng = np.random.default_rng(23)
    pix = [(flat % n, flat // n), (n // 2, n // 2), (n // 2 + 1234, n // 2 - 777)]
    pix += [tuple(rng.integers(n // 4, 3 * n // 4, 2)) for _ in range(2)]
    pix = np.array(pix, np.int32)
    got = img.cpu().numpy()[pix[:, 1], pix[:, 0]]
    peak = img.abs().max().item()
    del img
    p = synth.to_numpy(prob)
    del prob
    ref = oracle_mod.image_at(dict(q), p["u"], p["v"], p["w"], p["wt"], p["vis"], pix, flags=UNIFORM)
    assert np.max(np.abs(got - ref.real)) <= 1e-4 * peak, (got, ref.real, peak)
