"""GPU (sm_103a, librick) against the FP64 oracle on identical seeded inputs.

Tolerance: max |D_gpu - D_oracle| <= 1e-4 * max |D_oracle| for FP32 images.
Grid correction divides pixel (x, y) by c(x) c(y), which falls to ~1e-6 at
the corners for the Gaussian kernel; FP32 rounding of the FFT (~1e-7 of the
plane) is amplified by the same factor, so for corrected images the 1e-4
bound is applied to c(x) c(y) D (the image before the division) everywhere,
and to D itself where c(x) c(y) >= 1/4.  Gridded planes are compared at 1e-5
of their largest cell.  Integer work (drop and entry counts) is exact.
"""
import math

import numpy as np
import pytest
import torch

import synth

pytestmark = pytest.mark.gpu

KB, GAUSS = synth.KERNEL_KB, synth.KERNEL_GAUSS
CORRECT, REAL, APPLY_N, UNIFORM = synth.FLAG_CORRECT, synth.FLAG_REAL, synth.FLAG_APPLY_N, synth.FLAG_UNIFORM
TOL = 1e-4


@pytest.fixture(scope="module")
def rick():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2504_00959_gb300 import build
    build.build()
    import paper_2504_00959_gb300 as r
    r.load()
    return r


def _to(prob, dev="cuda"):
    return {k: (v.to(dev) if isinstance(v, torch.Tensor) else v) for k, v in prob.items()}


def _gpu_image(rick, prob, flags, chunks=1, **extra):
    prob = _to(prob)
    params = dict(prob["params"], flags=flags, **extra)
    im = rick.Imager(params)
    m = prob["u"].numel()
    edges = np.linspace(0, m, chunks + 1).astype(int)
    for a, b in zip(edges[:-1], edges[1:]):
        im.grid(prob["vis"][a:b].contiguous(), prob["u"][a:b].contiguous(), prob["v"][a:b].contiguous(),
                prob["w"][a:b].contiguous(), prob["wt"][a:b].contiguous())
    img = im.image()
    torch.cuda.synchronize()
    st = im.stats()
    im.close()
    return img.cpu().numpy(), st


def _oracle_image(oracle_mod, prob, flags):
    p = synth.to_numpy(prob)
    return oracle_mod.dirty_image(p["params"], p["u"], p["v"], p["w"], p["wt"], p["vis"], flags=flags)


def _rel_err(got, ref, mask=None):
    d = np.abs(got - ref)
    if mask is not None:
        d = d[mask]
    return float(d.max()) / float(np.abs(ref).max())


def _image_errors(oracle_mod, params, got, ref, flags):
    """(error bound ratio over the whole image, over the central region)."""
    if not flags & CORRECT:
        e = _rel_err(got, ref)
        return e, e
    c = oracle_mod.taper(params["n"], params["kernel"], params["support"], params.get("kernel_param", 0.0))
    cc = np.outer(c, c)
    whole = float(np.max(np.abs(got - ref) * cc)) / float(np.max(np.abs(ref) * cc))
    centre = _rel_err(got, ref, cc >= 0.25)
    return whole, centre


def _compare(rick, oracle_mod, prob, flags, tol=TOL, chunks=1, **extra):
    got, st = _gpu_image(rick, prob, flags, chunks=chunks, **extra)
    ref, sw, dropped = _oracle_image(oracle_mod, prob, flags & ~REAL)
    if flags & REAL:
        ref = ref.real
    whole, centre = _image_errors(oracle_mod, prob["params"], got, ref, flags)
    assert whole <= tol and centre <= tol, (whole, centre, tol)
    assert st["n_dropped"] == dropped
    assert abs(st["sum_weights"] - sw) <= 1e-5 * max(1.0, abs(sw))
    return got, ref, st


# ----------------------------------------------------------------- config 1

@pytest.mark.parametrize("flags", [REAL, CORRECT | REAL, CORRECT, CORRECT | REAL | APPLY_N])
def test_config1_full_image(rick, oracle_mod, flags):
    """256^2, 8 w-planes, 1e5 visibilities, Gaussian support 7, 2 deg."""
    prob = synth.config1()
    _compare(rick, oracle_mod, prob, flags)


def test_config1_planes_match_oracle_grid(rick, oracle_mod):
    prob = synth.config1()
    p = synth.to_numpy(prob)
    ref, sw, _ = oracle_mod.grid(p["params"], p["u"], p["v"], p["w"], p["wt"], p["vis"])
    im = rick.Imager(dict(prob["params"]))
    g = _to(prob)
    im.grid(g["vis"], g["u"], g["v"], g["w"], g["wt"])
    planes = im.grid_planes().cpu().numpy()
    im.close()
    scale = np.abs(ref).max()
    assert np.max(np.abs(planes - ref)) <= 1e-5 * scale
    # Eq. 3 with normalised taps keeps the weighted visibility sum
    tot = np.sum(p["wt"].astype(np.float64) * p["vis"].astype(np.complex128))
    assert abs(planes.astype(np.complex128).sum() - tot) <= 1e-5 * np.sum(np.abs(p["vis"]))


@pytest.mark.parametrize("m,support,tile", [(4000, 7, 32), (40000, 8, 32), (20000, 7, 16), (20000, 8, 64),
                                             (60000, 6, 32)])
def test_light_tiles_planes_match_oracle_grid(rick, oracle_mod, m, support, tile):
    """Sparse planes: tiles of 0 to a few dozen entries, so runs of
    consecutive light tiles share a staging round (at most 32 entries in
    all) and heavier ones take rounds of their own, in every mixture.  The
    gridded planes (natural rows) equal those of a pass over two lists of
    the same measurements (tile by tile, no shared rounds) to FP32
    reordering, and the oracle's Eq. 3 within the tap fit's error: each
    fitted tap is within 2e-6 of the kernel's peak (the bound k_fit_taps
    enforces), so a term of a cell is off by up to ~4e-6 of the term at the
    footprint's centre, whatever the cell's own tap; a sparse plane's peak
    cell holds one or a few terms while other cells sum several, hence 5e-5
    of the peak here (the dense config-1 planes hold 1e-5).  The image
    through the split transform (b-major rows) matches the oracle at 1e-4."""
    prob = synth.disk_problem(512, 4, m, synth.KERNEL_KB, support, 3.0, 60.0, 900 + m + support + tile,
                              weights="random")
    p = synth.to_numpy(prob)
    ref, _, _ = oracle_mod.grid(p["params"], p["u"], p["v"], p["w"], p["wt"], p["vis"])
    g = _to(prob)
    planes = []
    for parts in (1, 2):
        im = rick.Imager(dict(prob["params"], tile=tile))
        edges = np.linspace(0, m, parts + 1).astype(int)
        for a, b in zip(edges[:-1], edges[1:]):
            im.grid(g["vis"][a:b].contiguous(), g["u"][a:b].contiguous(), g["v"][a:b].contiguous(),
                    g["w"][a:b].contiguous(), g["wt"][a:b].contiguous())
        planes.append(im.grid_planes().cpu().numpy())
        im.close()
    peak = np.abs(ref).max()
    assert np.max(np.abs(planes[0] - planes[1])) <= 1e-6 * peak
    assert np.max(np.abs(planes[0] - ref)) <= 5e-5 * peak
    _compare(rick, oracle_mod, prob, CORRECT | REAL | rick.FFT_SPLIT, tile=tile)


def test_config1_entries_and_counters_exact(rick, oracle_mod):
    """Integer work: entry count = sum over gridded measurements of the tiles
    their footprint touches (computed from the oracle's placement)."""
    prob = synth.config1()
    p = synth.to_numpy(prob)
    k, fu, fv = oracle_mod.place(p["params"], p["u"], p["v"], p["w"])
    ok = k >= 0
    S = p["params"]["support"]
    T = 32
    nt = ((fu[ok] + S - 1) // T - fu[ok] // T + 1) * ((fv[ok] + S - 1) // T - fv[ok] // T + 1)
    _, st = _gpu_image(rick, prob, CORRECT | REAL, tile=T)
    assert st["n_gridded"] == int(ok.sum())
    assert st["n_entries"] == int(nt.sum())
    assert st["n_dropped"] == int((~ok).sum())


# ------------------------------------------------------- shapes and tiles

@pytest.mark.parametrize("n,tile,kernel,support", [(200, 32, KB, 7), (96, 64, KB, 8), (64, 16, GAUSS, 5),
                                                   (72, 16, KB, 16)])
def test_ragged_and_tiles(rick, oracle_mod, n, tile, kernel, support):
    """Grid sides that are not multiples of the tile (a ragged last tile) and
    every tile size, KB and Gaussian, supports up to 16."""
    prob = synth.disk_problem(n, 4, 20000, kernel, support, 3.0, 60.0, 101 + n, weights="random")
    _compare(rick, oracle_mod, prob, CORRECT | REAL, tile=tile)


@pytest.mark.parametrize("n,nw,kernel,support,tile", [(16, 1, KB, 1, 16), (32, 2, KB, 2, 16),
                                                       (34, 3, KB, 3, 16), (8, 1, GAUSS, 4, 16),
                                                       (64, 1, KB, 6, 32)])
def test_degenerate_shapes(rick, oracle_mod, n, nw, kernel, support, tile):
    """The smallest supports (a one-cell footprint, one and two cell pairs per
    row), a single w-plane (w ignored), the smallest grid the tile allows and
    a ragged tile, against the oracle."""
    prob = synth.disk_problem(n, nw, 3000, kernel, support, 3.0, 60.0, 131 + n + support, weights="random",
                              fill=0.35)
    _compare(rick, oracle_mod, prob, CORRECT | REAL, tile=tile)
    _compare(rick, oracle_mod, prob, APPLY_N, tile=tile)


def test_kernel_too_sharp_for_its_taps_is_refused(rick):
    """The Gaussian's default width for support 2 (sigma = 1/3 cell) is too
    sharp for degree-10 tap polynomials: creation fails and says why."""
    with pytest.raises(rick.RickError, match="too sharp"):
        rick.Imager(synth.make_params(32, 2, 1e-3, -60.0, 60.0, GAUSS, 2))


def test_plane_groups_equal_all_planes(rick, oracle_mod):
    prob = synth.disk_problem(128, 8, 30000, KB, 7, 4.0, 80.0, 103)
    a, _, _ = _compare(rick, oracle_mod, prob, CORRECT | REAL, plane_group=3)
    b, _ = _gpu_image(rick, prob, CORRECT | REAL)
    assert np.max(np.abs(a - b)) <= 1e-5 * np.abs(b).max()


@pytest.mark.parametrize("chunks", [3, 17, 20])
def test_chunks_accumulate(rick, oracle_mod, chunks):
    """Several grid() calls equal one (17 and 20 chunks also exercise the
    read-modify-write gridding pass beyond 16 chunks: with 17 it reads one
    list, the path that stages runs of light tiles together)."""
    prob = synth.disk_problem(128, 4, 40000, GAUSS, 7, 2.0, 50.0, 107)
    _compare(rick, oracle_mod, prob, CORRECT | REAL, chunks=chunks)


def test_uniform_weighting(rick, oracle_mod):
    prob = synth.disk_problem(128, 4, 40000, KB, 7, 2.0, 50.0, 109, fill=0.3)
    _compare(rick, oracle_mod, prob, CORRECT | REAL | UNIFORM)


def test_uniform_weighting_with_chunks_and_add_density(rick, oracle_mod):
    prob = synth.disk_problem(128, 4, 40000, KB, 7, 2.0, 50.0, 113, fill=0.3)
    g = _to(prob)
    im = rick.Imager(dict(prob["params"], flags=CORRECT | REAL | UNIFORM))
    halves = [(0, 15000), (15000, 40000)]
    for a, b in halves:
        im.add_density(g["vis"][a:b], g["u"][a:b], g["v"][a:b], g["w"][a:b], g["wt"][a:b])
    for a, b in halves:
        im.grid(g["vis"][a:b], g["u"][a:b], g["v"][a:b], g["w"][a:b], g["wt"][a:b])
    got = im.image().cpu().numpy()
    im.close()
    ref, _, _ = _oracle_image(oracle_mod, prob, CORRECT | UNIFORM)
    whole, centre = _image_errors(oracle_mod, prob["params"], got, ref.real, CORRECT)
    assert whole <= TOL and centre <= TOL


# ------------------------------------------------------------- edge cases

def test_empty_input_gives_zero_image(rick):
    prob = synth.disk_problem(64, 4, 0, KB, 7, 2.0, 50.0, 1)
    got, st = _gpu_image(rick, prob, CORRECT | REAL)
    assert np.all(got == 0) and st["n_gridded"] == 0


def test_all_dropped(rick, oracle_mod):
    prob = synth.disk_problem(64, 4, 1000, KB, 7, 2.0, 50.0, 3)
    prob["u"] = prob["u"] + 1e7  # far outside the grid
    got, st = _gpu_image(rick, prob, CORRECT | REAL)
    assert st["n_dropped"] == 1000 and np.all(got == 0)


def test_non_finite_inputs_are_dropped_and_counted(rick, oracle_mod):
    prob = synth.disk_problem(64, 4, 2000, KB, 7, 2.0, 50.0, 5, fill=0.4)
    prob["u"][3] = float("nan")
    prob["v"][10] = float("inf")
    prob["w"][20] = float("nan")
    prob["wt"][30] = float("nan")
    prob["vis"][40] = complex(float("nan"), 0.0)
    _, st = _gpu_image(rick, prob, CORRECT | REAL)
    assert st["n_dropped"] == 5
    keep = torch.ones(2000, dtype=torch.bool)
    keep[[3, 10, 20, 30, 40]] = False
    clean = {k: (v[keep] if isinstance(v, torch.Tensor) else v) for k, v in prob.items()}
    # uncorrected images: only the order of FP32 sums may differ
    a, _ = _gpu_image(rick, prob, REAL)
    b, _ = _gpu_image(rick, clean, REAL)
    assert np.max(np.abs(a - b)) <= 1e-6 * np.abs(b).max()


def test_single_visibility(rick, oracle_mod):
    n = 64
    pixel_rad = math.radians(10.0) / n
    du = 1 / (n * pixel_rad)
    params = synth.make_params(n, 5, pixel_rad, -40.0, 40.0, KB, 7, 0.0, CORRECT | REAL)
    prob = dict(params=params, u=torch.tensor([5.3 * du]), v=torch.tensor([-11.7 * du]), w=torch.tensor([17.0]),
                wt=torch.tensor([2.0]), vis=torch.tensor([0.3 + 0.9j], dtype=torch.complex64))
    _compare(rick, oracle_mod, prob, CORRECT | REAL)
    _compare(rick, oracle_mod, prob, 0)


def test_grid_edges_and_plane_boundaries(rick, oracle_mod):
    """Footprints touching the first and last cells, measurements exactly on
    plane boundaries and at w_min / w_max, at half-cell offsets."""
    n, S = 64, 7
    pixel_rad = math.radians(5.0) / n
    du = 1 / (n * pixel_rad)
    cells_lo = -n / 2 + S / 2 - 0.49        # first cell 0
    cells_hi = n / 2 - S / 2 - 1 + 0.49     # last cell n-1
    pos = np.array([cells_lo, cells_hi, 0.5, -0.5, 3.0, -7.5, 10.25]) * du
    uu, vv = np.meshgrid(pos, pos)
    m = uu.size
    w_edges = np.array([-40.0, 40.0, 0.0, -20.0, 20.0, -10.0, 10.0])
    ww = np.resize(w_edges, m)
    params = synth.make_params(n, 8, pixel_rad, -40.0, 40.0, KB, S, 0.0, CORRECT | REAL)
    rng = np.random.default_rng(9)
    prob = dict(params=params, u=torch.tensor(uu.ravel(), dtype=torch.float32),
                v=torch.tensor(vv.ravel(), dtype=torch.float32), w=torch.tensor(ww, dtype=torch.float32),
                wt=torch.ones(m), vis=torch.tensor(rng.standard_normal(m) + 1j * rng.standard_normal(m),
                                                   dtype=torch.complex64))
    _, _, st = _compare(rick, oracle_mod, prob, CORRECT | REAL)
    assert st["n_dropped"] == 0


def test_hot_tile(rick, oracle_mod):
    """2e5 measurements inside one cell next to 2e4 spread ones (heavy skew
    of the per-tile lists)."""
    n = 128
    prob = synth.disk_problem(n, 4, 20000, KB, 7, 3.0, 50.0, 11)
    du = 1 / (n * prob["params"]["pixel_rad"])
    g = torch.Generator().manual_seed(5)
    hot = 200000
    u = torch.cat([prob["u"], (3.2 + 0.3 * torch.rand(hot, generator=g)) * du])
    v = torch.cat([prob["v"], (-1.7 + 0.3 * torch.rand(hot, generator=g)) * du])
    w = torch.cat([prob["w"], torch.full((hot,), 1.0)])
    wt = torch.ones(u.numel())
    vis = torch.cat([prob["vis"], torch.complex(torch.randn(hot, generator=g), torch.randn(hot, generator=g))])
    _compare(rick, oracle_mod, dict(params=prob["params"], u=u, v=v, w=w, wt=wt, vis=vis), CORRECT | REAL)


@pytest.mark.parametrize("chunks,hot", [(1, 2000), (1, 20000), (17, 20000), (17, 120000)])
def test_heavy_tile_cta(rick, oracle_mod, chunks, hot):
    """`hot` measurements in a 3 x 3-cell patch, all inside one 32 x 32 tile
    of a 512^2 grid, beside 2e4 spread ones.  2e3 entries: a heavy tile, one
    CTA whose warps grid shares of the entries into private copies summed
    before the one store; 2e4: a huge tile (more than 8 warps x 512
    entries), shared by the CTAs of a thread-block cluster, whose sums are
    added through distributed shared memory.  With 17 grid() calls the last call
    holds only hot measurements (2353 of 4e4, or 8235 of 1.4e5) and is
    gridded in a pass of its own that adds onto the plane (the heavy or huge
    tile read back and summed onto)."""
    n = 512
    prob = synth.disk_problem(n, 2, 20000, KB, 7, 3.0, 50.0, 13)
    du = 1 / (n * prob["params"]["pixel_rad"])
    g = torch.Generator().manual_seed(6)
    u = torch.cat([prob["u"], (40.2 + 3.0 * torch.rand(hot, generator=g)) * du])
    v = torch.cat([prob["v"], (-21.7 + 3.0 * torch.rand(hot, generator=g)) * du])
    w = torch.cat([prob["w"], torch.full((hot,), -10.0)])
    wt = torch.ones(u.numel())
    vis = torch.cat([prob["vis"], torch.complex(torch.randn(hot, generator=g), torch.randn(hot, generator=g))])
    _compare(rick, oracle_mod, dict(params=prob["params"], u=u, v=v, w=w, wt=wt, vis=vis), REAL, chunks=chunks)


def test_tile_sides_in_turn(rick, oracle_mod):
    """Imagers with tile sides 32, 64, 16 and 32 again in one process, as the
    batch autotuner creates them: each tile side launches the gridder's
    kernels with its own shared-memory size, and every image must still
    match the oracle (a per-kernel shared-memory ceiling set for one tile
    side must not fail the launches of another)."""
    prob = synth.disk_problem(256, 4, 30000, KB, 7, 3.0, 50.0, 17)
    for tile in (32, 64, 16, 32):
        _compare(rick, oracle_mod, prob, CORRECT | REAL, tile=tile)


def test_hermitian_fold_matches_oracle(rick, oracle_mod):
    """Config 1 folded onto 4 w-planes over [0, 50] (RICK_HERMITIAN_FOLD)."""
    prob = synth.config1()
    prob["params"] = dict(prob["params"], nw=4, w_min=0.0)
    _compare(rick, oracle_mod, prob, CORRECT | REAL | synth.FLAG_FOLD)


def test_hermitian_fold_equals_unfolded_on_mirrored_planes(rick, oracle_mod):
    """The folded real image on 4 planes over [0, 50] against the unfolded one
    on 8 planes over [-50, 50] (mirrored plane centres): same sum in another
    FP32 order."""
    prob = synth.config1()
    a, _ = _gpu_image(rick, prob, CORRECT | REAL)
    folded = dict(prob, params=dict(prob["params"], nw=4, w_min=0.0))
    b, _ = _gpu_image(rick, folded, CORRECT | REAL | synth.FLAG_FOLD)
    q = prob["params"]
    c = oracle_mod.taper(q["n"], q["kernel"], q["support"], q.get("kernel_param", 0.0))
    cc = np.outer(c, c)
    assert float(np.max(np.abs(a - b) * cc)) <= 1e-5 * float(np.max(np.abs(a) * cc))


def test_repeatable_and_stream_ordered(rick):
    """Two images of the same problem, the second on a side stream, agree to
    FP32 reordering (uncorrected images, so no taper amplification)."""
    prob = _to(synth.config1())
    im = rick.Imager(dict(prob["params"], flags=REAL))
    im.grid(prob["vis"], prob["u"], prob["v"], prob["w"], prob["wt"])
    a = im.image().clone()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        b = im.image()
    torch.cuda.synchronize()
    im.close()
    assert torch.max(torch.abs(a - b)).item() <= 1e-6 * torch.max(torch.abs(a)).item()


def test_image_host_matches_device_path(rick):
    prob = synth.config1()
    im = rick.Imager(dict(prob["params"], flags=REAL))
    a = im.image_host(prob["vis"], prob["u"], prob["v"], prob["w"], prob["wt"])
    g = _to(prob)
    im.reset()
    im.grid(g["vis"], g["u"], g["v"], g["w"], g["wt"])
    b = im.image().cpu()
    im.close()
    assert torch.max(torch.abs(a - b)).item() <= 1e-6 * torch.max(torch.abs(b)).item()


def test_pipelined_host_path_matches_synchronous(rick):
    """Five images of alternating problems (different data, the second with
    weights) through rick_image_host_async with two output buffers in
    flight, against rick_image_host one by one: the slot reuse and the event
    ordering between the copy streams and the compute stream hold."""
    probs = [synth.config1(), synth.disk_problem(256, 8, 60000, KB, 7, 2.0, 50.0, 99, weights="random")]
    probs = [dict(p, **{k: p[k].contiguous() for k in ("vis", "u", "v", "w", "wt")}) for p in probs]
    pinned = [{k: p[k].pin_memory() for k in ("vis", "u", "v", "w", "wt")} for p in probs]
    im = rick.Imager(dict(probs[0]["params"], flags=REAL))
    ref = [im.image_host(p["vis"], p["u"], p["v"], p["w"], p["wt"] if j else None).clone()
           for j, p in enumerate(pinned)]
    outs = [torch.empty((256, 256)).pin_memory() for _ in range(5)]
    for i in range(5):
        p = pinned[i % 2]
        im.image_host_async(p["vis"], p["u"], p["v"], p["w"], p["wt"] if i % 2 else None, out=outs[i])
    im.synchronize()
    im.close()
    for i in range(5):
        r = ref[i % 2]
        assert torch.max(torch.abs(outs[i] - r)).item() <= 1e-6 * torch.max(torch.abs(r)).item(), i


def test_errors_are_returned_not_raised_on_device(rick):
    prob = _to(synth.config1())
    im = rick.Imager(dict(prob["params"]))
    with pytest.raises(rick.RickError):
        im.grid_planes(5, 10)  # beyond nw
    with pytest.raises(ValueError):
        im.grid(prob["vis"].cpu(), prob["u"], prob["v"], prob["w"])
    huge = dict(prob["params"], n=32768, nw=4096, plane_group=4096)
    with pytest.raises(rick.RickError) as e:
        rick.Imager(huge)
    assert e.value.status == 2  # RICK_ERR_OOM before any launch
    im.close()


# ---------------------------------------------------- config 2, full size

@pytest.fixture(scope="module")
def config2_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return synth.config2(device="cuda")


def _lattice(n, side, extra=()):
    """side x side pixels spanning the image edge to edge, plus extras."""
    xs = np.unique(np.linspace(0, n - 1, side).round().astype(np.int64))
    pix = {(int(x), int(y)) for y in xs for x in xs} | {tuple(int(t) for t in e) for e in extra}
    return np.array(sorted(pix), np.int32)


def test_config2_full_size_sampled(rick, oracle_mod, config2_gpu):
    """4096^2, 32 planes, 1e7 Earth-rotation visibilities, KB support 7: in the
    bench's launch configuration (automatic tile and plane group), a 16 x 16
    pixel lattice spanning the image edge to edge (plus the phase centre and
    the brightest pixel) against the oracle's per-pixel evaluation, before
    the taper division (the grid-corrected image times c(x) c(y)) and from an
    imager without grid correction; and the gridded-sum invariant over all
    planes."""
    prob = config2_gpu
    params = dict(prob["params"], flags=CORRECT | REAL)
    im = rick.Imager(params)
    im.grid(prob["vis"], prob["u"], prob["v"], prob["w"], prob["wt"])
    img = im.image()
    st = im.stats()
    n = params["n"]
    flat = int(torch.argmax(img.abs()).item())
    pix = _lattice(n, 16, [(flat % n, flat // n), (n // 2, n // 2)])
    assert pix.shape[0] >= 256
    p = synth.to_numpy(prob)
    ref0 = oracle_mod.image_at(params, p["u"], p["v"], p["w"], p["wt"], p["vis"], pix, flags=0).real
    c = oracle_mod.taper(n, synth.KERNEL_KB, 7, 0.0)
    got = img.cpu().numpy()[pix[:, 1], pix[:, 0]] * c[pix[:, 0]] * c[pix[:, 1]]
    peak0 = np.max(np.abs(ref0))
    assert np.max(np.abs(got - ref0)) <= TOL * peak0
    uncorrected = rick.Imager(dict(prob["params"], flags=REAL))
    uncorrected.grid(prob["vis"], prob["u"], prob["v"], prob["w"], prob["wt"])
    img0 = uncorrected.image()
    got0 = img0.cpu().numpy()[pix[:, 1], pix[:, 0]]
    assert np.max(np.abs(got0 - ref0)) <= TOL * peak0
    assert st["n_dropped"] == 0 and st["n_gridded"] == prob["u"].numel()
    # Eq. 3 keeps the weighted visibility sum: over all planes
    tot = 0.0
    for k0 in range(0, params["nw"], 8):
        pl = im.grid_planes(k0, 8)
        tot += pl.to(torch.complex128).sum().item()
        del pl
    ref_sum = (prob["wt"].double() * prob["vis"].to(torch.complex128)).sum().item()
    assert abs(tot - ref_sum) <= 1e-5 * (prob["wt"].double() * prob["vis"].abs().double()).sum().item()
    im.close()
    uncorrected.close()
