"""w-support > 1 (Eq. 3's kernel in w) on the GPU against the FP64 oracle:
images (1e-4 of the peak; corrected images as c(x) c(y) D, as in every image
comparison), gridded planes (1e-5 of the largest cell), the adjoint (1e-4)
and prediction (1e-4), with plane groups that split measurements' w-footprints
between passes."""
import numpy as np
import pytest
import torch

import synth

pytestmark = pytest.mark.gpu

KB, GAUSS = synth.KERNEL_KB, synth.KERNEL_GAUSS
CORRECT, REAL, APPLY_N, UNIFORM = synth.FLAG_CORRECT, synth.FLAG_REAL, synth.FLAG_APPLY_N, synth.FLAG_UNIFORM


@pytest.fixture(scope="module")
def rick():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2504_00959_gb300 import build
    build.build()
    import paper_2504_00959_gb300 as r
    r.load()
    return r


def _problem(kernel, sw, nw=8, n=128, m=30000, wmax=200.0, seed=401):
    """Disk problem with the plane range padded by sw/2 planes each side."""
    prob = synth.disk_problem(n, nw, m, kernel, 7, 6.0, wmax, seed, fill=0.42, weights="random")
    half = wmax / (1.0 - (sw + 1.0) / nw)
    prob["params"] = dict(prob["params"], w_min=-half, w_max=half, w_support=sw)
    return prob


def _gpu(rick, prob, flags, **extra):
    g = {k: prob[k].cuda() for k in ("vis", "u", "v", "w", "wt")}
    im = rick.Imager(dict(prob["params"], flags=flags, **extra))
    im.grid(g["vis"], g["u"], g["v"], g["w"], g["wt"])
    return im, g


@pytest.mark.parametrize("kernel,sw,flags,extra", [
    (KB, 4, CORRECT | REAL, {}),
    (KB, 2, CORRECT | REAL, {"plane_group": 3}),
    (GAUSS, 3, CORRECT | APPLY_N, {"plane_group": 3}),
    (KB, 4, CORRECT | REAL | UNIFORM, {"tile": 16}),
    (KB, 5, REAL, {"plane_group": 2}),
])
def test_image_matches_oracle(rick, oracle_mod, kernel, sw, flags, extra):
    prob = _problem(kernel, sw)
    im, _ = _gpu(rick, prob, flags, **extra)
    got = im.image().cpu().numpy()
    im.close()
    p = synth.to_numpy(prob)
    q = p["params"]
    ref, _, _ = oracle_mod.dirty_image(q, p["u"], p["v"], p["w"], p["wt"], p["vis"], flags=flags & ~REAL)
    if flags & REAL:
        ref = ref.real
    if flags & CORRECT:
        c = oracle_mod.taper(q["n"], kernel, 7, 0.0)
        cc = np.outer(c, c)
    else:
        cc = np.ones((q["n"], q["n"]))
    err = np.max(np.abs(got - ref) * cc) / np.max(np.abs(ref) * cc)
    assert err <= 1e-4, err


def test_planes_match_oracle_grid(rick, oracle_mod):
    prob = _problem(KB, 4)
    im, _ = _gpu(rick, prob, REAL)
    planes = im.grid_planes().cpu().numpy()
    im.close()
    p = synth.to_numpy(prob)
    ref, _, _ = oracle_mod.grid(p["params"], p["u"], p["v"], p["w"], p["wt"], p["vis"])
    assert np.max(np.abs(planes - ref)) <= 1e-5 * np.max(np.abs(ref))


@pytest.mark.parametrize("sw,extra", [(3, {"plane_group": 2}), (4, {})])
def test_degrid_matches_oracle(rick, oracle_mod, sw, extra):
    prob = _problem(KB, sw, seed=403)
    flags = CORRECT | REAL
    im, g = _gpu(rick, prob, flags, **extra)
    im.image()
    n = prob["params"]["n"]
    r = np.random.default_rng(7).standard_normal((n, n)).astype(np.float32)
    got = im.degrid(torch.from_numpy(r).cuda(), g["u"], g["v"], g["w"], g["wt"]).cpu().numpy()
    im.close()
    p = synth.to_numpy(prob)
    ref = oracle_mod.degrid(p["params"], p["u"], p["v"], p["w"], p["wt"], p["vis"], r.astype(np.complex128),
                            flags=CORRECT)
    assert np.max(np.abs(got - ref)) <= 1e-4 * np.max(np.abs(ref))


def test_predict_matches_oracle(rick, oracle_mod):
    prob = _problem(KB, 4, seed=405)
    q = prob["params"]
    n = q["n"]
    c = oracle_mod.taper(n, KB, 7, 0.0)
    model = np.random.default_rng(8).standard_normal((n, n)) * np.outer(c, c)
    im = rick.Imager(dict(q, flags=CORRECT | REAL))
    got = im.predict(torch.from_numpy(model.astype(np.float32)).cuda(), prob["u"].cuda(), prob["v"].cuda(),
                     prob["w"].cuda()).cpu().numpy()
    im.close()
    p = synth.to_numpy(prob)
    ref = oracle_mod.predict(q, p["u"], p["v"], p["w"], model.astype(np.complex128), flags=CORRECT)
    assert np.max(np.abs(got - ref)) <= 1e-4 * np.max(np.abs(ref))


def test_dot_product(rick, oracle_mod):
    """<A x, y> = <x, A^H y> with w-support 4 across plane groups of 3."""
    prob = _problem(KB, 4, seed=407)
    q = prob["params"]
    n = q["n"]
    im = rick.Imager(dict(q, flags=CORRECT | REAL, plane_group=3))
    g = {k: prob[k].cuda() for k in ("u", "v", "w", "wt")}
    m = g["u"].numel()
    gen = torch.Generator().manual_seed(11)
    x = torch.complex(torch.randn(m, generator=gen), torch.randn(m, generator=gen)).cuda()
    c = torch.from_numpy(oracle_mod.taper(n, KB, 7, 0.0))
    y = (torch.randn((n, n), generator=gen, dtype=torch.float64) * torch.outer(c, c)).float().cuda()
    im.reset()
    im.grid(x, g["u"], g["v"], g["w"], g["wt"])
    Ax = im.image()
    AHy = im.degrid(y, g["u"], g["v"], g["w"], g["wt"])
    im.close()
    lhs = (Ax.double() * y.double()).sum().item()
    rhs = (x.to(torch.complex128).conj() * AHy.to(torch.complex128)).sum().real.item()
    assert abs(lhs - rhs) <= 1e-5 * abs(lhs), (lhs, rhs)


def test_refuses_planes_too_coarse_for_the_w_term(rick):
    """A wide field (dw (1 - n) at the corners far beyond the w-kernel's
    passband) would divide the image by ~0: creation fails instead."""
    p = synth.make_params(1024, 8, np.radians(20.0) / 1024, -6000.0, 6000.0, KB, 7)
    with pytest.raises(rick.RickError, match="passband"):
        rick.Imager(dict(p, w_support=4))
    rick.Imager(dict(p, nw=8, w_support=1)).close()  # nearest-plane stacking has no such division


def test_parameter_checks(rick):
    prob = _problem(KB, 4)
    with pytest.raises(rick.RickError):
        rick.Imager(dict(prob["params"], w_support=9))  # more than nw = 8
    with pytest.raises(rick.RickError):
        rick.BatchImager(dict(prob["params"], flags=REAL), [(-300.0, 300.0), (-200.0, 200.0)])
