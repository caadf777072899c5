"""The adjoint (degridder) on the GPU: against the oracle's adjoint, the
dot-product identity <A x, y> = <x, A^H y> (1e-5, inner products in FP64),
a dense-matrix check on a tiny problem, and central finite differences of
L = ||D(V) - t||^2 (accumulated in FP64) through the torch.autograd.Function
on 1000 random visibilities of the 4096^2 / 32-plane / 1e7 workload."""
import math

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


def _to(prob, dev="cuda"):
    return {k: (v.to(dev) if isinstance(v, torch.Tensor) else v) for k, v in prob.items()}


def _forward(im, g, vis):
    im.reset()
    im.grid(vis, g["u"], g["v"], g["w"], g["wt"])
    return im.image()


@pytest.mark.parametrize("flags,extra", [(CORRECT | REAL, {}), (CORRECT, {}), (REAL, {"plane_group": 3}),
                                         (CORRECT | REAL | APPLY_N | UNIFORM, {}),
                                         (CORRECT | REAL, {"tile": 16})])
def test_degrid_matches_oracle_adjoint(rick, oracle_mod, flags, extra):
    prob = synth.disk_problem(96, 7, 20000, KB, 7, 6.0, 120.0, 201, weights="random", fill=0.4)
    g = _to(prob)
    im = rick.Imager(dict(prob["params"], flags=flags, **extra))
    _forward(im, g, g["vis"])
    n = prob["params"]["n"]
    rng = np.random.default_rng(3)
    if flags & REAL:
        r = rng.standard_normal((n, n)).astype(np.float32)
        r_c = r.astype(np.complex128)
    else:
        r = (rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))).astype(np.complex64)
        r_c = r.astype(np.complex128)
    got = im.degrid(torch.from_numpy(r).cuda(), g["u"], g["v"], g["w"], g["wt"]).cpu().numpy()
    im.close()
    p = synth.to_numpy(prob)
    ref = oracle_mod.degrid(p["params"], p["u"], p["v"], p["w"], p["wt"], p["vis"], r_c, flags=flags & ~REAL)
    assert np.max(np.abs(got - ref)) <= 1e-4 * np.max(np.abs(ref))


def test_degrid_matches_oracle_with_hermitian_fold(rick, oracle_mod):
    """The adjoint of the folded imager: mirrored measurements get conjugated
    gradients (w-planes over [0, 120] for w in [-120, 120])."""
    prob = synth.disk_problem(96, 4, 20000, KB, 7, 6.0, 120.0, 203, weights="random", fill=0.4)
    prob["params"] = dict(prob["params"], w_min=0.0)
    flags = CORRECT | REAL | synth.FLAG_FOLD
    g = _to(prob)
    im = rick.Imager(dict(prob["params"], flags=flags))
    _forward(im, g, g["vis"])
    n = prob["params"]["n"]
    r = np.random.default_rng(5).standard_normal((n, n)).astype(np.float32)
    got = im.degrid(torch.from_numpy(r).cuda(), g["u"], g["v"], g["w"], g["wt"]).cpu().numpy()
    im.close()
    p = synth.to_numpy(prob)
    ref = oracle_mod.degrid(p["params"], p["u"], p["v"], p["w"], p["wt"], p["vis"], r.astype(np.complex128),
                            flags=flags & ~REAL)
    assert np.max(np.abs(got - ref)) <= 1e-4 * np.max(np.abs(ref))


def _dot_test(rick, oracle_mod, prob, flags, seed=7, **extra):
    """<A x, y> against <x, A^H y> for random x (complex) and y (real image).
    With grid correction the operator scales pixel (x, y) by 1/(c(x) c(y)),
    up to ~1e6 at the corners; y is then weighted by c(x) c(y) so that those
    pixels do not turn FP32 rounding of A x into the whole inner product (the
    correction is still applied, and differentiated, in both directions)."""
    g = _to(prob)
    im = rick.Imager(dict(prob["params"], flags=flags, **extra))
    m = g["u"].numel()
    q = prob["params"]
    n = q["n"]
    gen = torch.Generator().manual_seed(seed)
    x = torch.complex(torch.randn(m, generator=gen), torch.randn(m, generator=gen)).cuda()
    y = torch.randn((n, n), generator=gen, dtype=torch.float64)
    if flags & CORRECT:
        c = torch.from_numpy(oracle_mod.taper(n, q["kernel"], q["support"], q.get("kernel_param", 0.0)))
        y = y * torch.outer(c, c)
    y = y.float().cuda()
    Ax = _forward(im, g, x)
    AHy = im.degrid(y, g["u"], g["v"], g["w"], g["wt"])
    lhs = (Ax.double() * y.double()).sum().item()
    rhs = (x.to(torch.complex128).conj() * AHy.to(torch.complex128)).sum().real.item()
    im.close()
    return lhs, rhs


@pytest.mark.parametrize("flags,extra", [(CORRECT | REAL, {}), (REAL, {}),
                                         (CORRECT | REAL | UNIFORM | APPLY_N, {"plane_group": 3}),
                                         (CORRECT | REAL | synth.FLAG_FOLD, {"nw": 4, "w_min": 0.0})])
def test_dot_product_config1(rick, oracle_mod, flags, extra):
    lhs, rhs = _dot_test(rick, oracle_mod, synth.config1(), flags, **extra)
    assert abs(lhs - rhs) <= 1e-5 * abs(lhs), (lhs, rhs)


def test_dense_matrix_tiny(rick):
    """A built column by column from unit visibilities with the GPU forward;
    the GPU adjoint must equal A^T y (real image)."""
    prob = synth.disk_problem(16, 2, 6, KB, 3, 20.0, 40.0, 211, fill=0.3)
    g = _to(prob)
    im = rick.Imager(dict(prob["params"], flags=CORRECT | REAL))
    m = 6
    cols = []
    for j in range(m):
        e = torch.zeros(m, dtype=torch.complex64, device="cuda")
        e[j] = 1.0
        re = _forward(im, g, e).double().flatten()
        e[j] = 1.0j
        imv = _forward(im, g, e).double().flatten()
        cols.append(torch.complex(re, -imv))  # d Re D / d Re V_j  and  d Re D / d Im V_j
    y = torch.randn(16 * 16, dtype=torch.float64, device="cuda")
    ref = torch.stack([(c * y).sum() for c in cols])  # grad_V = dD/dReV . y + i dD/dImV . y
    _forward(im, g, g["vis"])
    got = im.degrid(y.float().reshape(16, 16), g["u"], g["v"], g["w"], g["wt"]).to(torch.complex128)
    im.close()
    ref = torch.complex(ref.real, -ref.imag)
    assert torch.max(torch.abs(got - ref)).item() <= 1e-5 * torch.max(torch.abs(ref)).item()


# ------------------------------------------------- config 5 (full size)

@pytest.fixture(scope="module")
def config5():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    prob = synth.config2(device="cuda")
    sky = prob["sky"]
    gen = torch.Generator().manual_seed(synth.BASE_SEED + 5)
    flux_t = sky["flux"] * (1.0 + 0.1 * torch.randn(sky["flux"].shape[0], generator=gen, dtype=torch.float64))
    u, v, w = (prob[k].double() for k in ("u", "v", "w"))
    vis_t = synth.predict_point_sources(u, v, w, sky["l"], sky["m"], flux_t)
    return prob, vis_t


def test_dot_product_config5_full(rick, oracle_mod, config5):
    prob, _ = config5
    lhs, rhs = _dot_test(rick, oracle_mod, prob, CORRECT | REAL)
    assert abs(lhs - rhs) <= 1e-5 * abs(lhs), (lhs, rhs)


def test_finite_differences_config5(rick, config5):
    prob, vis_t = config5
    params = dict(prob["params"], flags=CORRECT | REAL)
    im = rick.Imager(params)
    g = prob
    with torch.no_grad():
        t = _forward(im, g, vis_t).double().clone()
    vis = g["vis"].clone().requires_grad_(True)
    D = rick.dirty_image(vis, g["u"], g["v"], g["w"], g["wt"], im)
    L = ((D.double() - t) ** 2).sum()
    L.backward()
    grad = vis.grad.detach().to(torch.complex128)
    m = g["u"].numel()
    gen = torch.Generator().manual_seed(99)
    idx = torch.randperm(m, generator=gen)[:1000].tolist()
    rms = torch.sqrt((g["vis"].abs() ** 2).mean()).item()
    h = 100.0 * rms

    def loss(vv):
        with torch.no_grad():
            return ((_forward(im, g, vv).double() - t) ** 2).sum().item()

    errs, scale = [], torch.max(torch.abs(grad[idx])).item()
    base = g["vis"].clone()
    for i in idx:
        for part in (1.0, 1.0j):
            vp = base.clone()
            vm = base.clone()
            vp[i] = base[i] + h * part
            vm[i] = base[i] - h * part
            step = (complex(vp[i].item()) - complex(vm[i].item())) / (2 * part)  # exact binary32 step
            fd = (loss(vp) - loss(vm)) / (2 * step.real)
            an = grad[i].real.item() if part == 1.0 else grad[i].imag.item()
            errs.append(abs(fd - an))
    im.close()
    assert max(errs) <= 1e-3 * scale, (max(errs), scale)
