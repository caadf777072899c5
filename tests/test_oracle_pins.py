"""Pins of the FP64 oracle against things other than itself (CPU only).

Each test checks the oracle against a library routine, a closed form, an
invariant of the method, or the brute-force direct DFT with the exact w-term
(Eq. 1), chosen so that a dropped term, a wrong sign or index, a transposed
operand or a wrong normalisation fails at least one of them.
"""
import math

import numpy as np
import pytest
import scipy.special as sp

import synth

KB, GAUSS = synth.KERNEL_KB, synth.KERNEL_GAUSS
CORRECT, APPLY_N, UNIFORM = synth.FLAG_CORRECT, synth.FLAG_APPLY_N, synth.FLAG_UNIFORM


def _np(prob):
    return synth.to_numpy(prob)


def _small(n=64, nw=4, m=2000, kernel=KB, support=8, fov=2.0, wmax=50.0, seed=7, **kw):
    return _np(synth.disk_problem(n, nw, m, kernel, support, fov, wmax, seed, **kw))


def _args(p):
    return (p["params"], p["u"], p["v"], p["w"], p["wt"], p["vis"])


def _away_from_decisions(p, margin=2e-3):
    """Mask of measurements whose placement is far from every binary32 decision
    boundary, so that definitions evaluated in FP64 must agree with them."""
    q = p["params"]
    n, S = q["n"], q["support"]
    s = n * q["pixel_rad"]
    pu = p["u"].astype(np.float64) * s + n / 2
    pv = p["v"].astype(np.float64) * s + n / 2
    fu = (pu - S / 2) - np.floor(pu - S / 2)
    fv = (pv - S / 2) - np.floor(pv - S / 2)
    ok = (fu > margin) & (fu < 1 - margin) & (fv > margin) & (fv < 1 - margin)
    if q["nw"] > 1:
        dw = (q["w_max"] - q["w_min"]) / q["nw"]
        t = (p["w"].astype(np.float64) - q["w_min"]) / dw
        ft = t - np.floor(t)
        ok &= (ft > margin) & (ft < 1 - margin)
    return ok


def _subset(p, mask):
    return dict(params=dict(p["params"]), u=p["u"][mask].copy(), v=p["v"][mask].copy(),
                w=p["w"][mask].copy(), wt=p["wt"][mask].copy(), vis=p["vis"][mask].copy())


# --------------------------------------------------------------------------
# building blocks against libraries and closed forms
# --------------------------------------------------------------------------

@pytest.mark.parametrize("n", [1, 2, 8, 64, 1024, 6, 12, 200])
@pytest.mark.parametrize("sign", [+1, -1])
def test_fft_matches_numpy(oracle_mod, n, sign):
    rng = np.random.default_rng(n)
    x = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    ref = np.fft.ifft(x) * n if sign > 0 else np.fft.fft(x)
    got = oracle_mod.fft(x, sign)
    assert np.max(np.abs(got - ref)) <= 1e-12 * max(1.0, np.max(np.abs(ref)))


@pytest.mark.parametrize("n", [8, 64, 12])
def test_plane_transform_definition(oracle_mod, n):
    """P[y,x] = sum G[jv,ju] exp(+2 pi i ((ju-n/2)(x-n/2) + (jv-n/2)(y-n/2)) / n),
    written out as a dense matrix product, and numpy's shifted ifft2."""
    rng = np.random.default_rng(3 + n)
    G = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    j = np.arange(n) - n // 2
    E = np.exp(2j * np.pi * np.outer(j, j) / n)  # E[x, ju]
    ref = E @ G @ E.T                            # rows: y, cols: x
    got = oracle_mod.plane_image(G, +1)
    assert np.max(np.abs(got - ref)) <= 1e-11 * np.max(np.abs(ref))
    ref_np = np.fft.fftshift(np.fft.ifft2(np.fft.ifftshift(G))) * n * n
    assert np.max(np.abs(got - ref_np)) <= 1e-11 * np.max(np.abs(ref))
    adj = oracle_mod.plane_image(G, -1)
    assert np.max(np.abs(adj - E.conj() @ G @ E.conj().T)) <= 1e-11 * np.max(np.abs(ref))


def test_bessel_i0_matches_scipy(oracle_mod):
    for x in np.concatenate([np.linspace(0, 5, 51), np.linspace(5, 45, 41)]):
        ref = sp.i0(x)
        assert abs(oracle_mod.bessel_i0(x) - ref) <= 1e-13 * ref


@pytest.mark.parametrize("support", [4, 7, 8])
def test_kernel_definitions(oracle_mod, support):
    xs = np.linspace(-support / 2, support / 2, 37)
    sigma = support / 6.0
    beta = 2.34 * support
    for x in xs:
        g = oracle_mod.kernel_value(GAUSS, support, 0.0, x)
        assert abs(g - math.exp(-x * x / (2 * sigma * sigma))) <= 1e-15
        k = oracle_mod.kernel_value(KB, support, 0.0, x)
        ref = sp.i0(beta * math.sqrt(max(0.0, 1 - (2 * x / support) ** 2)))
        assert abs(k - ref) <= 1e-13 * ref
    # explicit parameters override the defaults
    assert abs(oracle_mod.kernel_value(GAUSS, support, 2.0, 1.0) - math.exp(-1 / 8)) < 1e-15


def kb_taper(n, support, beta):
    """Closed-form Fourier transform of the Kaiser-Bessel window over
    [-S/2, S/2], normalised to 1 at the centre (S sinh(sqrt(b^2 - (pi S xi)^2)) /
    sqrt(...), with sin for the oscillating branch)."""
    xi = (np.arange(n) - n // 2) / n
    a = beta ** 2 - (np.pi * support * xi) ** 2
    out = np.empty(n)
    pos, neg = a > 0, a < 0
    out[pos] = np.sinh(np.sqrt(a[pos])) / np.sqrt(a[pos])
    out[neg] = np.sin(np.sqrt(-a[neg])) / np.sqrt(-a[neg])
    out[a == 0] = 1.0
    return out / (np.sinh(beta) / beta)


def gauss_taper(n, support, sigma):
    """Closed-form Fourier transform of the Gaussian truncated to [-S/2, S/2]
    (complex error functions), normalised to 1 at the centre."""
    xi = (np.arange(n) - n // 2) / n
    a = support / 2
    c = 2j * np.pi * sigma ** 2 * xi
    s2 = sigma * math.sqrt(2)
    val = np.exp(-2 * np.pi ** 2 * sigma ** 2 * xi ** 2) * (sp.erf((a - c) / s2) + sp.erf((a + c) / s2))
    return np.real(val) / (2 * sp.erf(a / s2))


@pytest.mark.parametrize("support", [5, 7, 8])
def test_taper_closed_forms(oracle_mod, support):
    n = 128
    got = oracle_mod.taper(n, KB, support, 0.0)
    assert np.max(np.abs(got - kb_taper(n, support, 2.34 * support))) < 1e-9
    got = oracle_mod.taper(n, GAUSS, support, 0.0)
    assert np.max(np.abs(got - gauss_taper(n, support, support / 6))) < 1e-9
    assert abs(got[n // 2] - 1.0) < 1e-14


def test_placement_matches_definition(oracle_mod):
    """Plane = floor((w - w_min) / dw) clamped, first cell = floor(p - S/2) + 1,
    footprint inside the grid, checked away from binary32 decision boundaries."""
    p = _small(n=128, nw=8, m=20000, support=7, wmax=60.0, fill=0.5, seed=11)
    ok = _away_from_decisions(p)
    q = p["params"]
    k, fu, fv = oracle_mod.place(q, p["u"], p["v"], p["w"])
    n, S = q["n"], q["support"]
    pu = p["u"].astype(np.float64) * n * q["pixel_rad"] + n / 2
    pv = p["v"].astype(np.float64) * n * q["pixel_rad"] + n / 2
    efu = np.floor(pu - S / 2).astype(np.int64) + 1
    efv = np.floor(pv - S / 2).astype(np.int64) + 1
    dw = (q["w_max"] - q["w_min"]) / q["nw"]
    ek = np.clip(np.floor((p["w"].astype(np.float64) - q["w_min"]) / dw), 0, q["nw"] - 1)
    inside = (efu >= 0) & (efu + S <= n) & (efv >= 0) & (efv + S <= n)
    assert np.all((k[ok] >= 0) == inside[ok])
    sel = ok & inside
    assert sel.sum() > 10000 and (~inside).sum() > 100
    assert np.array_equal(k[sel], ek[sel])
    assert np.array_equal(fu[sel], efu[sel]) and np.array_equal(fv[sel], efv[sel])


# --------------------------------------------------------------------------
# special cases and invariants of the method
# --------------------------------------------------------------------------

def test_delta_kernel_equals_numpy_ifft2(oracle_mod):
    """Nw = 1, w = 0, support 1 and integer-cell u, v: the image is numpy's
    shifted ifft2 of the summed cells times n^2, over the weight sum."""
    n, m = 64, 3000
    rng = np.random.default_rng(5)
    ju = rng.integers(0, n, m)
    jv = rng.integers(0, n, m)
    params = synth.make_params(n, 1, 1.0 / n, 0.0, 0.0, GAUSS, 1, 0.0, 0)
    u = (ju - n // 2).astype(np.float32)
    v = (jv - n // 2).astype(np.float32)
    w = np.zeros(m, np.float32)
    wt = rng.uniform(0.5, 2.0, m).astype(np.float32)
    vis = (rng.standard_normal(m) + 1j * rng.standard_normal(m)).astype(np.complex64)
    img, sw, dropped = oracle_mod.dirty_image(params, u, v, w, wt, vis)
    assert dropped == 0
    G = np.zeros((n, n), np.complex128)
    np.add.at(G, (jv, ju), wt.astype(np.float64) * vis.astype(np.complex128))
    ref = np.fft.fftshift(np.fft.ifft2(np.fft.ifftshift(G))) * n * n / wt.astype(np.float64).sum()
    assert abs(sw - wt.astype(np.float64).sum()) < 1e-9
    assert np.max(np.abs(img - ref)) <= 1e-12 * np.max(np.abs(ref))


@pytest.mark.parametrize("kernel,support", [(GAUSS, 7), (KB, 7), (KB, 8)])
@pytest.mark.parametrize("flags", [0, CORRECT, CORRECT | APPLY_N])
def test_point_source_at_phase_centre(oracle_mod, kernel, support, flags):
    p = _small(n=64, nw=6, m=3000, kernel=kernel, support=support, seed=21)
    p["vis"] = np.ones_like(p["vis"])
    img, sw, _ = oracle_mod.dirty_image(*_args(p), flags=flags)
    assert abs(img[32, 32] - 1.0) < 1e-12
    a = np.abs(img)
    if flags == 0:
        assert a.max() <= 1.0 + 1e-12
        assert np.unravel_index(np.argmax(a), a.shape) == (32, 32)


def test_grid_sum_equals_weighted_visibility_sum(oracle_mod):
    p = _small(n=64, nw=5, m=4000, kernel=KB, support=7, seed=23, weights="random", fill=0.4)
    planes, sw, dropped = oracle_mod.grid(*_args(p))
    ref = np.sum(p["wt"].astype(np.float64) * p["vis"].astype(np.complex128))
    assert dropped == 0
    assert abs(planes.sum() - ref) <= 1e-12 * np.sum(np.abs(p["vis"]) * p["wt"])
    assert abs(sw - p["wt"].astype(np.float64).sum()) < 1e-9


def test_dropped_measurements(oracle_mod):
    """Out-of-grid and non-finite measurements are dropped and counted, and
    leave the image exactly as without them."""
    p = _small(n=64, nw=4, m=1000, support=7, seed=29)
    q = dict(p)
    extra_u = np.array([1e9, np.nan, 0.0, 0.0, -1e30], np.float32)
    extra_v = np.array([0.0, 0.0, np.inf, 0.0, 0.0], np.float32)
    extra_w = np.array([0.0, 0.0, 0.0, np.nan, 0.0], np.float32)
    q = dict(params=p["params"], u=np.concatenate([p["u"], extra_u]), v=np.concatenate([p["v"], extra_v]),
             w=np.concatenate([p["w"], extra_w]), wt=np.concatenate([p["wt"], np.ones(5, np.float32)]),
             vis=np.concatenate([p["vis"], np.ones(5, np.complex64)]))
    a, swa, da = oracle_mod.dirty_image(*_args(p))
    b, swb, db = oracle_mod.dirty_image(*_args(q))
    assert da == 0 and db == 5 and swa == swb
    assert np.array_equal(a, b)


def test_hermitian_completion_gives_twice_real_part(oracle_mod):
    """Gridding (u,v,w,V) together with (-u,-v,-w,V*) (w-planes symmetric about
    0) images to 2 Re of the one-sided image, with zero imaginary part."""
    # fill 0.4 keeps every footprint off column/row 0, whose mirror (cell n)
    # lies outside the grid
    p = _small(n=64, nw=6, m=3000, kernel=KB, support=7, wmax=80.0, seed=31, fov=6.0, fill=0.4)
    p = _subset(p, _away_from_decisions(p))
    img, sw, _ = oracle_mod.dirty_image(*_args(p), flags=0)
    h = dict(params=p["params"], u=np.concatenate([p["u"], -p["u"]]), v=np.concatenate([p["v"], -p["v"]]),
             w=np.concatenate([p["w"], -p["w"]]), wt=np.concatenate([p["wt"], p["wt"]]),
             vis=np.concatenate([p["vis"], np.conj(p["vis"])]))
    full, sw2, _ = oracle_mod.dirty_image(*_args(h), flags=0)
    peak = np.max(np.abs(full))
    assert np.max(np.abs(full.imag)) <= 1e-12 * peak
    assert np.max(np.abs(full - np.real(img))) <= 1e-12 * peak  # 2 Re(img) / 2 (weight sum doubles)


def test_hermitian_fold_keeps_the_real_image(oracle_mod):
    """Folding (w < 0 -> (-u, -v, -w, V*)) onto nw planes over [0, W] gives the
    real image of the unfolded measurements on 2 nw planes over [-W, W] (their
    plane centres mirror each other), while the imaginary part changes."""
    p = _small(n=64, nw=8, m=3000, kernel=KB, support=7, wmax=80.0, seed=33, fov=6.0, fill=0.4)
    p = _subset(p, _away_from_decisions(p))
    assert np.any(p["w"] < 0) and np.any(p["w"] > 0)
    whole, _, _ = oracle_mod.dirty_image(*_args(p), flags=CORRECT)
    q = dict(p, params=dict(p["params"], nw=4, w_min=0.0, w_max=p["params"]["w_max"]))
    folded, _, _ = oracle_mod.dirty_image(*_args(q), flags=CORRECT | synth.FLAG_FOLD)
    peak = np.max(np.abs(whole.real))
    assert np.max(np.abs(folded.real - whole.real)) <= 1e-12 * peak
    assert np.max(np.abs(folded.imag - whole.imag)) >= 1e-3 * peak


def test_hermitian_fold_adjoint_dot_product(oracle_mod):
    """With the fold the imager is real-linear (mirrored measurements enter as
    V*): sum_pix r Re(A x) = Re <A^H r, x> for real r, where the degridder
    conjugates the gradients of mirrored measurements."""
    p = _small(n=32, nw=2, m=700, support=7, seed=59, weights="random", fov=8.0, wmax=90.0)
    q = dict(p["params"], w_min=0.0, w_max=90.0)
    rng = np.random.default_rng(3)
    m = p["u"].shape[0]
    x = (rng.standard_normal(m) + 1j * rng.standard_normal(m)).astype(np.complex64)
    r = rng.standard_normal((32, 32))
    flags = CORRECT | synth.FLAG_FOLD
    Ax, _, _ = oracle_mod.dirty_image(q, p["u"], p["v"], p["w"], p["wt"], x, flags=flags)
    g = oracle_mod.degrid(q, p["u"], p["v"], p["w"], p["wt"], x, r.astype(np.complex128), flags=flags)
    lhs = float(np.sum(r * Ax.real))
    rhs = float(np.real(np.vdot(g, x.astype(np.complex128))))
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)
    # without the conjugation of mirrored gradients the identity fails
    g0 = oracle_mod.degrid(q, p["u"], p["v"], p["w"], p["wt"], x, r.astype(np.complex128), flags=flags)
    neg = p["w"] < 0
    g0[neg] = np.conj(g0[neg])
    assert abs(lhs - float(np.real(np.vdot(g0, x.astype(np.complex128))))) >= 1e-6 * abs(lhs)


def test_linearity(oracle_mod):
    p = _small(n=32, nw=3, m=800, support=7, seed=37)
    rng = np.random.default_rng(1)
    v2 = (rng.standard_normal(p["vis"].shape[0]) + 1j * rng.standard_normal(p["vis"].shape[0]))
    a, b = 0.7 - 0.2j, -1.3 + 0.5j
    va = p["vis"].astype(np.complex128)
    comb = (a * va + b * v2).astype(np.complex64)
    i1, _, _ = oracle_mod.dirty_image(p["params"], p["u"], p["v"], p["w"], p["wt"], p["vis"])
    i2, _, _ = oracle_mod.dirty_image(p["params"], p["u"], p["v"], p["w"], p["wt"], v2.astype(np.complex64))
    i3, _, _ = oracle_mod.dirty_image(p["params"], p["u"], p["v"], p["w"], p["wt"], comb)
    ref = a * i1 + b * i2
    assert np.max(np.abs(i3 - ref)) <= 1e-6 * np.max(np.abs(ref))  # complex64 rounding of comb


@pytest.mark.parametrize("kernel,support", [(KB, 7), (KB, 8), (GAUSS, 7)])
@pytest.mark.parametrize("flags", [0, CORRECT | APPLY_N])
def test_single_visibility_closed_form(oracle_mod, kernel, support, flags):
    """One measurement images to a separable sum of its normalised taps times
    the plane's phase screen; every factor is written out here from the
    definitions (scipy's I0, the kernel formulas, the plane centre w_k)."""
    n, nw = 32, 5
    pixel_rad = math.radians(12.0) / n
    du = 1.0 / (n * pixel_rad)
    u, v, w = np.float32(3.37 * du), np.float32(-5.81 * du), np.float32(23.7)
    params = synth.make_params(n, nw, pixel_rad, -40.0, 40.0, kernel, support, 0.0, flags)
    img, sw, _ = oracle_mod.dirty_image(params, np.array([u]), np.array([v]), np.array([w]),
                                        np.array([1.5], np.float32), np.array([0.8 - 0.3j], np.complex64))

    def g(x):
        if kernel == GAUSS:
            s = support / 6
            return np.exp(-x * x / (2 * s * s))
        return sp.i0(2.34 * support * np.sqrt(np.maximum(0.0, 1 - (2 * x / support) ** 2)))

    def axis(c):
        p = float(c) * n * pixel_rad + n / 2
        f = math.floor(p - support / 2) + 1
        t = np.arange(support)
        taps = g(f + t - p)
        taps = taps / taps.sum()
        x = np.arange(n)
        return (taps[None, :] * np.exp(2j * np.pi * np.outer(x - n // 2, f + t - n // 2) / n)).sum(1)

    dw = 80.0 / nw
    k = int(math.floor((float(w) + 40.0) / dw))
    wk = -40.0 + (k + 0.5) * dw
    l = (np.arange(n) - n // 2) * pixel_rad
    L, M = np.meshgrid(l, l)  # L[y, x] = l(x), M[y, x] = m(y)
    r2 = L * L + M * M
    nm1 = -r2 / (1 + np.sqrt(1 - r2))
    ref = complex(np.complex64(0.8 - 0.3j)) * np.outer(axis(v), axis(u)) * np.exp(2j * np.pi * wk * nm1)
    if flags & CORRECT:
        t = kb_taper(n, support, 2.34 * support) if kernel == KB else gauss_taper(n, support, support / 6)
        ref = ref / np.outer(t, t)
    if flags & APPLY_N:
        ref = ref * (1 + nm1)
    assert abs(sw - 1.5) < 1e-12
    assert np.max(np.abs(img - ref)) <= 1e-9 * np.max(np.abs(ref))


def test_uniform_weighting(oracle_mod):
    """Uniform weighting with unit weights: each measurement weighs 1 / (number
    of gridded measurements sharing its nearest cell), so the weight sum is
    the number of occupied cells and the grid sum is sum V / count."""
    p = _small(n=32, nw=3, m=6000, support=7, seed=41, fill=0.35)
    q = p["params"]
    n = q["n"]
    # nearest cell computed in FP64; measurements within 1e-4 of a half cell,
    # where the binary32 decision could differ, are removed from the problem
    pu = p["u"].astype(np.float64) * n * q["pixel_rad"] + n / 2
    pv = p["v"].astype(np.float64) * n * q["pixel_rad"] + n / 2
    keep = (np.abs(pu + 0.5 - np.round(pu + 0.5)) > 1e-4) & (np.abs(pv + 0.5 - np.round(pv + 0.5)) > 1e-4)
    p = _subset(p, keep)
    pu, pv = pu[keep], pv[keep]
    planes, sw, dropped = oracle_mod.grid(*_args(p), flags=UNIFORM)
    assert dropped == 0
    cu = np.floor(pu + 0.5).astype(np.int64)
    cv = np.floor(pv + 0.5).astype(np.int64)
    cells = cv * n + cu
    uniq, inv, counts = np.unique(cells, return_inverse=True, return_counts=True)
    assert abs(sw - len(uniq)) < 1e-9
    ref = np.sum(p["vis"].astype(np.complex128) / counts[inv])
    assert abs(planes.sum() - ref) < 1e-9 * np.sum(np.abs(p["vis"]))


# --------------------------------------------------------------------------
# against the direct DFT with the exact w-term (Eq. 1)
# --------------------------------------------------------------------------

def _alias_bound(kernel, support, kparam, xi_max, taper_fn):
    """max over the measurement's sub-cell offset and |xi| <= xi_max of
    |sum_t g_t e^{2 pi i x_t xi} / c(xi) - 1| for normalised taps: the 1D
    relative error of gridding + grid correction against the exact phase."""
    xi = np.linspace(-xi_max, xi_max, 257)
    n = 4096
    c_full = taper_fn(n)
    c = np.interp(xi, (np.arange(n) - n // 2) / n, c_full)
    worst = 0.0
    for phi in np.linspace(0, 1, 1001, endpoint=False):
        p = 100.0 + phi
        f = math.floor(p - support / 2) + 1
        x = f + np.arange(support) - p
        if kernel == GAUSS:
            g = np.exp(-x * x / (2 * kparam * kparam))
        else:
            g = sp.i0(kparam * np.sqrt(np.maximum(0.0, 1 - (2 * x / support) ** 2)))
        g = g / g.sum()
        gd = (g[None, :] * np.exp(2j * np.pi * np.outer(xi, x))).sum(1)
        worst = max(worst, np.max(np.abs(gd / c - 1)))
    return worst * 1.02


def _dft_problem(nw, seed=43, n=64, m=1500, wmax=150.0, fov=10.0, support=8):
    """Three point sources inside the central half of a 10 degree field,
    visibilities from Eq. 2 (coherent, so w errors do not average away)."""
    p = _small(n=n, nw=nw, m=m, kernel=KB, support=support, fov=fov, wmax=wmax, seed=seed)
    q = p["params"]
    dl = q["pixel_rad"]
    src = [(9, -7, 1.0), (-12, 4, 0.6), (3, 14, 0.8)]
    u = p["u"].astype(np.float64)
    v = p["v"].astype(np.float64)
    w = p["w"].astype(np.float64)
    vis = np.zeros(u.shape[0], np.complex128)
    for (ix, iy, fl) in src:
        l, mm = ix * dl, iy * dl
        r2 = l * l + mm * mm
        nm1 = -r2 / (1 + math.sqrt(1 - r2))
        vis += fl * np.exp(-2j * np.pi * (u * l + v * mm + w * nm1))
    p["vis"] = vis.astype(np.complex64)
    return p, src


def test_against_direct_dft_with_exact_w_term(oracle_mod):
    """w-stacking with grid correction vs the brute-force DFT with the exact
    w-term over the central half of the image.  Bound derived from the method:
    per measurement, the relative error is at most (1+e_a)^2 - 1 from gridding
    (e_a the 1D bound above) plus (1+e_a)^2 * 2 pi (dw/2) |n-1| from snapping w
    to the plane centre."""
    nw = 32
    p, src = _dft_problem(nw)
    q = p["params"]
    n, S = q["n"], q["support"]
    beta = 2.34 * S
    xs = np.arange(n // 4, 3 * n // 4)
    pix = np.array([(x, y) for y in xs for x in xs], np.int32)
    ws = oracle_mod.image_at(*_args(p), pix, flags=CORRECT)
    img, sw, _ = oracle_mod.dirty_image(*_args(p), flags=CORRECT)
    assert np.max(np.abs(ws - img[pix[:, 1], pix[:, 0]])) < 1e-10 * np.max(np.abs(img))
    ref = oracle_mod.dft(*_args(p), pix, flags=CORRECT)
    e_a = _alias_bound(KB, S, beta, 0.25, lambda nn: kb_taper(nn, S, beta))
    dl = q["pixel_rad"]
    l = (pix[:, 0] - n // 2) * dl
    mm = (pix[:, 1] - n // 2) * dl
    r2 = l * l + mm * mm
    nm1 = np.abs(-r2 / (1 + np.sqrt(1 - r2)))
    dw = (q["w_max"] - q["w_min"]) / nw
    amp = np.sum(np.abs(p["vis"].astype(np.complex128)) * p["wt"]) / sw
    bound = amp * (((1 + e_a) ** 2 - 1) + (1 + e_a) ** 2 * 2 * np.pi * (dw / 2) * nm1)
    err = np.abs(ws - ref)
    assert np.all(err <= bound), (err.max(), bound.min())
    # the pixels of the sources carry the fluxes
    for (ix, iy, fl) in src:
        i = np.flatnonzero((pix[:, 0] == n // 2 + ix) & (pix[:, 1] == n // 2 + iy))[0]
        assert abs(ref[i].real - fl) < 0.1
        assert abs(ws[i] - ref[i]) < 0.02 * fl


@pytest.mark.parametrize("fold", [False, True])
def test_predict_against_measurement_equation(oracle_mod, fold):
    """Prediction of a model of three point-source pixels against Eq. 2 evaluated
    directly per measurement, within the bound of the imaging pin: per axis
    gridding + grid correction (e_a), plus the phase error of snapping w to
    the plane centre.  With the Hermitian fold (the model is real) on half the
    planes over [0, W] the same bound holds."""
    nw = 32
    p, src = _dft_problem(nw)
    q = dict(p["params"])
    if fold:
        q = dict(q, nw=nw // 2, w_min=0.0)
    n, S = q["n"], q["support"]
    dl = q["pixel_rad"]
    model = np.zeros((n, n), np.complex128)
    for (ix, iy, fl) in src:
        model[n // 2 + iy, n // 2 + ix] = fl
    flags = CORRECT | (synth.FLAG_FOLD if fold else 0)
    got = oracle_mod.predict(q, p["u"], p["v"], p["w"], model, flags=flags)
    u, v, w = (p[k].astype(np.float64) for k in ("u", "v", "w"))
    ref = np.zeros(u.shape[0], np.complex128)
    bound = np.zeros(u.shape[0])
    e_a = _alias_bound(KB, S, 2.34 * S, 0.25, lambda nn: kb_taper(nn, S, 2.34 * S))
    dw = (q["w_max"] - q["w_min"]) / q["nw"]
    for (ix, iy, fl) in src:
        l, mm = ix * dl, iy * dl
        nm1 = -(l * l + mm * mm) / (1 + math.sqrt(1 - l * l - mm * mm))
        ref += fl * np.exp(-2j * np.pi * (u * l + v * mm + w * nm1))
        bound += fl * (((1 + e_a) ** 2 - 1) + (1 + e_a) ** 2 * 2 * np.pi * (dw / 2) * abs(nm1))
    sgn = np.where(p["w"] < 0, -1.0, 1.0).astype(np.float32) if fold else np.ones_like(p["w"])
    placed = oracle_mod.place(q, sgn * p["u"], sgn * p["v"], sgn * p["w"])[0] >= 0
    assert np.all(got[~placed] == 0)  # footprints off the grid: no prediction
    err = np.abs(got - ref)[placed]
    assert np.all(err <= bound[placed]), (err.max(), bound.min())


def test_w_error_shrinks_with_more_planes(oracle_mod):
    """The w-quantisation error at a source falls as planes are added (the
    coherent error scales like dw^2), down to the gridding floor."""
    errs = []
    for nw in (4, 8, 16):
        p, src = _dft_problem(nw, seed=47, wmax=400.0)
        n = p["params"]["n"]
        pix = np.array([(n // 2 + ix, n // 2 + iy) for (ix, iy, _) in src], np.int32)
        ws = oracle_mod.image_at(*_args(p), pix, flags=CORRECT)
        ref = oracle_mod.dft(*_args(p), pix, flags=CORRECT)
        errs.append(np.max(np.abs(ws - ref)))
    assert errs[1] < errs[0] / 2.5 and errs[2] < errs[1] / 2.5, errs


def _kb_ft(xi, support, beta):
    """Closed-form Fourier transform of the Kaiser-Bessel window over
    [-S/2, S/2] at frequency xi (cycles per unit), normalised to 1 at 0."""
    a = beta ** 2 - (np.pi * support * np.asarray(xi, dtype=np.float64)) ** 2
    out = np.ones_like(a)
    pos, neg = a > 0, a < 0
    out[pos] = np.sinh(np.sqrt(a[pos])) / np.sqrt(a[pos])
    out[neg] = np.sin(np.sqrt(-a[neg])) / np.sqrt(-a[neg])
    out[a == 0] = 1.0
    return out / (np.sinh(beta) / beta)


def _w_alias_bound(sw, xi_max):
    """max over the measurement's sub-plane offset and |xi| <= xi_max of
    |sum_t h_t e^{2 pi i x_t xi} / h^(xi) - 1| for the normalised KB w-taps of
    support sw: the relative error of gridding in w + correction in w."""
    beta = 2.34 * sw
    xi = np.linspace(-xi_max, xi_max, 129)
    worst = 0.0
    for phi in np.linspace(0, 1, 401, endpoint=False):
        pw = 50.0 + phi
        fk = math.floor(pw - sw / 2) + 1
        x = fk + np.arange(sw) - pw
        h = sp.i0(beta * np.sqrt(np.maximum(0.0, 1 - (2 * x / sw) ** 2)))
        h = h / h.sum()
        hd = (h[None, :] * np.exp(2j * np.pi * np.outer(xi, x))).sum(1)
        worst = max(worst, np.max(np.abs(hd / _kb_ft(xi, sw, beta) - 1)))
    return worst * 1.02


def _padded_w(q, sw, wmax):
    """Plane range of nw planes padded by sw/2 planes each side of [-wmax, wmax],
    so every measurement's w-footprint lies on the planes."""
    nw = q["nw"]
    half = wmax / (1.0 - (sw + 1.0) / nw)
    return dict(q, w_min=-half, w_max=half, w_support=sw)


def test_w_gridding_against_direct_dft(oracle_mod):
    """Eq. 3's kernel in w (w-support 4 on 16 planes): against the direct DFT
    with the exact w-term over the central half, within the bound of uv
    gridding + correction (e_a per axis) and w gridding + correction (e_w);
    nearest-plane w-stacking on the same planes (w snapped by up to dw/2, a
    phase error of up to pi dw |n-1|) is several times further off."""
    nw, sw, wmax = 16, 4, 400.0
    p, src = _dft_problem(nw, seed=47, wmax=wmax)
    q = _padded_w(p["params"], sw, wmax)
    n, S = q["n"], q["support"]
    xs = np.arange(n // 4, 3 * n // 4)
    pix = np.array([(x, y) for y in xs for x in xs], np.int32)
    img, sw_sum, _ = oracle_mod.dirty_image(q, p["u"], p["v"], p["w"], p["wt"], p["vis"], flags=CORRECT)
    ws = img[pix[:, 1], pix[:, 0]]
    at = oracle_mod.image_at(q, p["u"], p["v"], p["w"], p["wt"], p["vis"], pix, flags=CORRECT)
    assert np.max(np.abs(at - ws)) < 1e-10 * np.max(np.abs(ws))
    ref = oracle_mod.dft(q, p["u"], p["v"], p["w"], p["wt"], p["vis"], pix, flags=CORRECT)
    beta = 2.34 * S
    e_a = _alias_bound(KB, S, beta, 0.25, lambda nn: kb_taper(nn, S, beta))
    dl = q["pixel_rad"]
    r2 = (((pix[:, 0] - n // 2) * dl) ** 2 + ((pix[:, 1] - n // 2) * dl) ** 2)
    nm1 = r2 / (1 + np.sqrt(1 - r2))
    dw = (q["w_max"] - q["w_min"]) / nw
    e_w = _w_alias_bound(sw, dw * nm1.max())
    amp = np.sum(np.abs(p["vis"].astype(np.complex128)) * p["wt"]) / sw_sum
    bound = amp * ((1 + e_a) ** 2 * (1 + e_w) - 1)
    err = np.abs(ws - ref)
    assert np.all(err <= bound), (err.max(), bound)
    q1 = dict(q, w_support=1)
    near, _, _ = oracle_mod.dirty_image(q1, p["u"], p["v"], p["w"], p["wt"], p["vis"], flags=CORRECT)
    assert np.max(np.abs(near[pix[:, 1], pix[:, 0]] - ref)) > 5 * err.max()


def test_w_gridding_keeps_the_gridded_sum(oracle_mod):
    """Normalised taps in u, v and w: the planes of a w-support-5 grid sum to
    the weighted visibility sum."""
    p = _small(n=64, nw=10, m=2000, support=7, seed=53, weights="random")
    q = _padded_w(p["params"], 5, 50.0)
    planes, sw, _ = oracle_mod.grid(q, p["u"], p["v"], p["w"], p["wt"], p["vis"])
    placed = oracle_mod.place(q, p["u"], p["v"], p["w"])[0] >= 0
    total = np.sum((p["wt"].astype(np.float64) * p["vis"].astype(np.complex128))[placed])
    assert abs(planes.sum() - total) <= 1e-12 * np.sum(np.abs(p["vis"]) * p["wt"])


def test_w_gridding_adjoint_dot_product(oracle_mod):
    p = _small(n=32, nw=6, m=700, support=7, seed=59, weights="random", fov=8.0, wmax=90.0)
    q = _padded_w(p["params"], 3, 90.0)
    rng = np.random.default_rng(6)
    m = p["u"].shape[0]
    x = (rng.standard_normal(m) + 1j * rng.standard_normal(m)).astype(np.complex64)
    y = rng.standard_normal((32, 32)) + 1j * rng.standard_normal((32, 32))
    for flags in (CORRECT, CORRECT | APPLY_N | UNIFORM):
        Ax, _, _ = oracle_mod.dirty_image(q, p["u"], p["v"], p["w"], p["wt"], x, flags=flags)
        AHy = oracle_mod.degrid(q, p["u"], p["v"], p["w"], p["wt"], x, y, flags=flags)
        lhs = np.vdot(y, Ax)
        rhs = np.vdot(AHy, x.astype(np.complex128))
        assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


def test_phase_screen_sign_matters(oracle_mod):
    """Guards the w-term: with the screen's sign flipped (w -> -w in the data
    while the DFT keeps +w), the source pixel loses most of its flux."""
    p, src = _dft_problem(16, seed=53, wmax=400.0)
    n = p["params"]["n"]
    pix = np.array([(n // 2 + ix, n // 2 + iy) for (ix, iy, _) in src], np.int32)
    ref = oracle_mod.dft(*_args(p), pix, flags=CORRECT)
    flipped = dict(p)
    flipped["w"] = -p["w"]
    ws = oracle_mod.image_at(*_args(flipped), pix, flags=CORRECT)
    assert np.max(np.abs(ws - ref)) > 0.2


# --------------------------------------------------------------------------
# adjoint
# --------------------------------------------------------------------------

@pytest.mark.parametrize("flags", [0, CORRECT, CORRECT | APPLY_N | UNIFORM])
def test_adjoint_dot_product(oracle_mod, flags):
    p = _small(n=32, nw=4, m=700, support=7, seed=59, weights="random", fov=8.0, wmax=90.0)
    rng = np.random.default_rng(2)
    m = p["u"].shape[0]
    x = (rng.standard_normal(m) + 1j * rng.standard_normal(m)).astype(np.complex64)
    y = rng.standard_normal((32, 32)) + 1j * rng.standard_normal((32, 32))
    Ax, _, _ = oracle_mod.dirty_image(p["params"], p["u"], p["v"], p["w"], p["wt"], x, flags=flags)
    AHy = oracle_mod.degrid(p["params"], p["u"], p["v"], p["w"], p["wt"], x, y, flags=flags)
    lhs = np.vdot(y, Ax)                          # <A x, y>
    rhs = np.vdot(AHy, x.astype(np.complex128))   # <x, A^H y>
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


def test_adjoint_dense_matrix(oracle_mod):
    """Tiny problem: build A column by column from unit visibilities, compare
    A^H y with the oracle's degridder."""
    p = _small(n=8, nw=2, m=5, support=3, seed=61, fov=20.0, wmax=40.0, fill=0.3)
    m = p["u"].shape[0]
    cols = []
    for j in range(m):
        e = np.zeros(m, np.complex64)
        e[j] = 1.0
        img, _, _ = oracle_mod.dirty_image(p["params"], p["u"], p["v"], p["w"], p["wt"], e, flags=CORRECT)
        cols.append(img.reshape(-1))
    A = np.stack(cols, 1)
    rng = np.random.default_rng(4)
    y = rng.standard_normal((8, 8)) + 1j * rng.standard_normal((8, 8))
    got = oracle_mod.degrid(p["params"], p["u"], p["v"], p["w"], p["wt"], p["vis"], y, flags=CORRECT)
    ref = A.conj().T @ y.reshape(-1)
    assert np.max(np.abs(got - ref)) <= 1e-12 * np.max(np.abs(ref))
