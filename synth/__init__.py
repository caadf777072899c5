"""Seeded synthetic inputs for the w-stacking imager (stand-ins for the LOFAR
HBA observations of the paper's Sec. 4.1, which are not available).

This module is shared by the oracle tests, the GPU tests and the benchmark.
It only produces inputs: coordinates from an Earth-rotation synthesis of a
random array (textbook baseline-to-uvw rotation, Thompson, Moran & Swenson
eq. 4.1), visibilities of a random point-source sky (the measurement equation,
Eq. 2, summed over point sources) plus complex Gaussian noise, or i.i.d.
Gaussian visibilities.  None of the imager's arithmetic lives here: no
placement, kernel, gridding, FFT, phase screen or normalisation.

Every random draw comes from a CPU ``torch.Generator`` seeded explicitly, so
a problem is the same whichever device it is finally put on; only the
deterministic arithmetic (rotation, sky prediction) runs on the requested
device.  Default seed = 20250401 + configuration number.

A problem is a dict: ``params`` (n, nw, pixel_rad, w_min, w_max, kernel,
support, kernel_param, flags) and float32 tensors ``u``, ``v``, ``w``, ``wt``
and complex64 ``vis``, all on ``device``.
"""
import math

import torch

KERNEL_GAUSS = 0
KERNEL_KB = 1
FLAG_CORRECT = 1
FLAG_REAL = 2
FLAG_APPLY_N = 4
FLAG_UNIFORM = 8
C_LIGHT = 299_792_458.0
BASE_SEED = 20250401


def _gen(seed):
    g = torch.Generator(device="cpu")
    g.manual_seed(int(seed))
    return g


def make_params(n, nw, pixel_rad, w_min, w_max, kernel, support, kernel_param=0.0,
                flags=FLAG_CORRECT | FLAG_REAL):
    return dict(n=int(n), nw=int(nw), pixel_rad=float(pixel_rad), w_min=float(w_min),
                w_max=float(w_max), kernel=int(kernel), support=int(support),
                kernel_param=float(kernel_param), flags=int(flags))


# --------------------------------------------------------------------------
# coordinates
# --------------------------------------------------------------------------

def antenna_disk(n_ant, diameter_m, gen):
    """East/north positions uniform in a disk of the given diameter (heights 0)."""
    r = 0.5 * diameter_m * torch.sqrt(torch.rand(n_ant, generator=gen, dtype=torch.float64))
    th = 2.0 * math.pi * torch.rand(n_ant, generator=gen, dtype=torch.float64)
    return r * torch.cos(th), r * torch.sin(th)


def earth_rotation_rows(n_ant, diameter_m, hours, dt_s, dec_deg, lat_deg, m_rows, seed,
                        device="cpu"):
    """Baseline vectors (metres, equatorial frame) and hour angles of m_rows
    (baseline, integration) rows drawn uniformly at random.

    Returns float64 tensors Lx, Ly, Lz, H (radians) on ``device``, plus the
    declination in radians.
    """
    gen = _gen(seed)
    east, north = antenna_disk(n_ant, diameter_m, gen)
    lat = math.radians(lat_deg)
    # local (E, N, U=0) -> equatorial (X, Y, Z) at latitude lat
    X = -math.sin(lat) * north
    Y = east
    Z = math.cos(lat) * north
    ii, jj = torch.triu_indices(n_ant, n_ant, offset=1)
    nb = ii.shape[0]
    nt = int(round(hours * 3600.0 / dt_s))
    rows = torch.randint(0, nb * nt, (int(m_rows),), generator=gen, dtype=torch.int64)
    b = rows // nt
    t = rows % nt
    Lx = (X[jj] - X[ii])[b].to(device)
    Ly = (Y[jj] - Y[ii])[b].to(device)
    Lz = (Z[jj] - Z[ii])[b].to(device)
    H = ((-0.5 * hours + (t.to(torch.float64) + 0.5) * dt_s / 3600.0) * (2.0 * math.pi / 24.0)).to(device)
    return Lx, Ly, Lz, H, math.radians(dec_deg)


def rows_to_uvw(Lx, Ly, Lz, H, dec, freq_hz):
    """Textbook rotation of equatorial baselines to (u, v, w) in wavelengths."""
    lam = C_LIGHT / freq_hz
    sH, cH = torch.sin(H), torch.cos(H)
    sd, cd = math.sin(dec), math.cos(dec)
    u = (sH * Lx + cH * Ly) / lam
    v = (-sd * cH * Lx + sd * sH * Ly + cd * Lz) / lam
    w = (cd * cH * Lx - cd * sH * Ly + sd * Lz) / lam
    return u, v, w


# --------------------------------------------------------------------------
# visibilities
# --------------------------------------------------------------------------

def point_sky(n_src, half_width, seed):
    """n_src point sources, ln(flux) ~ N(0, 1), (l, m) uniform in a square of
    the given half width (direction cosines)."""
    gen = _gen(seed)
    flux = torch.exp(torch.randn(n_src, generator=gen, dtype=torch.float64))
    l = (2.0 * torch.rand(n_src, generator=gen, dtype=torch.float64) - 1.0) * half_width
    m = (2.0 * torch.rand(n_src, generator=gen, dtype=torch.float64) - 1.0) * half_width
    return l, m, flux


def predict_point_sources(u, v, w, l, m, flux, chunk=None):
    """Measurement equation (Eq. 2) for point sources:
    V = sum_s flux_s / n_s exp(-2 pi i (u l_s + v m_s + w (n_s - 1))).
    u, v, w: float64 tensors on any device; returns complex64 there."""
    dev = u.device
    l, m, flux = l.to(dev), m.to(dev), flux.to(dev)
    r2 = l * l + m * m
    n = torch.sqrt(1.0 - r2)
    nm1 = -r2 / (1.0 + n)
    amp = (flux / n).to(torch.float32)
    out = torch.empty(u.shape[0], dtype=torch.complex64, device=dev)
    if chunk is None:
        chunk = (1 << 18) if dev.type == "cuda" else (1 << 14)
    for s in range(0, u.shape[0], chunk):
        e = min(s + chunk, u.shape[0])
        turns = -(u[s:e, None] * l[None, :] + v[s:e, None] * m[None, :] + w[s:e, None] * nm1[None, :])
        turns = turns - torch.round(turns)
        ang = (2.0 * math.pi * turns).to(torch.float32)
        re = (torch.cos(ang) * amp[None, :]).sum(dim=1)
        im = (torch.sin(ang) * amp[None, :]).sum(dim=1)
        out[s:e] = torch.complex(re, im)
    return out


def complex_noise(m, sigma, gen):
    re = torch.randn(m, generator=gen, dtype=torch.float32) * sigma
    im = torch.randn(m, generator=gen, dtype=torch.float32) * sigma
    return torch.complex(re, im)


# --------------------------------------------------------------------------
# problems
# --------------------------------------------------------------------------

def disk_problem(n, nw, m, kernel, support, fov_deg, w_max, seed, kernel_param=0.0,
                 fill=0.45, flags=FLAG_CORRECT | FLAG_REAL, device="cpu", point_source=1.0,
                 weights="unit"):
    """u, v uniform in a disk of radius fill * n * du, w uniform in
    [-w_max, w_max], V = N(0,1) + i N(0,1) + point_source (a source at the
    phase centre).  The 256^2 / 8 planes / 1e5 measurement configuration with a
    Gaussian kernel of support 7 over a 2 degree field is
    ``disk_problem(256, 8, 100_000, KERNEL_GAUSS, 7, 2.0, 50.0, BASE_SEED + 1)``."""
    gen = _gen(seed)
    pixel_rad = math.radians(fov_deg) / n
    du = 1.0 / (n * pixel_rad)
    radius = fill * n * du
    r = radius * torch.sqrt(torch.rand(m, generator=gen, dtype=torch.float64))
    th = 2.0 * math.pi * torch.rand(m, generator=gen, dtype=torch.float64)
    u = (r * torch.cos(th)).to(torch.float32)
    v = (r * torch.sin(th)).to(torch.float32)
    w = ((2.0 * torch.rand(m, generator=gen, dtype=torch.float64) - 1.0) * w_max).to(torch.float32)
    vis = complex_noise(m, 1.0, gen) + point_source
    if weights == "unit":
        wt = torch.ones(m, dtype=torch.float32)
    else:
        wt = (0.5 + torch.rand(m, generator=gen, dtype=torch.float64)).to(torch.float32)
    params = make_params(n, nw, pixel_rad, -w_max, w_max, kernel, support, kernel_param, flags)
    return dict(params=params, u=u.to(device), v=v.to(device), w=w.to(device),
                wt=wt.to(device), vis=vis.to(torch.complex64).to(device))


def config1(device="cpu", seed=BASE_SEED + 1):
    """256x256 grid, 8 w-planes, 1e5 N(0,1)+iN(0,1)+1 visibilities, u,v uniform
    in a disk of radius 0.45 n du, w uniform in [-50, 50], unit weights,
    Gaussian support 7, FOV 2 degrees."""
    return disk_problem(256, 8, 100_000, KERNEL_GAUSS, 7, 2.0, 50.0, seed, device=device)


def earth_rotation_problem(n, nw, m, kernel, support, n_ant, diameter_m, hours, dt_s,
                           freq_hz, dec_deg, seed, lat_deg=-30.0, n_src=200, noise=0.1,
                           kernel_param=0.0, fill=0.45, flags=FLAG_CORRECT | FLAG_REAL,
                           device="cpu"):
    """Earth-rotation synthesis problem: the uv cell is set so that the longest
    drawn |u| or |v| sits at fill * n cells from the centre, the field of view
    is 1 / du, w_min / w_max are the data extremes, and the visibilities are
    a point-source sky (sources uniform in the central 80 % of the field) plus
    complex N(0, noise) noise.  The 4096^2 / 32 planes / 1e7 measurement
    configuration (256 antennas in a 20 km disk, 6 h of 10 s integrations at
    1.4 GHz, declination -30) is ``config2()``."""
    Lx, Ly, Lz, H, dec = earth_rotation_rows(n_ant, diameter_m, hours, dt_s, dec_deg, lat_deg,
                                             m, seed, device)
    u, v, w = rows_to_uvw(Lx, Ly, Lz, H, dec, freq_hz)
    del Lx, Ly, Lz, H
    umax = float(torch.maximum(u.abs().max(), v.abs().max()))
    du = umax / (fill * n)
    pixel_rad = 1.0 / (n * du)
    l, mm, flux = point_sky(n_src, 0.4 * n * pixel_rad, seed + 1000)
    vis = predict_point_sources(u, v, w, l, mm, flux)
    gen = _gen(seed + 2000)
    vis = vis + complex_noise(m, noise, gen).to(vis.device)
    u32, v32, w32 = u.to(torch.float32), v.to(torch.float32), w.to(torch.float32)
    del u, v, w
    w_min, w_max = float(w32.min()), float(w32.max())
    params = make_params(n, nw, pixel_rad, w_min, w_max, kernel, support, kernel_param, flags)
    wt = torch.ones(m, dtype=torch.float32, device=u32.device)
    return dict(params=params, u=u32, v=v32, w=w32, wt=wt, vis=vis.to(torch.complex64),
                sky=dict(l=l, m=mm, flux=flux))


def config2(device="cpu", m=10_000_000, n=4096, nw=32, seed=BASE_SEED + 2):
    """4096x4096 grid, 32 w-planes, 1e7 visibilities from 256 antennas in a
    20 km disk, 6 h Earth-rotation synthesis at dec -30, 10 s integrations,
    1.4 GHz, 200 point sources + N(0, 0.1) noise, Kaiser-Bessel support 7
    (beta = 2.34 * 7)."""
    return earth_rotation_problem(n, nw, m, KERNEL_KB, 7, 256, 20_000.0, 6.0, 10.0, 1.4e9,
                                  -30.0, seed, device=device)


def to_numpy(prob):
    """The same problem as numpy arrays on the host (for the oracle)."""
    return dict(params=dict(prob["params"]),
                u=prob["u"].detach().cpu().numpy(), v=prob["v"].detach().cpu().numpy(),
                w=prob["w"].detach().cpu().numpy(), wt=prob["wt"].detach().cpu().numpy(),
                vis=prob["vis"].detach().cpu().numpy())
