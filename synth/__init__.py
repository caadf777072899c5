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
FLAG_FOLD = 32
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


def config3(device="cpu", m=200_000_000, n=16384, nw=128, fov_deg=5.0, support=8, seed=BASE_SEED + 3,
            n_ant=512, diameter_m=60_000.0, hours=8.0, dt_s=2.0, freq_hz=1.4e9, dec_deg=-45.0,
            flags=FLAG_CORRECT | FLAG_REAL | FLAG_UNIFORM, batch=50_000_000):
    """SKA-like scale: 16384^2 grid over a 5 degree field (du = 11.46 wavelengths),
    128 w-planes, 2e8 in-grid rows of an Earth-rotation synthesis of 512
    antennas in a 60 km disk over 8 h at dec -45, 1.4 GHz (rows whose
    footprint would leave the grid are re-drawn; the integration step is 2 s
    so that enough in-grid rows exist), Kaiser-Bessel support 8 (beta 18.72),
    uniform weighting.  Visibilities: N(0,1) + i N(0,1) plus a unit source at
    the phase centre."""
    pixel_rad = math.radians(fov_deg) / n
    du = 1.0 / (n * pixel_rad)
    lim = (n / 2 - support / 2 - 1) * du
    us, vs, ws = [], [], []
    kept, it = 0, 0
    while kept < m:
        Lx, Ly, Lz, H, dec = earth_rotation_rows(n_ant, diameter_m, hours, dt_s, dec_deg, -30.0, batch,
                                                 seed * 1000 + it, device)
        u, v, w = rows_to_uvw(Lx, Ly, Lz, H, dec, freq_hz)
        del Lx, Ly, Lz, H
        ok = (u.abs() <= lim) & (v.abs() <= lim)
        take = min(int(ok.sum()), m - kept)
        idx = torch.nonzero(ok).flatten()[:take]
        us.append(u[idx].to(torch.float32))
        vs.append(v[idx].to(torch.float32))
        ws.append(w[idx].to(torch.float32))
        kept += take
        it += 1
        del u, v, w, ok, idx
    u = torch.cat(us)
    v = torch.cat(vs)
    w = torch.cat(ws)
    del us, vs, ws
    gen = _gen(seed + 7)
    vis = torch.empty(m, dtype=torch.complex64, device=u.device)
    step = 1 << 24
    for s0 in range(0, m, step):
        e0 = min(m, s0 + step)
        vis[s0:e0] = (complex_noise(e0 - s0, 1.0, gen) + 1.0).to(u.device)
    params = make_params(n, nw, pixel_rad, float(w.min()), float(w.max()), KERNEL_KB, support, 0.0, flags)
    return dict(params=params, u=u, v=v, w=w, wt=torch.ones(m, dtype=torch.float32, device=u.device), vis=vis)


def channels_problem(nchan=64, n=2048, nw=16, f_lo=0.95e9, f_hi=1.75e9, m_lo=1_000_000, m_hi=20_000_000,
                     n_ant=256, diameter_m=20_000.0, hours=6.0, dt_s=10.0, dec_deg=-30.0, support=7,
                     kernel=KERNEL_KB, seed=BASE_SEED + 4, flags=FLAG_CORRECT | FLAG_REAL, device="cpu",
                     lat_deg=-30.0):
    """Multi-channel problem: nchan frequencies f_c = f_lo + c (f_hi - f_lo)/(nchan-1),
    each with floor(exp(U(ln m_lo, ln m_hi))) rows of the same Earth-rotation
    track (a simulated flagging of uneven depth), its own w-range, and a uv
    cell fixed for all channels by the longest |u|, |v| at f_hi placed at
    0.45 n cells.  Visibilities are N(0,1) + i N(0,1) plus a unit source at
    the phase centre.  The 64-channel, 2048^2, 16-plane configuration is the
    default.  Returns params, channel (w_min, w_max) ranges, offsets and the
    concatenated float32 / complex64 tensors on ``device``."""
    gen = _gen(seed)
    lnm = torch.empty(nchan, dtype=torch.float64).uniform_(math.log(m_lo), math.log(m_hi), generator=gen)
    counts = [int(math.floor(math.exp(float(x)))) for x in lnm]
    freqs = [f_lo + c * (f_hi - f_lo) / max(nchan - 1, 1) for c in range(nchan)]
    parts = []
    umax = 0.0
    for c in range(nchan):
        Lx, Ly, Lz, H, dec = earth_rotation_rows(n_ant, diameter_m, hours, dt_s, dec_deg, lat_deg, counts[c],
                                                 seed * 1000 + c, device)
        u, v, w = rows_to_uvw(Lx, Ly, Lz, H, dec, freqs[c])
        del Lx, Ly, Lz, H
        if counts[c] > 0:
            umax = max(umax, float(torch.maximum(u.abs().max(), v.abs().max())) * f_hi / freqs[c])
        parts.append((u.to(torch.float32), v.to(torch.float32), w.to(torch.float32)))
    du = umax / (0.45 * n)
    pixel_rad = 1.0 / (n * du)
    u = torch.cat([p[0] for p in parts])
    v = torch.cat([p[1] for p in parts])
    w = torch.cat([p[2] for p in parts])
    ranges = [(float(p[2].min()), float(p[2].max())) if p[2].numel() else (-1.0, 1.0) for p in parts]
    ranges = [(a, b) if b > a else (a - 1.0, a + 1.0) for a, b in ranges]
    m = u.numel()
    vis = (complex_noise(m, 1.0, gen) + 1.0).to(torch.complex64).to(u.device)
    offsets = [0]
    for cnt in counts:
        offsets.append(offsets[-1] + cnt)
    params = make_params(n, nw, pixel_rad, 0.0, 1.0, kernel, support, 0.0, flags)
    return dict(params=params, ranges=ranges, offsets=offsets, freqs=freqs, u=u, v=v, w=w,
                wt=torch.ones(m, dtype=torch.float32, device=u.device), vis=vis)


def to_numpy(prob):
    """The same problem as numpy arrays on the host (for the oracle)."""
    return dict(params=dict(prob["params"]),
                u=prob["u"].detach().cpu().numpy(), v=prob["v"].detach().cpu().numpy(),
                w=prob["w"].detach().cpu().numpy(), wt=prob["wt"].detach().cpu().numpy(),
                vis=prob["vis"].detach().cpu().numpy())
