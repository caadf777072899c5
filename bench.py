"""Benchmark of the w-stacking imager hot path on GB300.

One step = the whole path for one dirty image: reset, placement + counting
sort (and the uniform-weighting density), gridding of every w-plane, the
per-plane inverse FFT, the phase-screen stack and the finalisation.  Inputs
are resident in HBM when the timed region starts; every step writes and reads
all planes (hundreds of GB at the default size), far more than L2, so no L2
flush is needed.

Default workload (``--workload large``): a 16384^2 grid over a 5 degree
field, 128 w-planes in plane groups, 2e8 visibilities of a 512-antenna,
60 km, 8 h Earth-rotation synthesis at dec -45 (1.4 GHz), Kaiser-Bessel
support 8, uniform weighting computed on the device.  ``--workload wstack``:
the 4096^2 / 32-plane / 1e7-visibility image (256 antennas, 20 km, 6 h,
dec -30, 200-source sky + noise, Kaiser-Bessel support 7).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--workload large|wstack|channels|adjoint|small|densechannel]

Multi-GPU (torchrun): one image over all ranks -- every rank takes all
measurements and transforms and stacks its share of the w-planes, and one
NCCL all-reduce per step sums the images (strong scaling); value = the
image's visibilities per step / the slowest rank's time per step.

The line carries the gridder's roofline (``roofline``), the fused stack's
(``roofline_other``), per-phase GB/s, NVML energy per image, the end-to-end
rate through the C ABI with host buffers (``e2e``), and -- from the FP64
oracle, on rank 0 at N = 1 -- the CPU baseline (``cpu_baseline``) and the
error of the timed image against the oracle at sampled pixels (``parity``).
``--impl reference`` times the FP64 oracle alone on the host cores, one
bounded sample of the same workload per step (rank 0 only).
"""
import argparse
import ctypes
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "visibilities/sec end-to-end (grid+FFT+w-stack), % roofline, J/solution"
WORKLOADS = {
    "large": ("plain w-stacking at SKA-like scale: 16384x16384 grid, 128 w-planes in plane groups, 2e8 "
              "visibilities (512 antennas, 60 km disk, 8 h synthesis, dec -45, 1.4 GHz, 5 deg FOV), "
              "Kaiser-Bessel support 8, uniform weighting computed on the device, FP32"),
    "wstack": ("plain w-stacking, 4096x4096 grid, 32 w-planes, 1e7 visibilities (256 antennas, 20 km disk, "
               "6 h synthesis, dec -30, 10 s, 1.4 GHz, 200 sources + noise), Kaiser-Bessel support 7, FP32"),
}
DATA = {
    "large": "synthetic: seeded Earth-rotation synthesis, N(0,1) visibilities + a unit source at the phase "
             "centre (the paper's LOFAR data is not available)",
    "wstack": "synthetic: seeded Earth-rotation synthesis + point-source sky (the paper's LOFAR data is not "
              "available)",
}


def make_problem(workload, device, nvis=None, nw=None):
    """The seeded synthetic problem of a single-image workload and its flags."""
    import synth
    if workload == "large":
        kw = {}
        if nvis:
            kw["m"] = nvis
        if nw:
            kw["nw"] = nw
        prob = synth.config3(device=device, **kw)
        return prob, dict(prob["params"])
    prob = synth.config2(device=device, m=nvis or 10_000_000, nw=nw or 32)
    return prob, dict(prob["params"], flags=synth.FLAG_CORRECT | synth.FLAG_REAL)


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def _kernel_hash(name):
    with open(os.path.join(ROOT, "paper_2504_00959_gb300", "csrc", name), "rb") as f:
        return hashlib.sha256(f.read()).hexdigest()[:16]


def _traffic(kernel_file, workload_key):
    """DRAM bytes per launch from a committed ncu summary, if it was taken on
    the current source of the kernel (else None)."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as f:
            d = json.load(f)
        e = d[workload_key]
        if e.get("source_sha256_16") != _kernel_hash(kernel_file):
            return None
        return float(e["dram_bytes_per_launch"])
    except Exception:
        return None


# ------------------------------------------------------------------ clocks
class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id):
        self.gpu_id = gpu_id
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu_id), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.thread.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[3:7]):
                if val.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------------ energy
class Nvml:
    def __init__(self, uuid):
        self.ok = False
        try:
            self.lib = ctypes.CDLL("libnvidia-ml.so.1")
            if self.lib.nvmlInit_v2() != 0:
                return
            self.h = ctypes.c_void_p()
            if self.lib.nvmlDeviceGetHandleByUUID(uuid.encode(), ctypes.byref(self.h)) != 0:
                return
            self.ok = True
        except Exception:
            self.ok = False

    def energy_mj(self):
        if not self.ok:
            return None
        e = ctypes.c_ulonglong(0)
        if self.lib.nvmlDeviceGetTotalEnergyConsumption(self.h, ctypes.byref(e)) != 0:
            return None
        return int(e.value)


# ------------------------------------------------------------ CPU baseline
ORACLE_SLICE = 2_000_000    # measurements of the placement and gridding sample
ORACLE_MAX_FFT_N = 4096     # largest plane the FFT sample transforms


def oracle_round(prob_np, plane, on_plane_idx):
    """One bounded sample of the FP64 oracle on the host cores, the same
    workload, each piece through the oracle's own entry points.  The oracle's
    dirty image (oracle_dirty_image) computes the effective weights once (one
    placement pass, two with uniform weighting), then for every plane places
    all measurements again, grids those on the plane (taps + S^2 updates),
    zeroes, transforms (FP64 FFT) and screens the plane, and finalises once.
    Measured here (the unit costs do not depend on the weights, so the
    samples run without uniform weighting and its n^2 density array):
      t_pass  oracle.grid(slice, no plane): weights + one placement pass of a
              slice of the measurements (two passes, 1 thread)
      t_zero  oracle.grid(no measurement, one plane): zeroing of one plane
      t_k0    oracle.grid(measurements on the plane, no plane)
      t_k     oracle.grid(measurements on the plane, the plane): t_k0 + t_zero
              + their gridding (1 thread)
      t_plane oracle.dirty_image(one measurement, plane) minus the same with
              no plane, at n or at 4096 for larger n: one plane's zeroing,
              FFT and screen (OpenMP)
      t_fin   oracle.dirty_image(one measurement, no plane): the
              finalisation of n^2 pixels (OpenMP)
    Returns the unit costs and the wall time of the round."""
    import oracle
    p = prob_np
    q = p["params"]
    q0 = dict(q, flags=int(q.get("flags", 0)) & ~8)
    n = int(q["n"])
    uniform = bool(int(q.get("flags", 0)) & 8)
    m_all = p["u"].shape[0]
    ms = min(m_all, ORACLE_SLICE)
    keys = ("u", "v", "w", "wt", "vis")
    sl = {k: p[k][:ms] for k in keys}
    on = {k: p[k][on_plane_idx] for k in keys}
    one = {k: p[k][:1] for k in keys}
    none = {k: p[k][:0] for k in keys}
    t_round = time.perf_counter()

    def timed(fn, *a, **kw):
        t0 = time.perf_counter()
        fn(*a, **kw)
        return time.perf_counter() - t0

    args = lambda d: (d["u"], d["v"], d["w"], d["wt"], d["vis"])  # noqa: E731
    t_pass = timed(oracle.grid, q0, *args(sl), k0=0, k1=0)
    t_zero = timed(oracle.grid, q0, *args(none), k0=plane, k1=plane + 1)
    t_k0 = timed(oracle.grid, q0, *args(on), k0=0, k1=0)
    t_k = timed(oracle.grid, q0, *args(on), k0=plane, k1=plane + 1)
    n_s = min(n, ORACLE_MAX_FFT_N)
    qs = dict(q0, n=n_s)
    t_fin_s = timed(oracle.dirty_image, qs, *args(one), k0=0, k1=0)
    t_pl_s = timed(oracle.dirty_image, qs, *args(one), k0=plane, k1=plane + 1) - t_fin_s
    # an FFT of n^2 points costs ~ n^2 log n^2; the screen and finalisation ~ n^2
    fft_scale = (n / n_s) ** 2 * math.log2(float(n) * n) / math.log2(float(n_s) * n_s)
    m_on = int(on_plane_idx.shape[0])
    return {"c_place": t_pass / (2 * ms), "c_grid": max(t_k - t_k0 - t_zero, 0.0) / max(m_on, 1),
            "t_plane": max(t_pl_s, 0.0) * fft_scale, "t_fin": t_fin_s * (n / n_s) ** 2, "n_s": n_s,
            "fft_scale": fft_scale, "slice": ms, "on_plane": m_on, "plane": plane,
            "wall": time.perf_counter() - t_round, "passes_w": 2 if uniform else 1}


def oracle_image_seconds(r, m_all, m_gridded, nw):
    """Seconds of the oracle's whole dirty image from one round's unit costs:
    weights (1 or 2 placement passes) + nw x (a placement pass + one plane's
    zeroing, FFT and screen) + the gridding of every gridded measurement +
    the finalisation."""
    return (r["passes_w"] * m_all * r["c_place"] + nw * (m_all * r["c_place"] + r["t_plane"]) +
            m_gridded * r["c_grid"] + r["t_fin"])


def oracle_plane_sample(prob_np):
    """The sampled plane (the one holding the mean number of the first
    ORACLE_SLICE measurements) and the indices of the measurements on it among
    the first 10 x ORACLE_SLICE."""
    import numpy as np

    import oracle
    p = prob_np
    q = p["params"]
    nw = int(q["nw"])
    m_all = p["u"].shape[0]
    mm = min(m_all, 10 * ORACLE_SLICE)
    kk, _, _ = oracle.place(q, p["u"][:mm], p["v"][:mm], p["w"][:mm])
    cnt = np.bincount(kk[:ORACLE_SLICE][kk[:ORACLE_SLICE] >= 0], minlength=nw)
    plane = int(np.argmin(np.abs(cnt - cnt.mean())))
    idx = np.nonzero(kk == plane)[0]
    del np
    return plane, idx


def oracle_sample(prob_np, m_gridded, rounds=3):
    """The FP64 oracle's rate on this workload (visibilities/s) from the median
    of `rounds` bounded samples (oracle_round) on a plane holding a typical
    number of measurements.  Returns (value, description, threads, seconds)."""
    import numpy as np

    import oracle
    p = prob_np
    q = p["params"]
    n, nw = int(q["n"]), int(q["nw"])
    m_all = p["u"].shape[0]
    plane, idx = oracle_plane_sample(p)
    t0 = time.perf_counter()
    rs = [oracle_round(p, plane, idx) for _ in range(max(rounds, 1))]
    wall = time.perf_counter() - t0
    secs = [oracle_image_seconds(r, m_all, m_gridded, nw) for r in rs]
    med = statistics.median(secs)
    r = rs[secs.index(med)] if med in secs else rs[0]
    threads = oracle.num_threads()
    desc = (f"median of {len(rs)} rounds (image estimates {', '.join('%.0f' % x for x in secs)} s); per round: "
            f"weights + placement of {r['slice']} measurements ({r['c_place'] * 1e9:.0f} ns per measurement "
            f"and pass, 1 thread), gridding of {r['on_plane']} measurements on plane {plane} "
            f"({r['c_grid'] * 1e6:.2f} us per measurement, 1 thread), one plane's zeroing + FFT + screen at "
            f"{r['n_s']}^2 "
            f"({r['t_plane'] / r['fft_scale']:.2f} s, {threads} threads"
            + (f", x{r['fft_scale']:.1f} for {n}^2 by n^2 log n^2" if r['n_s'] != n else "") +
            f"); image = {r['passes_w']} weight pass(es) + {nw} x (placement pass of {m_all} + plane) + "
            f"gridding of {m_gridded} + finalisation; measured {wall:.1f} s")
    del np
    return m_all / med, desc, threads, wall, {"placement_and_gridding": 1, "fft_and_screen": threads}


def parity_check(prob_np, params, image, side=8):
    """Error of a GPU image against the FP64 oracle (oracle_image_at: the same
    discrete algorithm evaluated per pixel) at a side x side lattice of
    pixels spanning the image edge to edge, the phase centre and the GPU
    image's brightest pixel.  With grid correction both sides are compared
    before the division by the taper (the GPU pixel times c(x) c(y)).
    Returns max |gpu - oracle| / max |oracle| over the sampled pixels."""
    import numpy as np

    import oracle
    q = dict(params)
    n = int(q["n"])
    flags = int(params["flags"])
    img = np.asarray(image)
    lat = np.unique(np.linspace(0, n - 1, side).round().astype(np.int64))
    pix = [(int(x), int(y)) for y in lat for x in lat]
    pk = int(np.argmax(np.abs(img)))
    pix += [(n // 2, n // 2), (pk % n, pk // n)]
    pix = np.array(sorted(set(pix)), dtype=np.int32)
    t0 = time.perf_counter()
    ref = oracle.image_at(q, prob_np["u"], prob_np["v"], prob_np["w"], prob_np["wt"], prob_np["vis"], pix,
                          flags=flags & ~1)
    secs = time.perf_counter() - t0
    got = img[pix[:, 1], pix[:, 0]]
    if flags & 1:
        c = oracle.taper(n, int(q["kernel"]), int(q["support"]), float(q.get("kernel_param", 0.0) or 0.0))
        got = got * c[pix[:, 0]] * c[pix[:, 1]]
    if flags & 2:
        ref = ref.real
    err = float(np.max(np.abs(got - ref)) / max(np.max(np.abs(ref)), 1e-300))
    del np
    return {"max_abs_err_over_peak": err, "bound": 1e-4, "ok": err <= 1e-4, "pixels": int(pix.shape[0]),
            "reference": "FP64 oracle (oracle_image_at) at a %dx%d pixel lattice edge to edge + phase centre + "
                         "brightest pixel, before the taper division" % (len(lat), len(lat)),
            "oracle_seconds": secs}


# ------------------------------------------------------------------ main
def aggregate(ms_local, job_units_per_step, steps, world, device):
    """Slowest rank's timed-region milliseconds and the whole-job throughput:
    the job (all ranks together) processes job_units_per_step units per
    step, value = job_units_per_step * steps / slowest time."""
    import torch
    import torch.distributed as dist
    ms = float(ms_local)
    if world > 1:
        t = torch.tensor([ms], device=device, dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    return ms, job_units_per_step * steps / (ms / 1e3)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--nvis", type=int, default=0, help="measurements (0: the workload's own count)")
    ap.add_argument("--nw", type=int, default=0, help="w-planes (0: the workload's own count)")
    ap.add_argument("--tile", type=int, default=0, help="gridder tile side (0 = automatic)")
    ap.add_argument("--fold", action="store_true",
                    help="Hermitian fold (real image): measurements with w < 0 mirrored, half the w-planes "
                         "over [0, max |w|] at the same plane spacing")
    ap.add_argument("--w-support", type=int, default=0,
                    help="planes per measurement (Eq. 3's kernel in w); the plane range is padded by "
                         "nw / (nw - w_support) so every footprint lies on the planes")
    ap.add_argument("--fft2d", action="store_true",
                    help="cuFFT's 2D plan + a separate stack pass (RICK_FFT_2D) instead of the split transform")
    ap.add_argument("--no-cpu-baseline", action="store_true",
                    help="skip the FP64 oracle (CPU baseline and parity of the timed image)")
    ap.add_argument("--no-e2e", action="store_true", help="skip the host-buffer end-to-end leg")
    ap.add_argument("--workload", choices=["large", "wstack", "channels", "adjoint", "small", "densechannel"],
                    default="large",
                    help="large: 16384^2 / 128 planes / 2e8 measurements with uniform weighting, in plane "
                         "groups (default); wstack: the 4096^2 / 32-plane / 1e7 image; channels: 64 channels "
                         "batched vs imaged one by one; adjoint: image + loss gradient through the adjoint "
                         "degridder on the wstack workload; small: 256^2 / 8 planes / 1e5, microseconds per "
                         "image; densechannel: the densest channel of the 64 imaged alone (2048^2 / 16 planes "
                         "/ 2e7)")
    args = ap.parse_args()

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if args.impl == "reference":
        return run_reference(args, rank, world)
    if args.workload == "channels":
        return run_channels(args, rank, world)
    if args.workload == "adjoint":
        return run_adjoint(args, rank, world)
    if args.workload == "small":
        return run_small(args, rank, world)
    if args.workload == "densechannel":
        return run_dense_channel(args, rank, world)
    return run_image(args, rank, world)


def workload_config(wl, params, m, world, args):
    """The `config` object of a single-image workload's line (the same in the
    GPU arm and the reference arm)."""
    n, nw = int(params["n"]), int(params["nw"])
    desc = WORKLOADS[wl]
    if args.fold:
        desc += "; Hermitian fold: %d w-planes over [0, max |w|]" % nw
    if args.w_support > 1:
        desc += "; w-support %d on %d planes" % (args.w_support, nw)
    return {"workload": desc, "n": n, "nw": nw, "nvis": int(m), "kernel": "kaiser-bessel",
            "support": int(params["support"]), "uniform_weighting": bool(int(params["flags"]) & 8),
            "l2": "inputs larger than L2 (%.2f GB of planes written and read every step)" % (8.0 * nw * n * n / 1e9),
            "parallelism": ("%d GPUs: w-planes sharded, NCCL all-reduce of the image" % world) if world > 1
            else "single GPU"}


def _nvml_for(dev):
    import torch
    props = torch.cuda.get_device_properties(dev)
    uuid = str(getattr(props, "uuid", ""))
    uuid = uuid if uuid.startswith("GPU-") else ("GPU-" + uuid if uuid else "")
    return (Nvml(uuid) if uuid else None), (uuid if uuid else dev.index)


def run_image(args, rank, world):
    """One dirty image per step of a single-image workload (large or wstack)."""
    import torch
    import torch.distributed as dist

    import synth
    import paper_2504_00959_gb300 as rick
    from paper_2504_00959_gb300 import build as rick_build
    rick_build.build()
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    if world > 1:
        dist.init_process_group("nccl", device_id=dev)

    wl = args.workload
    prob, params = make_problem(wl, dev, args.nvis or None, args.nw or None)
    params["tile"] = args.tile
    if args.fft2d:
        params["flags"] = params["flags"] | rick.FFT_2D
    if args.fold:
        wabs = max(abs(params["w_min"]), abs(params["w_max"]))
        params = dict(params, nw=max(params["nw"] // 2, 1), w_min=0.0, w_max=wabs,
                      flags=params["flags"] | synth.FLAG_FOLD)
    if args.w_support > 1:
        lo, hi, nwp = params["w_min"], params["w_max"], params["nw"]
        mid, half = 0.5 * (lo + hi), 0.5 * (hi - lo) * nwp / (nwp - args.w_support)
        params = dict(params, w_min=mid - half, w_max=mid + half, w_support=args.w_support)
    im = rick.Imager(params, device=dev)
    n, nw = params["n"], params["nw"]
    img = torch.empty((n, n), dtype=torch.float32, device=dev)
    m = prob["u"].numel()
    k0, k1 = 0, nw
    if world > 1:
        # one image over all ranks: rank r transforms and stacks the w-planes
        # of its share, and one all-reduce sums the images
        from paper_2504_00959_gb300.sharded import plane_share
        k0, k1 = plane_share(nw, rank, world)
        im.set_plane_range(k0, k1)

    def step():
        im.reset()
        im.grid(prob["vis"], prob["u"], prob["v"], prob["w"], prob["wt"])
        im.image(out=img)
        if world > 1:
            dist.all_reduce(img)

    for _ in range(max(args.warmup, 0)):
        step()
    torch.cuda.synchronize()
    st = im.stats()

    nvml, clock_id = _nvml_for(dev)
    clocks = ClockSampler(clock_id)
    im.set_timing(True)
    start = torch.cuda.Event(enable_timing=True)
    end = torch.cuda.Event(enable_timing=True)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    e0 = nvml.energy_mj() if nvml else None
    start.record()
    for _ in range(args.steps):
        step()
    end.record()
    torch.cuda.synchronize()
    e1 = nvml.energy_mj() if nvml else None
    if world > 1:
        dist.barrier()
    clk = clocks.stop()
    ms = start.elapsed_time(end)
    tm = im.timing()
    st = im.stats()  # raises if a bounded wait of the fused column kernel ran out
    ms, value = aggregate(ms, m, args.steps, world, dev)
    if world > 1 and e0 is not None and e1 is not None:
        ej = torch.tensor([float(e1 - e0)], dtype=torch.float64, device=dev)
        dist.all_reduce(ej)  # the job's energy: every rank's GPU
        e0, e1 = 0, float(ej.item())
    steps = max(args.steps, 1)
    ms_step = ms / steps

    # ------------------------------------------------ rooflines and phases
    # algorithmic bytes per step: the gridder reads each gridded measurement
    # once (u, v, w, weight, visibility: 24 B) and writes every plane cell
    # once (8 B); cuFFT at least two read + write passes over the planes;
    # the stack reads every plane once and writes the image (4 B per pixel,
    # plus the complex accumulator between plane groups); the prep reads the
    # measurements twice (count, scatter; a third time for the uniform-
    # weighting density) and writes one 16 B entry per (measurement, tile)
    peak, peak_kind = _peaks()
    cells = float(k1 - k0) * n * n  # this rank's planes
    groups = -(-(k1 - k0) // max(st["plane_group"], 1))
    uniform = bool(params["flags"] & synth.FLAG_UNIFORM)
    grid_ms = tm["grid_ms"] / steps
    grid_bytes = 24.0 * st["n_gridded"] + 8.0 * cells
    stack_ms = tm["stack_ms"] / steps
    stack_bytes = 8.0 * cells + 4.0 * n * n + (2 * 8.0 * n * n * (groups - 1) if groups > 1 else 0.0)
    split = tm["colfft_calls"] > 0  # the split transform: cuFFT rows, k_colfft, k_colstack
    fft_ms = tm["fft_ms"] / steps
    fft_bytes = (1 if split else 2) * 2 * 8.0 * cells  # one read + write pass per dimension
    colfft_ms = tm["colfft_ms"] / steps
    colfft_bytes = 2 * 8.0 * cells if split else 0.0
    prep_ms = tm["prep_ms"] / steps
    prep_bytes = (3 if uniform else 2) * 24.0 * m + 16.0 * st["n_entries"]
    phases = {
        "prep": {"ms": prep_ms, "algorithmic_gb": prep_bytes / 1e9},
        "grid": {"ms": grid_ms, "algorithmic_gb": grid_bytes / 1e9},
        ("fft_cufft_rows" if split else "fft_cufft"): {"ms": fft_ms, "algorithmic_gb": fft_bytes / 1e9},
        "stack": {"ms": stack_ms, "algorithmic_gb": stack_bytes / 1e9},
    }
    if split:
        phases["colfft"] = {"ms": colfft_ms, "algorithmic_gb": colfft_bytes / 1e9}
    for v in phases.values():
        v["gbs"] = v["algorithmic_gb"] / v["ms"] * 1e3 if v["ms"] > 0 else None
        v["frac_of_" + peak_kind] = v["gbs"] / peak if v["gbs"] else None
    # committed DRAM counters (profiles/traffic.json): small-case ncu captures
    # of the 4096^2 x 32 x 1e7 workload, and of k_colfft on 2 planes of 16384^2
    # scaled to a launch of the 16384^2 x 128 x 2e8 one
    plain = params.get("w_support", 1) <= 1 and not params["flags"] & synth.FLAG_FOLD
    default_size = wl == "wstack" and (n, nw, m) == (4096, 32, 10_000_000) and plain
    large_size = wl == "large" and (n, nw, m) == (16384, 128, 200_000_000) and plain
    traffic = _traffic("rick_grid.cu", "k_grid@4096x32x1e7") if default_size else None
    stack_name = ("k_colstack (last 16-point column factor + w-screen + stack, Eq. 1)" if split
                  else "k_stack (w-screen + stack, Eq. 1)")
    stack_traffic = _traffic("rick_stack.cu", "k_colstack@4096x32x1e7") if (default_size and split) else None
    launches_grid = max(tm["grid_calls"] / steps, 1)
    launches_stack = max(tm["stack_calls"] / steps, 1)
    rl_grid = {"kernel": "k_grid_tiles + k_grid_heavy (gridding, Eq. 3)", "bound": "hbm",
               "achieved": grid_bytes / grid_ms / 1e6, "peak": peak, "unit": "GB/s",
               "frac": grid_bytes / grid_ms / 1e6 / peak, "traffic": traffic, "peak_kind": peak_kind,
               "algorithmic_bytes_per_launch": grid_bytes / launches_grid, "launch_ms": grid_ms / launches_grid,
               "launches_per_step": launches_grid}
    rl_stack = {"kernel": stack_name, "bound": "hbm", "achieved": stack_bytes / stack_ms / 1e6, "peak": peak,
                "unit": "GB/s", "frac": stack_bytes / stack_ms / 1e6 / peak, "traffic": stack_traffic,
                "peak_kind": peak_kind, "algorithmic_bytes_per_launch": stack_bytes / launches_stack,
                "launch_ms": stack_ms / launches_stack, "launches_per_step": launches_stack}
    own = [(grid_ms, rl_grid), (stack_ms, rl_stack)]
    if split:
        launches_cf = max(tm["colfft_calls"] / steps, 1)
        own.append((colfft_ms, {
            "kernel": "k_colfft (first n/16-point column factor of the plane transform, TMA-fed)", "bound": "hbm",
            "achieved": colfft_bytes / colfft_ms / 1e6, "peak": peak, "unit": "GB/s",
            "frac": colfft_bytes / colfft_ms / 1e6 / peak,
            "traffic": (_traffic("rick_colfft.cu", "k_colfft@4096x32x1e7") if default_size else
                        _traffic("rick_colfft.cu", "k_colfft@16384x128x2e8") if large_size else None),
            "peak_kind": peak_kind,
            "algorithmic_bytes_per_launch": colfft_bytes / launches_cf, "launch_ms": colfft_ms / launches_cf,
            "launches_per_step": launches_cf}))
    own.sort(key=lambda t: -t[0])
    rl, rl_other = own[0][1], [o[1] for o in own[1:]]

    # ------------------------------------------------ end to end, host buffers
    e2e = None
    if not args.no_e2e and world > 1:
        # every rank uploads the inputs, images its share, the ranks sum the
        # images and every rank downloads the image
        hv, hu, hvv, hw, hwt = (torch.empty(prob[k].shape, dtype=prob[k].dtype, pin_memory=True).copy_(prob[k])
                                for k in ("vis", "u", "v", "w", "wt"))
        himg = torch.empty((n, n), dtype=torch.float32, pin_memory=True)
        dv, du, dvv, dww, dwt = (torch.empty_like(prob[k]) for k in ("vis", "u", "v", "w", "wt"))

        def e2e_step():
            for d, h_ in ((dv, hv), (du, hu), (dvv, hvv), (dww, hw), (dwt, hwt)):
                d.copy_(h_, non_blocking=True)
            im.reset()
            im.grid(dv, du, dvv, dww, dwt)
            im.image(out=img)
            dist.all_reduce(img)
            himg.copy_(img, non_blocking=True)

        e2e_step()
        torch.cuda.synchronize()
        dist.barrier()
        ksteps = max(min(args.steps, 5), 1)
        t0 = time.perf_counter()
        for _ in range(ksteps):
            e2e_step()
        torch.cuda.synchronize()
        te_t = torch.tensor([(time.perf_counter() - t0) / ksteps], dtype=torch.float64, device=dev)
        dist.all_reduce(te_t, op=dist.ReduceOp.MAX)
        te = float(te_t.item())
        e2e = {"value": m / te, "unit": "vis/s", "ms_per_step": te * 1e3,
               "h2d_bytes_per_step": int(world * m * (8 + 4 + 4 + 4 + 4)), "d2h_bytes_per_step": int(world * n * n * 4),
               "api": "Imager.grid + image on each rank's plane share from pinned host copies, NCCL all-reduce, "
                      "image download; %d steps, slowest rank" % ksteps}
        del hv, hu, hvv, hw, hwt, himg, dv, du, dvv, dww, dwt
    elif not args.no_e2e:
        # pinned host copies of the inputs, filled straight from the device
        hv, hu, hvv, hw, hwt = (torch.empty(prob[k].shape, dtype=prob[k].dtype, pin_memory=True).copy_(prob[k])
                                for k in ("vis", "u", "v", "w", "wt"))
        himg = torch.empty((n, n), dtype=torch.float32, pin_memory=True)
        himg2 = torch.empty((n, n), dtype=torch.float32, pin_memory=True)
        im.image_host(hv, hu, hvv, hw, hwt, out=himg)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ksteps = max(min(args.steps, 3), 1)
        for _ in range(ksteps):
            im.image_host(hv, hu, hvv, hw, hwt, out=himg)
        te_sync = (time.perf_counter() - t0) / ksteps
        # a stream of images through the pipelined call: upload of image i+1
        # and download of image i-1 under the imaging of image i
        for j in range(2):
            im.image_host_async(hv, hu, hvv, hw, hwt, out=(himg, himg2)[j % 2])
        im.synchronize()
        ksteps = max(min(args.steps, 20), 2)
        t0 = time.perf_counter()
        for j in range(ksteps):
            im.image_host_async(hv, hu, hvv, hw, hwt, out=(himg, himg2)[j % 2])
        im.synchronize()
        te = (time.perf_counter() - t0) / ksteps
        e2e = {"value": m / te, "unit": "vis/s", "ms_per_step": te * 1e3,
               "h2d_bytes_per_step": int(m * (8 + 4 + 4 + 4 + 4)), "d2h_bytes_per_step": int(n * n * 4),
               "api": "rick_image_host_async over %d images, then rick_synchronize (pinned host buffers)" % ksteps,
               "unpipelined_ms_per_step": te_sync * 1e3}
        del hv, hu, hvv, hw, hwt, himg, himg2
        if hasattr(torch._C, "_host_emptyCache"):
            torch._C._host_emptyCache()  # return the pinned staging memory before the CPU leg

    # ------------------------------------------------ FP64 oracle: CPU baseline and parity
    cpu = parity = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        image_cpu = img.cpu().numpy()
        im.close()
        prob_np = synth.to_numpy(prob)
        prob_np["params"] = dict(params)
        del prob
        parity = parity_check(prob_np, params, image_cpu)
        v, desc, threads, secs, by_phase = oracle_sample(prob_np, st["n_gridded"])
        cpu = {"value": v, "unit": "vis/s", "cores": threads, "kind": "oracle", "sample": desc,
               "threads_by_phase": by_phase, "seconds": secs}
    else:
        im.close()

    energy = None
    if e0 is not None and e1 is not None:
        energy = (e1 - e0) / 1e3 / steps

    config = workload_config(wl, params, m, world, args)
    # whole step against HBM: prep + gridder + FFT (2 passes) + stack
    step_bytes = prep_bytes + grid_bytes + fft_bytes + colfft_bytes + stack_bytes
    out = {
        "metric": METRIC, "value": value, "unit": "vis/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "strong",
        "vs_baseline": None, "dtype": "f32", "data": DATA[wl], "config": config,
        "roofline": rl, "roofline_other": rl_other, "phases": phases,
        "roofline_frac_end_to_end": step_bytes / (ms_step / 1e3) / 1e9 / peak,
        "energy_j_per_solution": energy, "e2e": e2e, "cpu_baseline": cpu, "parity": parity,
        "gpu_launches": int(tm["kernel_launches"]), "clocks": clk,
        "launch": {"tile": st["tile"], "plane_group": st["plane_group"], "plane_groups": groups,
                   "planes_of_rank0": [k0, k1], "workspace_gb": st["workspace_bytes"] / 1e9},
    }
    if rank == 0:
        print(json.dumps(out))
    if world > 1:
        dist.destroy_process_group()


def run_channels(args, rank, world):
    """64 frequency channels (0.95-1.75 GHz), 2048^2 grid and 16 w-planes each,
    1e6-2e7 measurements per channel (log-uniform): one autotuned batched
    step (captured CUDA graph) against the plain loop of one imager per
    channel (reset, grid, FFT + stack), at equal accuracy.  Also reports the
    green productivity of Eq. 4 (alpha = 1) of the batch against the loop."""
    import torch

    import synth
    import paper_2504_00959_gb300 as rick
    from paper_2504_00959_gb300 import build as rick_build
    rick_build.build()
    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", "0")))
    torch.cuda.set_device(dev)
    prob = synth.channels_problem(device=dev)
    q = dict(prob["params"], flags=synth.FLAG_CORRECT | synth.FLAG_REAL)
    offs = prob["offsets"]
    nchan, n = len(prob["ranges"]), q["n"]
    m = offs[-1]
    tile, group, prep_blocks, tune_ms = rick.autotune_batch(q, prob["ranges"], prob["vis"], prob["u"], prob["v"],
                                                            prob["w"], prob["wt"], offs)
    bi = rick.BatchImager(dict(q, tile=tile, plane_group=group), prob["ranges"])
    bi.set_prep_blocks(prep_blocks)
    out = torch.empty((nchan, n, n), device=dev)
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    props = torch.cuda.get_device_properties(dev)
    uuid = str(getattr(props, "uuid", ""))
    uuid = uuid if uuid.startswith("GPU-") else ("GPU-" + uuid if uuid else "")
    nvml = Nvml(uuid) if uuid else None
    with torch.cuda.stream(s):
        for _ in range(max(args.warmup, 1)):
            bi.images(prob["vis"], prob["u"], prob["v"], prob["w"], prob["wt"], offs, out=out, use_graph=True)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s.synchronize()
        j0 = nvml.energy_mj() if nvml else None
        e0.record(s)
        for _ in range(args.steps):
            bi.images(prob["vis"], prob["u"], prob["v"], prob["w"], prob["wt"], offs, out=out, use_graph=True)
        e1.record(s)
        s.synchronize()
        j1 = nvml.energy_mj() if nvml else None
    t_batch = e0.elapsed_time(e1) / args.steps
    batch_img = out.clone()
    # one more batched step outside the timed region, eagerly (not from the
    # graph) with the phase timers on: where the step's time goes
    with torch.cuda.stream(s):
        bi.set_timing(True)
        bi.images(prob["vis"], prob["u"], prob["v"], prob["w"], prob["wt"], offs, out=out, use_graph=False)
        s.synchronize()
        tb = bi.timing()
        bi.set_timing(False)
    batch_phases = {k: round(tb[k + "_ms"], 3) for k in ("prep", "grid", "fft", "colfft", "stack")}
    # the plain loop: one imager per channel, created once
    ims = [rick.Imager(dict(q, tile=tile, w_min=lo, w_max=hi)) for (lo, hi) in prob["ranges"]]
    loop_out = torch.empty_like(out)

    def loop_step():
        for c in range(nchan):
            a, b = offs[c], offs[c + 1]
            im = ims[c]
            im.reset()
            im.grid(prob["vis"][a:b], prob["u"][a:b], prob["v"][a:b], prob["w"][a:b], prob["wt"][a:b])
            im.image(out=loop_out[c])

    ksteps = max(1, min(args.steps, 10))
    loop_phases = []

    def time_loop():
        for _ in range(max(args.warmup, 1)):
            loop_step()
        torch.cuda.synchronize()
        # phase times of one loop step (timers on), then the timed steps (off)
        for im in ims:
            im.set_timing(True)
        loop_step()
        torch.cuda.synchronize()
        ph = dict.fromkeys(("prep", "grid", "fft", "colfft", "stack"), 0.0)
        for im in ims:
            tm = im.timing()
            for k in ph:
                ph[k] += tm[k + "_ms"]
            im.set_timing(False)
        loop_phases.append({k: round(v, 3) for k, v in ph.items()})
        f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        k0 = nvml.energy_mj() if nvml else None
        f0.record()
        for _ in range(ksteps):
            loop_step()
        f1.record()
        torch.cuda.synchronize()
        k1 = nvml.energy_mj() if nvml else None
        return f0.elapsed_time(f1) / ksteps, k0, k1

    # the per-channel loop with the library's default single-image path, and
    # with the split transform (the batch's); the faster one is the reference
    t_loop, k0, k1 = time_loop()
    loop_default = loop_out.clone()
    for im in ims:
        im.close()
    ims = [rick.Imager(dict(q, tile=tile, w_min=lo, w_max=hi, flags=q["flags"] | rick.FFT_SPLIT))
           for (lo, hi) in prob["ranges"]]
    t_loop_split, s0, s1 = time_loop()
    t_loop_default = t_loop
    loop_kind = "default single-image path"
    if t_loop_split < t_loop:
        t_loop, k0, k1, loop_kind = t_loop_split, s0, s1, "split transform"
        loop_phase = loop_phases[1]
    else:
        loop_out.copy_(loop_default)
        loop_phase = loop_phases[0]
    err = max(((batch_img[c] - loop_out[c]).abs().max() / loop_out[c].abs().max().clamp_min(1e-30)).item()
              for c in range(nchan))
    e_batch = (j1 - j0) / 1e3 / args.steps if j0 is not None and j1 is not None else None
    e_loop = (k1 - k0) / 1e3 / ksteps if k0 is not None and k1 is not None else None
    gp = None
    if e_batch and e_loop:
        gp = (t_loop / t_batch) / (e_batch / e_loop)
    for im in ims:
        im.close()
    bi.close()
    if rank == 0:
        print(json.dumps({
            "metric": "visibilities/sec, 64-channel batched imaging vs the per-channel loop",
            "value": m / (t_batch / 1e3), "unit": "vis/s", "higher_is_better": True, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_batch, "dtype": "f32",
            "data": "synthetic: 64 channels of an Earth-rotation synthesis, N(0,1) visibilities + a central source",
            "config": {"workload": "64 channels x 2048^2 x 16 w-planes, 1e6-2e7 visibilities per channel",
                       "nvis": m, "tile": tile, "plane_group": group, "prep_blocks_per_sm": prep_blocks or 8,
                       "autotune_ms": tune_ms},
            "loop_ms_per_step": t_loop, "loop_path": loop_kind, "speedup_vs_loop": t_loop / t_batch,
            "loop_ms_default_path": t_loop_default, "loop_ms_split_transform": t_loop_split,
            "batch_phases_ms": batch_phases, "loop_phases_ms": loop_phase,
            "max_rel_diff_batch_vs_loop": err, "energy_j_batch": e_batch, "energy_j_loop": e_loop,
            "green_productivity_eq4": gp}))


def run_adjoint(args, rank, world):
    """Differentiable imaging on the 4096^2 / 32-plane / 1e7 workload: one
    step is the dirty image D(V) and the gradient of L = ||D - t||^2 with
    respect to V through the hand-written adjoint (torch.autograd.Function
    whose backward recomputes the w-planes from dL/dD and degrids them).
    The target t is the image of the same measurements with every
    visibility scaled by 1 + 0.1 N(0, 1) (a perturbed sky)."""
    import torch

    import synth
    import paper_2504_00959_gb300 as rick
    from paper_2504_00959_gb300 import build as rick_build
    rick_build.build()
    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", "0")))
    torch.cuda.set_device(dev)
    prob = synth.config2(device=dev, m=args.nvis or 10_000_000, nw=args.nw or 32)
    params = dict(prob["params"], flags=synth.FLAG_CORRECT | synth.FLAG_REAL, tile=args.tile)
    im = rick.Imager(params, device=dev)
    m = prob["u"].numel()
    n, nw = params["n"], params["nw"]
    g = torch.Generator(device=dev).manual_seed(synth.BASE_SEED + 5)
    scale = 1.0 + 0.1 * torch.randn(m, device=dev, generator=g)
    with torch.no_grad():
        target = rick.dirty_image(prob["vis"] * scale, prob["u"], prob["v"], prob["w"], prob["wt"], im).clone()
    vis = prob["vis"].clone().requires_grad_(True)

    def step():
        vis.grad = None
        d = rick.dirty_image(vis, prob["u"], prob["v"], prob["w"], prob["wt"], im)
        loss = ((d - target) ** 2).sum()
        loss.backward()
        return loss

    for _ in range(max(args.warmup, 1)):
        step()
    torch.cuda.synchronize()
    props = torch.cuda.get_device_properties(dev)
    uuid = str(getattr(props, "uuid", ""))
    uuid = uuid if uuid.startswith("GPU-") else ("GPU-" + uuid if uuid else "")
    nvml = Nvml(uuid) if uuid else None
    clocks = ClockSampler(uuid if uuid else 0)
    im.set_timing(True)
    s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    clocks.start()
    j0 = nvml.energy_mj() if nvml else None
    s0.record()
    for _ in range(args.steps):
        step()
    s1.record()
    torch.cuda.synchronize()
    j1 = nvml.energy_mj() if nvml else None
    clk = clocks.stop()
    ms = s0.elapsed_time(s1) / max(args.steps, 1)
    tm = im.timing()
    st = im.stats()
    peak, peak_kind = _peaks()
    # backward = spread (8 B/cell written) + forward FFT (two passes, read +
    # write) + gather (planes read once, 16 B of u, v, w, weight + 8 B of
    # gradient per measurement) + the measurement sort (two passes of 16 B)
    deg_ms = tm["degrid_ms"] / max(tm["degrid_calls"], 1)
    deg_bytes = 8.0 * nw * n * n + 32.0 * nw * n * n + 8.0 * nw * n * n + 24.0 * m + 32.0 * m
    fwd_ms = (tm["prep_ms"] + tm["grid_ms"] + tm["fft_ms"] + tm["stack_ms"]) / max(tm["stack_calls"], 1)
    if rank == 0:
        print(json.dumps({
            "metric": "visibilities/sec, dirty image + loss gradient through the adjoint degridder",
            "value": m / (ms / 1e3), "unit": "vis/s", "higher_is_better": True, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "dtype": "f32", "data": DATA["wstack"],
            "config": {"workload": "differentiable imaging: " + WORKLOADS["wstack"], "n": n, "nw": nw, "nvis": m,
                       "tile": st["tile"], "plane_group": st["plane_group"],
                       "loss": "sum (D - t)^2, t = image of V (1 + 0.1 N(0,1))"},
            "phases": {"forward_ms": fwd_ms, "backward_degrid_ms": deg_ms,
                       "backward_algorithmic_gb": deg_bytes / 1e9,
                       "backward_gbs": deg_bytes / deg_ms / 1e6,
                       "backward_frac_of_" + peak_kind: deg_bytes / deg_ms / 1e6 / peak},
            "energy_j_per_solution": (j1 - j0) / 1e3 / max(args.steps, 1) if j0 is not None and j1 is not None
            else None,
            "gpu_launches": int(tm["kernel_launches"]), "clocks": clk}))
    im.close()


def run_small(args, rank, world):
    """The 256^2 / 8-plane / 1e5-measurement image (2 degree field, Gaussian
    support 7): bound by launch latency, so reported in microseconds per
    image, from CUDA events around the steps and from the host clock."""
    import torch

    import synth
    import paper_2504_00959_gb300 as rick
    from paper_2504_00959_gb300 import build as rick_build
    rick_build.build()
    if rank != 0:
        return
    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", "0")))
    torch.cuda.set_device(dev)
    prob = synth.config1(device=dev)
    params = dict(prob["params"], flags=synth.FLAG_CORRECT | synth.FLAG_REAL, tile=args.tile)
    im = rick.Imager(params, device=dev)
    n, nw = params["n"], params["nw"]
    m = prob["u"].numel()
    img = torch.empty((n, n), dtype=torch.float32, device=dev)

    def step():
        im.reset()
        im.grid(prob["vis"], prob["u"], prob["v"], prob["w"], prob["wt"])
        im.image(out=img)

    for _ in range(max(args.warmup, 3)):
        step()
    torch.cuda.synchronize()
    im.set_timing(False)
    s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    steps = max(args.steps, 1)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    s0.record()
    for _ in range(steps):
        step()
    s1.record()
    torch.cuda.synchronize()
    host_us = (time.perf_counter() - t0) / steps * 1e6
    dev_us = s0.elapsed_time(s1) / steps * 1e3
    im.set_timing(True)
    step()
    torch.cuda.synchronize()
    tm = im.timing()
    st = im.stats()
    im.close()
    print(json.dumps({
        "metric": "microseconds per image, 256^2 x 8 planes x 1e5 visibilities", "value": dev_us, "unit": "us",
        "higher_is_better": False, "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": dev_us / 1e3, "dtype": "f32",
        "data": "synthetic: uv uniform in a disk of radius 0.45 N du, w uniform in [-50, 50], "
                "N(0,1) visibilities + a unit source at the phase centre",
        "config": {"workload": "256x256 grid, 8 w-planes, 1e5 visibilities, 2 degree field, Gaussian support 7, "
                               "FP32 (launch-latency bound)", "n": n, "nw": nw, "nvis": m, "tile": st["tile"],
                   "plane_group": st["plane_group"]},
        "host_us_per_image": host_us, "visibilities_per_s": m / (dev_us / 1e6),
        "gpu_launches_per_image": int(tm["kernel_launches"])}))


def run_dense_channel(args, rank, world):
    """The densest channel of the 64-channel workload imaged alone: 2048^2 x
    16 w-planes, 2e7 measurements of the same Earth-rotation track (256
    antennas in a 20 km disk, 6 h of 10 s integrations, dec -30) at its top
    frequency, 1.75 GHz, with the uv cell set by the longest baseline at 0.45
    n cells; Kaiser-Bessel support 7.  Most of its gridding entries fall in
    tiles of hundreds to tens of thousands of entries (the heavy-tile path).
    Milliseconds per image and the gridding phase, CUDA events."""
    import torch

    import synth
    import paper_2504_00959_gb300 as rick
    from paper_2504_00959_gb300 import build as rick_build
    rick_build.build()
    if rank != 0:
        return
    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", "0")))
    torch.cuda.set_device(dev)
    prob = synth.earth_rotation_problem(2048, 16, 20_000_000, synth.KERNEL_KB, 7, 256, 20_000.0, 6.0, 10.0, 1.75e9,
                                        -30.0, synth.BASE_SEED + 5, device=dev)
    params = dict(prob["params"], flags=synth.FLAG_CORRECT | synth.FLAG_REAL, tile=args.tile)
    im = rick.Imager(params, device=dev)
    n, nw = params["n"], params["nw"]
    m = prob["u"].numel()
    img = torch.empty((n, n), dtype=torch.float32, device=dev)

    def step():
        im.reset()
        im.grid(prob["vis"], prob["u"], prob["v"], prob["w"], prob["wt"])
        im.image(out=img)

    for _ in range(max(args.warmup, 3)):
        step()
    torch.cuda.synchronize()
    im.set_timing(False)
    s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    steps = max(args.steps, 1)
    s0.record()
    for _ in range(steps):
        step()
    s1.record()
    torch.cuda.synchronize()
    ms = s0.elapsed_time(s1) / steps
    im.set_timing(True)
    step()
    torch.cuda.synchronize()
    tm = im.timing()
    st = im.stats()
    im.close()
    print(json.dumps({
        "metric": "visibilities per second, one dense 2048^2 x 16-plane channel", "value": m / (ms / 1e3),
        "unit": "vis/s", "higher_is_better": True, "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms, "dtype": "f32",
        "data": "synthetic: seeded Earth-rotation track, 200 point sources + N(0, 0.1) noise",
        "config": {"workload": "densest channel of the 64-channel set alone: 2048x2048 grid, 16 w-planes, "
                               "2e7 visibilities at 1.75 GHz, Kaiser-Bessel support 7, FP32", "n": n, "nw": nw,
                   "nvis": m, "tile": st["tile"], "plane_group": st["plane_group"]},
        "phases_ms": {k: round(tm[k + "_ms"], 4) for k in ("prep", "grid", "fft", "colfft", "stack")},
        "gpu_launches": int(tm["kernel_launches"])}))


def run_reference(args, rank, world):
    """The FP64 oracle on the host cores, on the same workload as the GPU arm:
    every step is one bounded sample (oracle_round: placement and gridding of
    a slice of the measurements, one plane's transform and screen), and the
    value is the whole image's rate from the median step's unit costs
    (oracle_image_seconds).  ms_per_step is the measured time of a sample
    step.  Rank 0 only; the other ranks exit without work."""
    if rank != 0:
        return
    wl = args.workload
    if wl not in WORKLOADS:
        print(json.dumps({"impl": "reference", "unavailable": "the oracle baseline covers the single-image "
                                                               "workloads (large, wstack) only"}))
        return
    import numpy as np

    import synth
    import oracle
    oracle.lib()
    prob, params = make_problem(wl, "cpu", args.nvis or None, args.nw or None)
    prob_np = synth.to_numpy(prob)
    del prob
    prob_np["params"] = dict(params)
    q = prob_np["params"]
    m = prob_np["u"].shape[0]
    k, _, _ = oracle.place(q, prob_np["u"], prob_np["v"], prob_np["w"])
    ok = (k >= 0) & np.isfinite(prob_np["wt"]) & np.isfinite(prob_np["vis"].real) & \
        np.isfinite(prob_np["vis"].imag)
    m_gridded = int(ok.sum())
    nw = int(q["nw"])
    plane, idx = oracle_plane_sample(prob_np)
    secs, walls, rounds = [], [], []
    for i in range(args.warmup + args.steps):
        r = oracle_round(prob_np, plane, idx)
        if i >= args.warmup:
            rounds.append(r)
            secs.append(oracle_image_seconds(r, m, m_gridded, nw))
            walls.append(r["wall"])
    med = statistics.median(secs) if secs else None
    value = m / med if med else None
    threads = oracle.num_threads()
    r = rounds[secs.index(med)] if med in secs else (rounds[0] if rounds else None)
    desc = ("per step: weights + placement of %d measurements (1 thread), gridding of the %d measurements on "
            "plane %d (1 thread), one plane's zeroing + FFT + screen at %d^2 (%d threads%s); value from the median "
            "step's unit costs: image = %d weight pass(es) + %d x (placement pass of %d + plane) + gridding of %d + "
            "finalisation (estimates %s s)" % (
                r["slice"], r["on_plane"], plane, r["n_s"], threads,
                (", x%.1f for %d^2 by n^2 log n^2" % (r["fft_scale"], q["n"])) if r["n_s"] != q["n"] else "",
                r["passes_w"], nw, m, m_gridded, ", ".join("%.0f" % x for x in secs))) if r else ""
    ms_step = statistics.mean(walls) * 1e3 if walls else None
    out = {
        "metric": METRIC, "value": value, "unit": "vis/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": DATA[wl], "impl": "reference",
        "config": workload_config(wl, params, m, world, args),
        "cpu_baseline": {"value": value, "unit": "vis/s", "cores": threads, "kind": "oracle", "sample": desc,
                         "threads_by_phase": {"placement_and_gridding": 1, "fft_and_screen": threads},
                         "image_seconds_estimate": med},
        "e2e": {"value": value, "unit": "vis/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    del np
    print(json.dumps(out))


if __name__ == "__main__":
    main()
