"""Benchmark of the w-stacking imager hot path on GB300.

One step = the whole path for one dirty image of the 4096^2 / 32 w-plane /
1e7-visibility workload (256 antennas in a 20 km disk, 6 h Earth-rotation
synthesis at dec -30, 10 s integrations, 1.4 GHz, 200-source sky + noise,
Kaiser-Bessel support 7): reset, placement + counting sort, gridding of all
planes, per-plane inverse FFT, phase-screen stack and finalisation.  Inputs
are resident in HBM when the timed region starts; the planes (4.3 GB) are
larger than L2, so no L2 flush is needed.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Multi-GPU (torchrun): every rank images its own copy of the workload (the path
has no exchange step: replicas, weak scaling); value = all ranks' visibilities
/ the slowest rank's time.  ``--impl reference`` times the FP64 CPU oracle on
the host cores on a bounded sample of the same workload (rank 0 only).
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
WORKLOAD = ("plain w-stacking, 4096x4096 grid, 32 w-planes, 1e7 visibilities (256 antennas, 20 km disk, "
            "6 h synthesis, dec -30, 10 s, 1.4 GHz, 200 sources + noise), Kaiser-Bessel support 7, FP32")
DATA = "synthetic: seeded Earth-rotation synthesis + point-source sky (the paper's LOFAR data is not available)"


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
def oracle_sample(prob_np, planes):
    """Time the FP64 oracle on planes [k0, k1) of the full workload: gridding
    (all measurements placed, those of the sample planes gridded) and the
    FFT + stack of the sample planes; extrapolate to the whole workload
    (gridding by the number of measurements, FFT + stack by the number of
    planes).  Returns (visibilities/s, sample description, threads)."""
    import numpy as np

    import oracle
    p = prob_np
    q = p["params"]
    k0, k1 = planes
    k, _, _ = oracle.place(q, p["u"], p["v"], p["w"])
    m_all = int((k >= 0).sum())
    m_s = int(((k >= k0) & (k < k1)).sum())
    t0 = time.perf_counter()
    oracle.grid(q, p["u"], p["v"], p["w"], p["wt"], p["vis"], k0=k0, k1=k1)
    t_grid = time.perf_counter() - t0
    t0 = time.perf_counter()
    oracle.dirty_image(q, p["u"], p["v"], p["w"], p["wt"], p["vis"], k0=k0, k1=k1)
    t_full = time.perf_counter() - t0
    t_rest = max(t_full - t_grid, 0.0)
    t_est = t_grid * (m_all / max(m_s, 1)) + t_rest * (q["nw"] / (k1 - k0))
    desc = (f"planes {k0}-{k1 - 1} of {q['nw']} ({m_s} of {m_all} visibilities gridded, all placed): "
            f"grid {t_grid:.2f} s scaled x{m_all / max(m_s, 1):.1f}, FFT+stack {t_rest:.2f} s scaled "
            f"x{q['nw'] / (k1 - k0):.0f}; measured {t_grid + t_full:.1f} s")
    del np
    return m_all / t_est, desc, oracle.num_threads(), t_grid + t_full


# ------------------------------------------------------------------ main
def aggregate(ms_local, units_per_step, steps, world, device):
    """Slowest rank's timed-region milliseconds and the whole-job throughput:
    every rank processes units_per_step units per step (replicas, weak
    scaling), value = world * units_per_step * steps / slowest time."""
    import torch
    import torch.distributed as dist
    ms = float(ms_local)
    if world > 1:
        t = torch.tensor([ms], device=device, dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    return ms, world * units_per_step * steps / (ms / 1e3)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--nvis", type=int, default=10_000_000)
    ap.add_argument("--nw", type=int, default=32, help="w-planes (profiling cases)")
    ap.add_argument("--tile", type=int, default=0, help="gridder tile side (0 = automatic)")
    ap.add_argument("--fold", action="store_true",
                    help="Hermitian fold (real image): measurements with w < 0 mirrored, half the w-planes "
                         "over [0, max |w|] at the same plane spacing")
    ap.add_argument("--w-support", type=int, default=0,
                    help="planes per measurement (Eq. 3's kernel in w); the plane range is padded by "
                         "nw / (nw - w_support) so every footprint lies on the planes")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true", help="skip the host-buffer end-to-end leg")
    ap.add_argument("--workload", choices=["wstack", "channels", "adjoint", "large", "small"], default="wstack",
                    help="wstack: the 4096^2 / 32-plane / 1e7 image (default); channels: 64 channels "
                         "batched vs imaged one by one; adjoint: image + loss gradient through the "
                         "adjoint degridder on the same workload; large: 16384^2 / 128 planes / 2e8 "
                         "measurements with uniform weighting, in plane groups; small: 256^2 / 8 planes / "
                         "1e5, microseconds per image")
    args = ap.parse_args()

    import torch
    import torch.distributed as dist

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        return run_reference(args, rank, world)
    if args.workload == "channels":
        return run_channels(args, rank, world)
    if args.workload == "adjoint":
        return run_adjoint(args, rank, world)
    if args.workload == "large":
        return run_large(args, rank, world)
    if args.workload == "small":
        return run_small(args, rank, world)

    import synth
    import paper_2504_00959_gb300 as rick
    from paper_2504_00959_gb300 import build as rick_build
    rick_build.build()

    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    if world > 1:
        dist.init_process_group("nccl", device_id=dev)

    prob = synth.config2(device=dev, m=args.nvis, nw=args.nw)
    params = dict(prob["params"], flags=synth.FLAG_CORRECT | synth.FLAG_REAL, tile=args.tile)
    if args.fold:
        wabs = max(abs(params["w_min"]), abs(params["w_max"]))
        params = dict(params, nw=max(args.nw // 2, 1), w_min=0.0, w_max=wabs,
                      flags=params["flags"] | synth.FLAG_FOLD)
    if args.w_support > 1:
        lo, hi, nwp = params["w_min"], params["w_max"], params["nw"]
        mid, half = 0.5 * (lo + hi), 0.5 * (hi - lo) * nwp / (nwp - args.w_support)
        params = dict(params, w_min=mid - half, w_max=mid + half, w_support=args.w_support)
    im = rick.Imager(params, device=dev)
    img = torch.empty((params["n"], params["n"]), dtype=torch.float32, device=dev)
    m = prob["u"].numel()

    def step():
        im.reset()
        im.grid(prob["vis"], prob["u"], prob["v"], prob["w"], prob["wt"])
        im.image(out=img)

    for _ in range(max(args.warmup, 0)):
        step()
    torch.cuda.synchronize()
    st = im.stats()

    props = torch.cuda.get_device_properties(dev)
    uuid = str(getattr(props, "uuid", ""))
    uuid = uuid if uuid.startswith("GPU-") else ("GPU-" + uuid if uuid else "")
    nvml = Nvml(uuid) if uuid else None
    clocks = ClockSampler(uuid if uuid else local)
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
    ms, value = aggregate(ms, m, args.steps, world, dev)
    ms_step = ms / max(args.steps, 1)

    # ------------------------------------------------ roofline (gridder)
    peak, peak_kind = _peaks()
    n, nw = params["n"], params["nw"]
    grid_launch_ms = tm["grid_ms"] / max(tm["grid_calls"], 1)
    grid_bytes = 16.0 * st["n_gridded"] + 8.0 * nw * n * n
    achieved = grid_bytes / (grid_launch_ms / 1e3) / 1e9
    # the committed DRAM counters were taken on the 4096^2 x 32 x 1e7 workload only
    default_size = (n, nw, m) == (4096, 32, 10_000_000) and params.get("w_support", 1) <= 1 \
        and not params["flags"] & synth.FLAG_FOLD
    traffic = _traffic("rick_grid.cu", "k_grid@4096x32x1e7") if default_size else None
    stack_ms = tm["stack_ms"] / max(tm["stack_calls"], 1)
    stack_bytes = 8.0 * nw * n * n + 4.0 * n * n
    fft_ms = tm["fft_ms"] / max(tm["fft_calls"], 1)
    fft_bytes = 2 * 2 * 8.0 * nw * n * n  # two passes, read + write
    prep_ms = tm["prep_ms"] / max(tm["prep_calls"], 1)
    prep_bytes = 2 * 24.0 * m + 16.0 * st["n_entries"]
    phases = {
        "prep": {"ms": prep_ms, "algorithmic_gb": prep_bytes / 1e9, "gbs": prep_bytes / prep_ms / 1e6},
        "grid": {"ms": grid_launch_ms, "algorithmic_gb": grid_bytes / 1e9, "gbs": achieved},
        "fft_cufft": {"ms": fft_ms, "algorithmic_gb": fft_bytes / 1e9, "gbs": fft_bytes / fft_ms / 1e6},
        "stack": {"ms": stack_ms, "algorithmic_gb": stack_bytes / 1e9, "gbs": stack_bytes / stack_ms / 1e6},
    }
    for v in phases.values():
        v["frac_of_" + peak_kind] = v["gbs"] / peak

    # ------------------------------------------------ end to end, host buffers
    e2e = None
    if not args.no_e2e:
        hv = prob["vis"].cpu().pin_memory()
        hu, hvv, hw, hwt = (prob[k].cpu().pin_memory() for k in ("u", "v", "w", "wt"))
        himg = torch.empty((n, n), dtype=torch.float32).pin_memory()
        himg2 = torch.empty((n, n), dtype=torch.float32).pin_memory()
        im.image_host(hv, hu, hvv, hw, hwt, out=himg)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ksteps = max(min(args.steps, 5), 1)
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

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        prob_np = synth.to_numpy(prob)
        v, desc, threads, secs = oracle_sample(prob_np, (15, 17))
        cpu = {"value": v, "unit": "vis/s", "cores": threads, "kind": "oracle", "sample": desc}

    energy = None
    if e0 is not None and e1 is not None:
        energy = (e1 - e0) / 1e3 / max(args.steps, 1)

    out = {
        "metric": METRIC, "value": value, "unit": "vis/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": DATA,
        "config": {"workload": WORKLOAD + ("; Hermitian fold: %d w-planes over [0, max |w|]" % nw if args.fold
                                           else "") +
                   ("; w-support %d on %d planes" % (args.w_support, nw) if args.w_support > 1 else ""),
                   "n": n, "nw": nw, "nvis": m, "kernel": "kaiser-bessel", "support": 7,
                   "tile": st["tile"], "plane_group": st["plane_group"],
                   "l2": "inputs larger than L2 (%.2f GB of planes written and read every step)" % (8.0 * nw * n * n / 1e9),
                   "parallelism": "replicas" if world > 1 else "single GPU"},
        "roofline": None,
        "roofline_other": None,
        "phases": phases,
        "energy_j_per_solution": energy,
        "e2e": e2e,
        "cpu_baseline": cpu,
        "gpu_launches": int(tm["kernel_launches"]),
        "clocks": clk,
        "roofline_frac_end_to_end": None,
    }
    # roofline of our dominant kernel (the longer of the gridder and the stack)
    # in `roofline`, the other in `roofline_other`
    rl_grid = {"kernel": "k_grid_tiles + k_grid_chunks (gridding, Eq. 3)", "bound": "hbm", "achieved": achieved,
               "peak": peak, "unit": "GB/s", "frac": achieved / peak, "traffic": traffic, "peak_kind": peak_kind,
               "algorithmic_bytes_per_launch": grid_bytes, "launch_ms": grid_launch_ms}
    split = n == 4096  # the library's default transform path at this size (cuFFT + k_colstack)
    stack_name = ("k_colstack (last 16-point column factor + w-screen + stack, Eq. 1)" if split
                  else "k_stack (w-screen + stack, Eq. 1)")
    stack_traffic = _traffic("rick_stack.cu", "k_colstack@4096x32x1e7") if (default_size and split) else None
    rl_stack = {"kernel": stack_name, "bound": "hbm", "achieved": stack_bytes / stack_ms / 1e6, "peak": peak,
                "unit": "GB/s", "frac": stack_bytes / stack_ms / 1e6 / peak, "traffic": stack_traffic,
                "peak_kind": peak_kind, "algorithmic_bytes_per_launch": stack_bytes, "launch_ms": stack_ms}
    if stack_ms > grid_launch_ms:
        out["roofline"], out["roofline_other"] = rl_stack, rl_grid
    else:
        out["roofline"], out["roofline_other"] = rl_grid, rl_stack
    # whole step against HBM: inputs + plane write + FFT (2 passes) + stack read + image
    step_bytes = 24.0 * m + 8.0 * nw * n * n + fft_bytes + stack_bytes
    out["roofline_frac_end_to_end"] = step_bytes / (ms_step / 1e3) / 1e9 / peak
    if rank == 0:
        print(json.dumps(out))
    im.close()
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
    tile, group, tune_ms = rick.autotune_batch(q, prob["ranges"], prob["vis"], prob["u"], prob["v"], prob["w"],
                                               prob["wt"], offs)
    bi = rick.BatchImager(dict(q, tile=tile, plane_group=group), prob["ranges"])
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

    for _ in range(max(args.warmup, 1)):
        loop_step()
    torch.cuda.synchronize()
    ksteps = max(1, min(args.steps, 10))
    f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    k0 = nvml.energy_mj() if nvml else None
    f0.record()
    for _ in range(ksteps):
        loop_step()
    f1.record()
    torch.cuda.synchronize()
    k1 = nvml.energy_mj() if nvml else None
    t_loop = f0.elapsed_time(f1) / ksteps
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
                       "nvis": m, "tile": tile, "plane_group": group, "autotune_ms": tune_ms},
            "loop_ms_per_step": t_loop, "speedup_vs_loop": t_loop / t_batch,
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
    prob = synth.config2(device=dev, m=args.nvis, nw=args.nw)
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
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "dtype": "f32", "data": DATA,
            "config": {"workload": "differentiable imaging: " + WORKLOAD, "n": n, "nw": nw, "nvis": m,
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


def run_large(args, rank, world):
    """The 16384^2 / 128-plane / 2e8-measurement image with uniform weighting
    (5 degree field, Kaiser-Bessel support 8): the planes (275 GB) do not fit
    at once, so every step grids, transforms and stacks plane group after
    plane group, re-reading the measurements for each group.  Reported
    beside the default line, not instead of it."""
    import torch

    import synth
    import paper_2504_00959_gb300 as rick
    from paper_2504_00959_gb300 import build as rick_build
    rick_build.build()
    if rank != 0:
        return
    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", "0")))
    torch.cuda.set_device(dev)
    prob = synth.config3(device=dev)
    params = dict(prob["params"], tile=args.tile)
    im = rick.Imager(params, device=dev)
    n, nw = params["n"], params["nw"]
    m = prob["u"].numel()
    img = torch.empty((n, n), dtype=torch.float32, device=dev)

    def step():
        im.reset()
        im.grid(prob["vis"], prob["u"], prob["v"], prob["w"], prob["wt"])
        im.image(out=img)

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
    im.close()
    peak, peak_kind = _peaks()
    steps = max(args.steps, 1)
    groups = -(-nw // max(st["plane_group"], 1))
    cells = float(nw) * n * n
    grid_ms = tm["grid_ms"] / steps
    grid_bytes = 16.0 * st["n_gridded"] + 8.0 * cells
    phases = {
        # every plane group sorts all measurements again: two passes of 24 B each
        "prep": (tm["prep_ms"] / steps, groups * 2 * 24.0 * m + 16.0 * st["n_entries"]),
        "grid": (grid_ms, grid_bytes),
        "fft_cufft": (tm["fft_ms"] / steps, 2 * 2 * 8.0 * cells),
        "stack": (tm["stack_ms"] / steps, 8.0 * cells + 2 * 8.0 * n * n * groups),
    }
    ph = {k: {"ms": t, "algorithmic_gb": b / 1e9, "gbs": b / t / 1e6, "frac_of_" + peak_kind: b / t / 1e6 / peak}
          for k, (t, b) in phases.items() if t > 0}
    print(json.dumps({
        "metric": "visibilities/sec end-to-end (grid+FFT+w-stack), 16384^2 x 128 planes, uniform weighting",
        "value": m / (ms / 1e3), "unit": "vis/s", "higher_is_better": True, "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "dtype": "f32",
        "data": "synthetic: seeded Earth-rotation synthesis (512 antennas, 60 km, 8 h, dec -45, 1.4 GHz), "
                "N(0,1) visibilities + a unit source at the phase centre",
        "config": {"workload": "16384x16384 grid, 128 w-planes in groups, 2e8 visibilities, 5 degree field, "
                               "Kaiser-Bessel support 8, uniform weighting, FP32",
                   "n": n, "nw": nw, "nvis": m, "support": params["support"], "tile": st["tile"],
                   "plane_group": st["plane_group"], "plane_groups": groups,
                   "l2": "inputs larger than L2 (%.0f GB of planes per step)" % (8.0 * cells / 1e9)},
        "roofline": {"kernel": "k_grid (gridding, Eq. 3)", "bound": "hbm", "achieved": grid_bytes / grid_ms / 1e6,
                     "peak": peak, "unit": "GB/s", "frac": grid_bytes / grid_ms / 1e6 / peak, "traffic": None,
                     "peak_kind": peak_kind, "algorithmic_bytes_per_step": grid_bytes, "grid_ms_per_step": grid_ms},
        "phases": ph,
        "roofline_frac_end_to_end": sum(b for _, b in phases.values()) / (ms / 1e3) / 1e9 / peak,
        "energy_j_per_solution": (j1 - j0) / 1e3 / steps if j0 is not None and j1 is not None else None,
        "gpu_launches": int(tm["kernel_launches"]), "clocks": clk}))


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


def run_reference(args, rank, world):
    """The FP64 oracle on the host cores: every step images a bounded sample
    (one w-plane of the full workload), extrapolated to the whole workload."""
    if rank != 0:
        return
    import synth
    import oracle
    oracle.lib()
    prob = synth.to_numpy(synth.config2(device="cpu", m=args.nvis))
    vals = []
    t_all = 0.0
    desc = ""
    threads = oracle.num_threads()
    for i in range(args.warmup + args.steps):
        v, desc, threads, secs = oracle_sample(prob, (16, 17))
        if i >= args.warmup:
            vals.append(v)
            t_all += secs
    value = statistics.median(vals) if vals else None
    m = prob["u"].shape[0]
    out = {
        "metric": METRIC, "value": value, "unit": "vis/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": (m / value * 1e3) if value else None, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": DATA, "impl": "reference",
        "config": {"workload": WORKLOAD, "n": prob["params"]["n"], "nw": prob["params"]["nw"], "nvis": m},
        "cpu_baseline": {"value": value, "unit": "vis/s", "cores": threads, "kind": "oracle", "sample": desc},
        "e2e": {"value": value, "unit": "vis/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(out))


if __name__ == "__main__":
    main()
