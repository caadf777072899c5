"""GB300 (sm_103a) w-stacking imager -- the hot path of RICK (arXiv 2504.00959).

Python binding over the C ABI of ``librick.so`` (include/rick.h).  PyTorch is
used for device memory and streams only; gridding (Eq. 3), the per-plane
inverse FFT (cuFFT), the w-term phase-screen stack (Eq. 1) and the adjoint
degridder all run in the library.  There is no CPU fallback: constructing an
``Imager`` without the built library, or with tensors that are not on a CUDA
device, raises.

Parameters are a mapping with keys ``n``, ``nw``, ``pixel_rad``, ``w_min``,
``w_max``, ``kernel`` (0 Gaussian, 1 Kaiser-Bessel), ``support``,
``kernel_param`` (0 = default sigma S/6 / beta 2.34 S), ``flags``
(GRID_CORRECT | REAL_IMAGE | APPLY_N | UNIFORM_WEIGHT | HERMITIAN_FOLD), and optionally
``plane_group``, ``tile`` and ``w_support``.
"""
import ctypes

import torch

from . import _lib
from ._lib import (APPLY_N, FFT_2D, FFT_SPLIT, GRID_CORRECT, HERMITIAN_FOLD, KERNEL_GAUSS, KERNEL_KB,  # noqa: F401
                   REAL_IMAGE, UNIFORM_WEIGHT,
                   RickError)

__all__ = ["Imager", "BatchImager", "autotune_batch", "DirtyImage", "dirty_image", "RickError", "load",
           "KERNEL_GAUSS", "KERNEL_KB",
           "GRID_CORRECT", "REAL_IMAGE", "APPLY_N", "UNIFORM_WEIGHT", "HERMITIAN_FOLD", "FFT_2D", "FFT_SPLIT"]


def load():
    """Load librick.so (raises when it is not built)."""
    return _lib.load()


def _params_struct(p):
    rp = _lib.RickParams()
    rp.n = int(p["n"])
    rp.nw = int(p["nw"])
    rp.pixel_rad = float(p["pixel_rad"])
    rp.w_min = float(p["w_min"])
    rp.w_max = float(p["w_max"])
    rp.kernel = int(p["kernel"])
    rp.support = int(p["support"])
    rp.kernel_param = float(p.get("kernel_param", 0.0) or 0.0)
    rp.plane_group = int(p.get("plane_group", 0) or 0)
    rp.tile = int(p.get("tile", 0) or 0)
    rp.flags = int(p.get("flags", GRID_CORRECT | REAL_IMAGE))
    rp.w_support = int(p.get("w_support", 0) or 0)
    return rp


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else ctypes.c_void_p(None)


class Imager:
    """One w-stacking problem (grid size, pixel scale, w-planes, kernel) on one GPU.

    ``grid`` may be called once per chunk of measurements; ``image`` runs the
    per-plane FFT and the w-stack for everything gridded since ``reset``.
    All work goes to the current torch CUDA stream of the imager's device.
    """

    def __init__(self, params, device=None):
        self.params = dict(params)
        self._L = _lib.load()
        if device is None:
            device = torch.device("cuda", torch.cuda.current_device())
        self.device = torch.device(device)
        if self.device.type != "cuda":
            raise ValueError("Imager needs a CUDA device")
        if self.device.index is None:
            self.device = torch.device("cuda", torch.cuda.current_device())
        self._rp = _params_struct(self.params)
        h = ctypes.c_void_p()
        with torch.cuda.device(self.device):
            _lib.check(self._L.rick_create(ctypes.byref(self._rp), ctypes.byref(h)))
        self._h = h
        self.generation = 0

    # -------------------------------------------------------------- helpers
    @property
    def n(self):
        return self._rp.n

    @property
    def real(self):
        return bool(self._rp.flags & REAL_IMAGE)

    def _sync_stream(self):
        s = torch.cuda.current_stream(self.device).cuda_stream
        _lib.check(self._L.rick_set_stream(self._h, ctypes.c_void_p(s)), self._h)

    def _vec(self, t, name, dtype, m=None):
        if t is None:
            return None
        if not isinstance(t, torch.Tensor) or t.device != self.device:
            raise ValueError(f"{name} must be a tensor on {self.device}")
        if t.dtype != dtype:
            raise ValueError(f"{name} must be {dtype} (got {t.dtype})")
        if not t.is_contiguous():
            raise ValueError(f"{name} must be contiguous")
        if m is not None and t.numel() != m:
            raise ValueError(f"{name} has {t.numel()} elements, expected {m}")
        return t

    def _inputs(self, vis, u, v, w, wt):
        m = u.numel()
        return (self._vec(vis, "vis", torch.complex64, m), self._vec(u, "u", torch.float32, m),
                self._vec(v, "v", torch.float32, m), self._vec(w, "w", torch.float32, m),
                self._vec(wt, "wt", torch.float32, m), m)

    # ------------------------------------------------------------------ API
    def reset(self):
        self._sync_stream()
        _lib.check(self._L.rick_reset(self._h), self._h)
        self.generation += 1

    def add_density(self, vis, u, v, w, wt=None):
        vis, u, v, w, wt, m = self._inputs(vis, u, v, w, wt)
        self._sync_stream()
        _lib.check(self._L.rick_add_density(self._h, _ptr(vis), _ptr(u), _ptr(v), _ptr(w), _ptr(wt), m), self._h)

    def grid(self, vis, u, v, w, wt=None):
        vis, u, v, w, wt, m = self._inputs(vis, u, v, w, wt)
        self._sync_stream()
        _lib.check(self._L.rick_grid(self._h, _ptr(vis), _ptr(u), _ptr(v), _ptr(w), _ptr(wt), m), self._h)
        self.generation += 1

    def image(self, out=None):
        n = self.n
        if out is None:
            out = torch.empty((n, n), dtype=torch.float32 if self.real else torch.complex64, device=self.device)
        self._vec(out, "out", torch.float32 if self.real else torch.complex64, n * n)
        self._sync_stream()
        _lib.check(self._L.rick_fft_and_stack(self._h, _ptr(out)), self._h)
        return out

    def grid_planes(self, k0=0, nk=None):
        nk = self._rp.nw - k0 if nk is None else nk
        out = torch.empty((nk, self.n, self.n), dtype=torch.complex64, device=self.device)
        self._sync_stream()
        _lib.check(self._L.rick_grid_planes(self._h, int(k0), int(nk), _ptr(out)), self._h)
        return out

    def degrid(self, image_grad, u, v, w, wt=None, out=None):
        n = self.n
        m = u.numel()
        image_grad = self._vec(image_grad.contiguous(), "image_grad",
                               torch.float32 if self.real else torch.complex64, n * n)
        u, v, w = (self._vec(u, "u", torch.float32, m), self._vec(v, "v", torch.float32, m),
                   self._vec(w, "w", torch.float32, m))
        wt = self._vec(wt, "wt", torch.float32, m)
        if out is None:
            out = torch.empty(m, dtype=torch.complex64, device=self.device)
        self._vec(out, "out", torch.complex64, m)
        self._sync_stream()
        _lib.check(self._L.rick_degrid(self._h, _ptr(image_grad), _ptr(u), _ptr(v), _ptr(w), _ptr(wt), m,
                                       _ptr(out)), self._h)
        return out

    def predict(self, model, u, v, w, out=None):
        """Model visibilities (complex64 [m]) of the model image at (u, v, w):
        the measurement equation evaluated by degridding (rick_predict)."""
        n = self.n
        m = u.numel()
        model = self._vec(model.contiguous(), "model", torch.float32 if self.real else torch.complex64, n * n)
        u, v, w = (self._vec(u, "u", torch.float32, m), self._vec(v, "v", torch.float32, m),
                   self._vec(w, "w", torch.float32, m))
        if out is None:
            out = torch.empty(m, dtype=torch.complex64, device=self.device)
        self._vec(out, "out", torch.complex64, m)
        self._sync_stream()
        _lib.check(self._L.rick_predict(self._h, _ptr(model), _ptr(u), _ptr(v), _ptr(w), m, _ptr(out)), self._h)
        return out

    def image_host(self, vis, u, v, w, wt=None, out=None):
        """End to end with host (CPU) tensors, through rick_image_host."""
        m = u.numel()
        for name, t, dt in (("vis", vis, torch.complex64), ("u", u, torch.float32), ("v", v, torch.float32),
                            ("w", w, torch.float32)):
            if t.device.type != "cpu" or t.dtype != dt or not t.is_contiguous() or t.numel() != m:
                raise ValueError(f"{name} must be a contiguous {dt} CPU tensor of {m} elements")
        if wt is not None and (wt.device.type != "cpu" or wt.dtype != torch.float32 or wt.numel() != m):
            raise ValueError("wt must be a float32 CPU tensor")
        n = self.n
        if out is None:
            out = torch.empty((n, n), dtype=torch.float32 if self.real else torch.complex64)
        self._sync_stream()
        _lib.check(self._L.rick_image_host(self._h, _ptr(vis), _ptr(u), _ptr(v), _ptr(w), _ptr(wt), m,
                                           _ptr(out)), self._h)
        self.generation += 1
        return out

    def image_host_async(self, vis, u, v, w, wt=None, out=None):
        """Pipelined image_host (rick_image_host_async): enqueues upload,
        imaging and download and returns at once; the inputs must stay
        unmodified and `out` (pinned CPU memory) unread until synchronize()."""
        m = u.numel()
        for name, t, dt in (("vis", vis, torch.complex64), ("u", u, torch.float32), ("v", v, torch.float32),
                            ("w", w, torch.float32)):
            if t.device.type != "cpu" or t.dtype != dt or not t.is_contiguous() or t.numel() != m:
                raise ValueError(f"{name} must be a contiguous {dt} CPU tensor of {m} elements")
        if wt is not None and (wt.device.type != "cpu" or wt.dtype != torch.float32 or wt.numel() != m):
            raise ValueError("wt must be a float32 CPU tensor")
        n = self.n
        if out is None:
            out = torch.empty((n, n), dtype=torch.float32 if self.real else torch.complex64).pin_memory()
        self._sync_stream()
        _lib.check(self._L.rick_image_host_async(self._h, _ptr(vis), _ptr(u), _ptr(v), _ptr(w), _ptr(wt), m,
                                                 _ptr(out)), self._h)
        self.generation += 1
        return out

    def synchronize(self):
        """Wait for everything enqueued on this imager (rick_synchronize)."""
        _lib.check(self._L.rick_synchronize(self._h), self._h)

    def set_prep_blocks(self, blocks_per_sm):
        """Blocks per SM of the sort kernels (rick_set_prep_blocks; 0 = default)."""
        _lib.check(self._L.rick_set_prep_blocks(self._h, int(blocks_per_sm)), self._h)

    def set_plane_range(self, k0, k1):
        """Grid, transform and stack only w-planes k0 .. k1-1 (rick_set_plane_range);
        call before grid (after reset)."""
        _lib.check(self._L.rick_set_plane_range(self._h, int(k0), int(k1)), self._h)

    def set_weight_sum(self, sum_w):
        """Normalise by sum_w instead of this imager's own weight sum
        (rick_set_weight_sum); sum_w < 0 returns to the own sum."""
        self._sync_stream()
        _lib.check(self._L.rick_set_weight_sum(self._h, float(sum_w)), self._h)

    def debug_colstack(self, skip_slot=-1, wait_ns=0):
        """Test hook of the fused column kernel's bounded waits
        (rick_debug_colstack): skip_slot >= 0 leaves that pipeline slot's copy
        out so every wait on it runs out after wait_ns; -1 restores."""
        _lib.check(self._L.rick_debug_colstack(self._h, int(skip_slot), int(wait_ns)), self._h)

    def stats(self):
        st = _lib.RickStats()
        _lib.check(self._L.rick_get_stats(self._h, ctypes.byref(st)), self._h)
        return {f: getattr(st, f) for f, _ in st._fields_}

    def set_timing(self, enable=True):
        _lib.check(self._L.rick_set_timing(self._h, 1 if enable else 0), self._h)

    def timing(self):
        t = _lib.RickTiming()
        _lib.check(self._L.rick_get_timing(self._h, ctypes.byref(t)), self._h)
        return {f: getattr(t, f) for f, _ in t._fields_}

    def close(self):
        if getattr(self, "_h", None):
            self._L.rick_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class BatchImager(Imager):
    """Many frequency channels imaged together (one sort, one gridder pass and
    one cuFFT batch per plane group, one stack per channel).  ``w_ranges`` is
    a sequence of (w_min, w_max) per channel; the other parameters are shared."""

    def __init__(self, params, w_ranges, device=None):
        self.params = dict(params)
        self._L = _lib.load()
        if device is None:
            device = torch.device("cuda", torch.cuda.current_device())
        self.device = torch.device(device)
        if self.device.type != "cuda":
            raise ValueError("BatchImager needs a CUDA device")
        if self.device.index is None:
            self.device = torch.device("cuda", torch.cuda.current_device())
        self.nchan = len(w_ranges)
        wmin = (ctypes.c_double * self.nchan)(*[float(a) for a, _ in w_ranges])
        wmax = (ctypes.c_double * self.nchan)(*[float(b) for _, b in w_ranges])
        self._rp = _params_struct(self.params)
        h = ctypes.c_void_p()
        with torch.cuda.device(self.device):
            _lib.check(self._L.rick_create_batch(ctypes.byref(self._rp), self.nchan, wmin, wmax, ctypes.byref(h)))
        self._h = h
        self.generation = 0

    def images(self, vis, u, v, w, wt, chan_offsets, out=None, use_graph=False):
        """Dirty images [nchan, n, n] of measurements grouped by channel:
        channel c is entries chan_offsets[c] .. chan_offsets[c+1]-1."""
        vis, u, v, w, wt, m = self._inputs(vis, u, v, w, wt)
        offs = [int(x) for x in chan_offsets]
        if len(offs) != self.nchan + 1 or offs[0] != 0 or offs[-1] != m:
            raise ValueError("chan_offsets must have nchan + 1 entries from 0 to the number of measurements")
        n = self.n
        if out is None:
            shape = (self.nchan, n, n)
            out = torch.empty(shape, dtype=torch.float32 if self.real else torch.complex64, device=self.device)
        self._vec(out, "out", torch.float32 if self.real else torch.complex64, self.nchan * n * n)
        self._offs = (ctypes.c_int64 * (self.nchan + 1))(*offs)
        self._sync_stream()
        _lib.check(self._L.rick_image_batch(self._h, _ptr(vis), _ptr(u), _ptr(v), _ptr(w), _ptr(wt),
                                            ctypes.cast(self._offs, ctypes.c_void_p), _ptr(out),
                                            1 if use_graph else 0), self._h)
        return out


def autotune_batch(params, w_ranges, vis, u, v, w, wt, chan_offsets):
    """Tile side, plane group and sort blocks per SM for batched imaging of
    this data, timed on the GPU (see rick_autotune_batch).  Returns (tile,
    plane_group, prep_blocks, ms); prep_blocks 0 = the default."""
    L = _lib.load()
    nchan = len(w_ranges)
    rp = _params_struct(params)
    wmin = (ctypes.c_double * nchan)(*[float(a) for a, _ in w_ranges])
    wmax = (ctypes.c_double * nchan)(*[float(b) for _, b in w_ranges])
    offs = (ctypes.c_int64 * (nchan + 1))(*[int(x) for x in chan_offsets])
    t, g, pb, ms = ctypes.c_int32(0), ctypes.c_int32(0), ctypes.c_int32(0), ctypes.c_double(0.0)
    _lib.check(L.rick_autotune_batch(ctypes.byref(rp), nchan, wmin, wmax, _ptr(vis), _ptr(u), _ptr(v), _ptr(w),
                                     _ptr(wt), ctypes.cast(offs, ctypes.c_void_p), ctypes.byref(t), ctypes.byref(g),
                                     ctypes.byref(pb), ctypes.byref(ms)))
    return t.value, g.value, pb.value, ms.value


class DirtyImage(torch.autograd.Function):
    """Differentiable dirty image D(V) (linear in V).  Backward: the hand-written
    adjoint degridder, grad_V = A^H grad_D, with w-planes recomputed from grad_D.
    The imager must not be regridded between forward and backward."""

    @staticmethod
    def forward(ctx, vis, u, v, w, wt, imager):
        imager.reset()
        imager.grid(vis.detach().contiguous(), u, v, w, wt)
        img = imager.image()
        ctx.imager = imager
        ctx.generation = imager.generation
        ctx.save_for_backward(u, v, w, wt if wt is not None else torch.empty(0, device=u.device))
        ctx.has_wt = wt is not None
        return img

    @staticmethod
    def backward(ctx, grad):
        u, v, w, wt = ctx.saved_tensors
        imager = ctx.imager
        if imager.generation != ctx.generation:
            raise RuntimeError("the imager was regridded between forward and backward")
        g = imager.degrid(grad.contiguous(), u, v, w, wt if ctx.has_wt else None)
        return g, None, None, None, None, None


def dirty_image(vis, u, v, w, wt, imager):
    """D = imager's dirty image of (vis, u, v, w, wt), differentiable in vis."""
    return DirtyImage.apply(vis, u, v, w, wt, imager)
