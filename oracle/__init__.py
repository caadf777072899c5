"""FP64 CPU oracle of the w-stacking imager (arXiv 2504.00959, Sec. 2.1, Eqs. 1-3).

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, ``__graft_entry__.smoke()``
and the CPU-baseline / reference legs of ``bench.py``; never by the product
package.  It shares no code with the CUDA library.  This module only marshals
numpy arrays into ``liboracle.so`` (built from ``rick_oracle.c``); all of the
arithmetic is in that C file.

Problem parameters are passed as a mapping with the keys ``n``, ``nw``,
``pixel_rad``, ``w_min``, ``w_max``, ``kernel`` (0 Gaussian, 1 Kaiser-Bessel),
``support``, ``kernel_param`` (sigma in cells or beta; 0 = default) and
``flags`` (bit 1 grid correction, 4 multiply by n, 8 uniform weighting, 32
Hermitian fold of the measurements with w < 0), and optionally ``w_support``
(planes per measurement, Eq. 3's kernel in w; 0 or 1 = the nearest plane).

Pins (tests/test_oracle_pins.py): FFT against numpy, I0 against scipy, taper
against the closed-form Fourier transforms of the truncated Gaussian and of
the Kaiser-Bessel window, the delta-kernel special case against
numpy.fft.ifft2, point source / sum / Hermitian / linearity invariants, the
single-measurement closed form, the direct DFT with the exact w-term within
the derived w-quantisation + aliasing bound, the adjoint's dot-product
identity and dense-matrix check, and the Hermitian fold against the unfolded
imager on mirrored w-planes.
"""
import ctypes
import os

import numpy as np

from . import build as _build

KERNEL_GAUSS = 0
KERNEL_KB = 1
FLAG_CORRECT = 1
FLAG_REAL = 2
FLAG_APPLY_N = 4
FLAG_UNIFORM = 8
FLAG_FOLD = 32

_lib = None

_f32p = np.ctypeslib.ndpointer(dtype=np.float32, flags="C_CONTIGUOUS")
_f64p = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")
_i32p = np.ctypeslib.ndpointer(dtype=np.int32, flags="C_CONTIGUOUS")
_CFG = [ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_double,
        ctypes.c_int, ctypes.c_int, ctypes.c_double]
_VIS = [ctypes.c_int64, _f32p, _f32p, _f32p, _f32p, _f32p]


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        L.oracle_bessel_i0.restype = ctypes.c_double
        L.oracle_bessel_i0.argtypes = [ctypes.c_double]
        L.oracle_kernel.restype = ctypes.c_double
        L.oracle_kernel.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double]
        L.oracle_fft.restype = None
        L.oracle_fft.argtypes = [ctypes.c_int, _f64p, ctypes.c_int]
        L.oracle_plane_image.restype = None
        L.oracle_plane_image.argtypes = [ctypes.c_int, _f64p, ctypes.c_int]
        L.oracle_taper.restype = ctypes.c_int
        L.oracle_taper.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_double, _f64p]
        L.oracle_place_batch.restype = ctypes.c_int
        L.oracle_place_batch.argtypes = _CFG + [ctypes.c_int64, _f32p, _f32p, _f32p, _i32p, _i32p, _i32p]
        L.oracle_grid.restype = ctypes.c_int64
        L.oracle_grid.argtypes = _CFG + [ctypes.c_uint] + _VIS + [ctypes.c_int, ctypes.c_int, _f64p,
                                                                ctypes.POINTER(ctypes.c_double)]
        L.oracle_dirty_image.restype = ctypes.c_int64
        L.oracle_dirty_image.argtypes = L.oracle_grid.argtypes
        L.oracle_image_at.restype = ctypes.c_int64
        L.oracle_image_at.argtypes = _CFG + [ctypes.c_uint] + _VIS + [ctypes.c_int, _i32p, _f64p,
                                                                    ctypes.POINTER(ctypes.c_double)]
        L.oracle_dft.restype = ctypes.c_int64
        L.oracle_dft.argtypes = _CFG + [ctypes.c_uint] + _VIS + [ctypes.c_int, _i32p, _f64p]
        L.oracle_degrid.restype = ctypes.c_int64
        L.oracle_degrid.argtypes = _CFG + [ctypes.c_uint] + _VIS + [_f64p, _f64p]
        L.oracle_predict.restype = ctypes.c_int64
        L.oracle_predict.argtypes = _CFG + [ctypes.c_uint, ctypes.c_int64, _f32p, _f32p, _f32p, _f64p, _f64p]
        L.oracle_num_threads.restype = ctypes.c_int
        L.oracle_num_threads.argtypes = []
        _lib = L
    return _lib


def _cfg(p):
    return (int(p["n"]), int(p["nw"]), float(p["pixel_rad"]), float(p["w_min"]),
            float(p["w_max"]), int(p["kernel"]), int(p["support"]),
            float(p.get("kernel_param", 0.0) or 0.0))


def _flags(p, flags):
    """The flags word, with the w-support of p (``w_support``, 0/1 = nearest
    plane) in bits 8..15."""
    f = int(p.get("flags", FLAG_CORRECT) if flags is None else flags) & 0xff
    return f | (int(p.get("w_support", 0) or 0) & 0xff) << 8


def _vis_args(u, v, w, wt, vis):
    u = np.ascontiguousarray(u, dtype=np.float32)
    v = np.ascontiguousarray(v, dtype=np.float32)
    w = np.ascontiguousarray(w, dtype=np.float32)
    m = u.shape[0]
    wt = np.ones(m, np.float32) if wt is None else np.ascontiguousarray(wt, dtype=np.float32)
    vis = np.ascontiguousarray(vis, dtype=np.complex64).view(np.float32)
    if not (v.shape[0] == w.shape[0] == wt.shape[0] == m and vis.shape[0] == 2 * m):
        raise ValueError("u, v, w, wt, vis must have the same length")
    return (m, u, v, w, wt, vis)


def _check(ret, what):
    if ret < 0:
        raise ValueError(f"oracle {what}: invalid arguments")
    return int(ret)


def bessel_i0(x):
    return lib().oracle_bessel_i0(float(x))


def kernel_value(kernel, support, kernel_param, x):
    return lib().oracle_kernel(int(kernel), int(support), float(kernel_param), float(x))


def fft(x, sign):
    """Unnormalised 1D DFT with exponent sign * 2 pi i (the oracle's own FFT)."""
    a = np.ascontiguousarray(x, dtype=np.complex128).copy()
    lib().oracle_fft(a.shape[0], a.view(np.float64), int(sign))
    return a


def plane_image(grid, sign=+1):
    """Shifted unnormalised 2D DFT of one plane (sign +1: the imaging transform)."""
    a = np.ascontiguousarray(grid, dtype=np.complex128).copy()
    lib().oracle_plane_image(a.shape[0], a.view(np.float64).reshape(-1), int(sign))
    return a


def taper(n, kernel, support, kernel_param=0.0):
    out = np.zeros(n, np.float64)
    _check(lib().oracle_taper(int(n), int(kernel), int(support), float(kernel_param), out), "taper")
    return out


def place(p, u, v, w):
    """Binary32 placement decisions: plane, first u cell, first v cell (-1 = dropped)."""
    u = np.ascontiguousarray(u, dtype=np.float32)
    v = np.ascontiguousarray(v, dtype=np.float32)
    w = np.ascontiguousarray(w, dtype=np.float32)
    m = u.shape[0]
    k = np.empty(m, np.int32)
    fu = np.empty(m, np.int32)
    fv = np.empty(m, np.int32)
    _check(lib().oracle_place_batch(*_cfg(p), m, u, v, w, k, fu, fv), "place")
    return k, fu, fv


def grid(p, u, v, w, wt, vis, k0=0, k1=None, flags=None):
    """Gridded planes [k1-k0, n, n] complex128 (no fftshift sign), sum of weights, drops."""
    n = int(p["n"])
    k1 = int(p["nw"]) if k1 is None else int(k1)
    out = np.zeros((max(k1 - k0, 0), n, n), np.complex128)
    sw = ctypes.c_double(0.0)
    d = _check(lib().oracle_grid(*_cfg(p), _flags(p, flags), *_vis_args(u, v, w, wt, vis), int(k0), k1,
                                 out.view(np.float64).reshape(-1), ctypes.byref(sw)), "grid")
    return out, sw.value, d


def dirty_image(p, u, v, w, wt, vis, k0=0, k1=None, flags=None):
    """Complex dirty image [n, n] complex128 (planes k0..k1-1), sum of weights, drops."""
    n = int(p["n"])
    k1 = int(p["nw"]) if k1 is None else int(k1)
    out = np.zeros((n, n), np.complex128)
    sw = ctypes.c_double(0.0)
    d = _check(lib().oracle_dirty_image(*_cfg(p), _flags(p, flags), *_vis_args(u, v, w, wt, vis), int(k0), k1,
                                        out.view(np.float64).reshape(-1), ctypes.byref(sw)), "dirty_image")
    return out, sw.value, d


def _pix(pix):
    pix = np.ascontiguousarray(np.asarray(pix, dtype=np.int32).reshape(-1, 2))
    return pix.shape[0], pix


def image_at(p, u, v, w, wt, vis, pix, flags=None):
    """The same dirty image evaluated at pixels pix[:, (x, y)] without FFTs."""
    npix, pa = _pix(pix)
    out = np.zeros(npix, np.complex128)
    sw = ctypes.c_double(0.0)
    _check(lib().oracle_image_at(*_cfg(p), _flags(p, flags), *_vis_args(u, v, w, wt, vis), npix, pa,
                                 out.view(np.float64), ctypes.byref(sw)), "image_at")
    return out


def dft(p, u, v, w, wt, vis, pix, flags=None):
    """Brute-force direct DFT with the exact w-term at pixels pix[:, (x, y)]."""
    npix, pa = _pix(pix)
    out = np.zeros(npix, np.complex128)
    _check(lib().oracle_dft(*_cfg(p), _flags(p, flags), *_vis_args(u, v, w, wt, vis), npix, pa,
                            out.view(np.float64)), "dft")
    return out


def degrid(p, u, v, w, wt, vis, r, flags=None):
    """Adjoint of V -> complex dirty image, applied to the complex image r [n, n]."""
    args = _vis_args(u, v, w, wt, vis)
    r = np.ascontiguousarray(r, dtype=np.complex128)
    out = np.zeros(args[0], np.complex128)
    _check(lib().oracle_degrid(*_cfg(p), _flags(p, flags), *args, r.view(np.float64).reshape(-1),
                               out.view(np.float64)), "degrid")
    return out


def predict(p, u, v, w, model, flags=None):
    """Model visibilities of the complex image model [n, n] at (u, v, w): the
    w-stacking evaluation of the measurement equation (unit weights, no
    normalisation)."""
    u = np.ascontiguousarray(u, dtype=np.float32)
    v = np.ascontiguousarray(v, dtype=np.float32)
    w = np.ascontiguousarray(w, dtype=np.float32)
    m = u.shape[0]
    model = np.ascontiguousarray(model, dtype=np.complex128)
    out = np.zeros(m, np.complex128)
    _check(lib().oracle_predict(*_cfg(p), _flags(p, flags), m, u, v, w, model.view(np.float64).reshape(-1),
                                out.view(np.float64)), "predict")
    return out


def num_threads():
    return int(lib().oracle_num_threads())
