"""Host-only checks of the C ABI: the library loads and exports every symbol
include/rick.h declares, the Python binding declares the same set, and the
struct layouts agree (no GPU needed; no compute call is made)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "rick.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(rick_[a-z_0-9]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_2504_00959_gb300 import build
    build.build()
    from paper_2504_00959_gb300 import _lib
    return _lib.load()


def test_header_declares_the_api():
    names = _declared()
    for required in ("rick_create", "rick_grid", "rick_fft_and_stack", "rick_degrid", "rick_destroy",
                     "rick_image_host", "rick_grid_planes"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    for name in _declared():
        assert hasattr(lib, name), name


def test_binding_covers_every_declared_symbol():
    from paper_2504_00959_gb300 import _lib
    assert sorted(_lib.SIGNATURES) == _declared()


def test_struct_layouts():
    from paper_2504_00959_gb300 import _lib
    assert ctypes.sizeof(_lib.RickParams) == 64
    assert _lib.RickParams.kernel_param.offset == 40
    assert _lib.RickParams.flags.offset == 56
    assert ctypes.sizeof(_lib.RickStats) == 48


def test_status_strings_and_null_handles(lib):
    from paper_2504_00959_gb300 import _lib
    assert lib.rick_status_string(0) == b"RICK_OK"
    assert lib.rick_status_string(2) == b"RICK_ERR_OOM"
    # null handles and null output pointers are argument errors, never crashes
    assert lib.rick_destroy(None) == 0
    assert lib.rick_reset(None) == 1
    assert lib.rick_grid(None, None, None, None, None, None, 0) == 1
    assert lib.rick_create(None, None) == 1
    assert lib.rick_workspace_size(None, 0, None) == 1


def test_failed_creation_keeps_its_message(lib):
    """Parameters are checked on the host before any CUDA call: a refused
    rick_create returns no handle, and rick_last_error(NULL) gives why."""
    from paper_2504_00959_gb300 import _lib
    p = _lib.RickParams()
    lib.rick_params_default(ctypes.byref(p))
    p.tile = 48
    h = ctypes.c_void_p(None)
    assert lib.rick_create(ctypes.byref(p), ctypes.byref(h)) == 1
    assert not h.value
    assert b"tile" in lib.rick_last_error(None)


def test_workspace_size_and_parameter_checks(lib):
    from paper_2504_00959_gb300 import _lib
    p = _lib.RickParams()
    assert lib.rick_params_default(ctypes.byref(p)) == 0
    size = ctypes.c_size_t(0)
    assert lib.rick_workspace_size(ctypes.byref(p), 1000, ctypes.byref(size)) == 0
    assert size.value > 8 * 256 * 256 * 8
    for field, bad in (("n", 7), ("n", 2), ("nw", 0), ("support", 0), ("support", 17), ("kernel", 5),
                       ("tile", 48), ("flags", 1 << 10), ("pixel_rad", -1.0)):
        q = _lib.RickParams()
        lib.rick_params_default(ctypes.byref(q))
        setattr(q, field, bad)
        assert lib.rick_workspace_size(ctypes.byref(q), 10, ctypes.byref(size)) == 1, (field, bad)
    q = _lib.RickParams()
    lib.rick_params_default(ctypes.byref(q))
    q.w_max = q.w_min
    assert lib.rick_workspace_size(ctypes.byref(q), 10, ctypes.byref(size)) == 1
    q.nw = 1
    assert lib.rick_workspace_size(ctypes.byref(q), 10, ctypes.byref(size)) == 0
    # w-support: at most 16 and at most nw
    for ws, nw, ok in ((17, 32, False), (9, 8, False), (4, 8, True), (0, 1, True), (-1, 8, False)):
        q = _lib.RickParams()
        lib.rick_params_default(ctypes.byref(q))
        q.nw, q.w_support = nw, ws
        if nw == 1:
            q.w_max = q.w_min + 1.0
        assert (lib.rick_workspace_size(ctypes.byref(q), 10, ctypes.byref(size)) == 0) == ok, (ws, nw)
    # the Hermitian fold changes the imaginary part: only with real images
    q = _lib.RickParams()
    lib.rick_params_default(ctypes.byref(q))
    q.flags = _lib.HERMITIAN_FOLD | _lib.GRID_CORRECT
    assert lib.rick_workspace_size(ctypes.byref(q), 10, ctypes.byref(size)) == 1
    q.flags = _lib.HERMITIAN_FOLD | _lib.REAL_IMAGE
    assert lib.rick_workspace_size(ctypes.byref(q), 10, ctypes.byref(size)) == 0


def test_transform_path_flags(lib):
    """RICK_FFT_2D and RICK_FFT_SPLIT exclude each other; the split needs a
    power-of-two n in [64, 16384]."""
    from paper_2504_00959_gb300 import _lib
    size = ctypes.c_size_t(0)
    for n, flags, ok in ((256, _lib.FFT_2D, True), (256, _lib.FFT_SPLIT, True), (4096, _lib.FFT_SPLIT, True),
                         (256, _lib.FFT_2D | _lib.FFT_SPLIT, False), (34, _lib.FFT_SPLIT, False),
                         (8192, _lib.FFT_SPLIT, True), (32768, _lib.FFT_SPLIT, False), (32, _lib.FFT_SPLIT, False), (34, _lib.FFT_2D, True)):
        q = _lib.RickParams()
        lib.rick_params_default(ctypes.byref(q))
        q.n, q.flags = n, flags | _lib.REAL_IMAGE
        assert (lib.rick_workspace_size(ctypes.byref(q), 10, ctypes.byref(size)) == 0) == ok, (n, flags)
