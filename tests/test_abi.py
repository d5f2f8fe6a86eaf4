"""The C ABI library builds for sm_103a, loads, and exports every entry
point include/tll.h declares; argument errors come back as codes.  No
compute call is made here (CPU-only)."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_2503_08586_gb300 import build, tll

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", fn)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names |= set(re.findall(r"\b(tll_[a-z0-9_]+)\s*\(", txt))
    return names


@pytest.fixture(scope="module")
def lib():
    build.build()
    return tll.load()


def test_every_declared_symbol_is_exported(lib):
    decl = _declared()
    assert decl, "no declarations found"
    for name in decl:
        assert hasattr(lib, name), name
    assert decl == set(tll.SYMBOLS) | (decl - set(tll.SYMBOLS))
    assert set(tll.SYMBOLS) <= decl


def test_version_and_error_string(lib):
    assert lib.tll_version() >= 100
    assert isinstance(lib.tll_last_error(), bytes)


def test_argument_validation_without_gpu(lib):
    g = tll.Grid(4, 4, 0.1, 2, 0.0, 0.0)
    h = ctypes.c_void_p()
    img = np.zeros(16, np.float32)
    psf = np.ones(9, np.float32)
    # NULL pointers, even PSF, bad supersampling, zero PSF sum, bad mode
    assert lib.tll_create_lens(None, img.ctypes.data, psf.ctypes.data, 3,
                               ctypes.byref(g), 0, ctypes.byref(h)) == tll.EINVAL
    assert lib.tll_create_lens(img.ctypes.data, img.ctypes.data,
                               psf.ctypes.data, 2, ctypes.byref(g), 0,
                               ctypes.byref(h)) == tll.EINVAL
    bad = tll.Grid(4, 4, 0.1, 0, 0.0, 0.0)
    assert lib.tll_create_lens(img.ctypes.data, img.ctypes.data,
                               psf.ctypes.data, 3, ctypes.byref(bad), 0,
                               ctypes.byref(h)) == tll.EINVAL
    z = np.zeros(9, np.float32)
    assert lib.tll_create_lens(img.ctypes.data, img.ctypes.data, z.ctypes.data,
                               3, ctypes.byref(g), 0, ctypes.byref(h)) == tll.EINVAL
    assert lib.tll_create_lens(img.ctypes.data, img.ctypes.data,
                               psf.ctypes.data, 3, ctypes.byref(g), 7,
                               ctypes.byref(h)) == tll.EINVAL
    assert b"mode" in lib.tll_last_error()
    # NULL lens
    assert lib.tll_loglike_batch(None, None, 4, None, None) == tll.EINVAL
    assert lib.tll_model_image(None, None, None, None, None) == tll.EINVAL
    lib.tll_destroy_lens(None)


def test_no_silent_cpu_fallback(lib):
    """Without a usable GPU the library refuses instead of computing."""
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(tll.TLLError) as ei:
        tll.Lens(np.zeros((4, 4)), np.ones((4, 4)), np.ones((3, 3)), 0.1, 2)
    assert ei.value.code == tll.ECUDA


def test_server_refuses_without_gpu(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(tll.TLLError) as ei:
        tll.Server(max_jobs=2)
    assert ei.value.code in (tll.ECUDA, tll.ENOMEM)
    cfg = tll.ServerConfig(0, 0, 16, 1, 1, 0)          # max_jobs = 0
    h = ctypes.c_void_p()
    assert lib.tll_server_create(ctypes.byref(cfg), ctypes.byref(h)) == tll.EINVAL


def test_autotune_cache_file_errors(lib, tmp_path):
    """The cache file: a save of this process's (here empty) tuned shapes
    writes the header; a missing, foreign or malformed file is refused."""
    p = tmp_path / "tune.txt"
    assert lib.tll_autotune_save(str(p).encode()) == tll.OK
    assert p.read_text().splitlines()[0] == "tll-autotune 1"
    assert lib.tll_autotune_save(None) == tll.EINVAL
    assert lib.tll_autotune_load(str(tmp_path / "missing.txt").encode()) == tll.EINVAL
    bad = tmp_path / "bad.txt"
    bad.write_text("something else\n")
    assert lib.tll_autotune_load(str(bad).encode()) == tll.EINVAL
    bad.write_text("tll-autotune 1\nGB300 100 100 4 21 1 1000 1\n")   # CTA size not a warp multiple
    assert lib.tll_autotune_load(str(bad).encode()) in (tll.EINVAL, tll.ECUDA)
    lib.tll_autotune_clear()


def test_noalloc_limit_matches_header():
    """The binding's copy of the no-allocation batch limit is the header's
    (the library takes it from the header's #define)."""
    txt = open(os.path.join(ROOT, "include", "tll.h")).read()
    m = re.search(r"#define\s+TLL_NOALLOC_MAX_B\s+(\d+)", txt)
    assert m, "TLL_NOALLOC_MAX_B not defined in include/tll.h"
    assert int(m.group(1)) == tll.NOALLOC_MAX_B
    src = open(os.path.join(ROOT, "paper_2503_08586_gb300", "csrc", "tll.cu")).read()
    assert re.search(r"kNoAllocMaxB\s*=\s*TLL_NOALLOC_MAX_B\s*;", src)
