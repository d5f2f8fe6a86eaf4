"""The no-allocation entry point, tll_loglike_batch_noalloc, through the C
ABI: two calls in a row, each compared with tll_loglike_batch on the same
inputs.  It exists for callers that cannot allocate device memory during a
call (device memory fully reserved by another allocator, or a loop that
cannot take cudaMalloc/cudaFree stalls); it uses a fixed scratch array
compiled into the library instead of a lens-owned buffer.  This file is
collected last so that a failure here does not stop the other tests."""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
from paper_2503_08586_gb300 import build, tll
from paper_2503_08586_gb300 import workloads as W

pytestmark = pytest.mark.gpu

LL_ABS = 1e-3   # the log-likelihood tolerance of the parity tests


def _batch(lib, fn, lens, p):
    out = torch.full((p.shape[0],), np.nan, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    rc = fn(lens.handle, ctypes.c_void_p(p.data_ptr()), p.shape[0],
            ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(stream))
    assert rc == tll.OK, lib.tll_last_error()
    torch.cuda.synchronize()
    return out.cpu().numpy()


def test_noalloc_matches_allocating_entry_point_twice():
    build.build()
    lib = tll.load()
    assert torch.cuda.is_available()
    sl, params = W.workload("plain64", oracle.columns_renderer, batch=300)
    lens = tll.Lens(sl.data, sl.noise, sl.psf, sl.pixel_scale, sl.sub, sl.x0, sl.y0)
    rng = np.random.Generator(np.random.PCG64(11))
    batches = [params, W.draw_prior(rng, 173)]      # two calls, different sizes
    for P in batches:
        p = torch.from_numpy(np.ascontiguousarray(P, np.float32)).cuda()
        ref = _batch(lib, lib.tll_loglike_batch, lens, p)
        got = _batch(lib, lib.tll_loglike_batch_noalloc, lens, p)
        assert np.all(np.isfinite(got))
        assert np.max(np.abs(got - ref)) <= LL_ABS
    # a batch over the stated maximum is refused with a clear error
    big = torch.zeros((tll.NOALLOC_MAX_B + 1, tll.NPARAM), dtype=torch.float32,
                      device="cuda")
    out = torch.zeros(tll.NOALLOC_MAX_B + 1, dtype=torch.float64, device="cuda")
    rc = lib.tll_loglike_batch_noalloc(lens.handle, ctypes.c_void_p(big.data_ptr()),
                                       big.shape[0], ctypes.c_void_p(out.data_ptr()),
                                       None)
    assert rc == tll.EINVAL and b"no-allocation limit" in lib.tll_last_error()
    lens.close()
