"""The no-allocation entry point, tll_loglike_batch_noalloc, through the C
ABI.  It is for callers that cannot allocate device memory during a call:
a process whose device memory is fully reserved by another allocator (a
framework's caching allocator, a fixed per-job budget), or a sampler loop
that cannot take cudaMalloc/cudaFree stalls.  Its per-vector scratch is a
fixed array compiled into the library instead of the lens-owned buffer that
tll_loglike_batch grows.  Two calls in a row of different sizes, then one
at the stated maximum (above the lens's initial scratch, where the
allocating entry point would have to grow its buffer), each compared bit
for bit with tll_loglike_batch on the same inputs (the same kernels on the
same data), and the lens's device footprint unchanged by the no-allocation
calls.  This file is collected last so that a failure here does not stop
the other tests."""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
from paper_2503_08586_gb300 import build, tll
from paper_2503_08586_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _batch(lib, fn, lens, p):
    out = torch.full((p.shape[0],), np.nan, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    rc = fn(lens.handle, ctypes.c_void_p(p.data_ptr()), p.shape[0],
            ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(stream))
    assert rc == tll.OK, lib.tll_last_error()
    torch.cuda.synchronize()
    return out.cpu().numpy()


def _footprint(lib, lens):
    b = ctypes.c_size_t()
    assert lib.tll_lens_footprint(lens.handle, ctypes.byref(b)) == tll.OK
    return b.value


def test_noalloc_matches_allocating_entry_point_twice():
    build.build()
    lib = tll.load()
    assert torch.cuda.is_available()
    sl, params = W.workload("plain64", oracle.columns_renderer, batch=300)
    lens = tll.Lens(sl.data, sl.noise, sl.psf, sl.pixel_scale, sl.sub, sl.x0, sl.y0)
    rng = np.random.Generator(np.random.PCG64(11))
    full = W.draw_prior(rng, tll.NOALLOC_MAX_B)
    full[:300] = params
    # two calls of different sizes, then one at the maximum; the lens's
    # footprint is read before any allocating call can grow its scratch
    batches = [params, W.draw_prior(rng, 173), full]
    before = _footprint(lib, lens)
    got = []
    for P in batches:
        p = torch.from_numpy(np.ascontiguousarray(P, np.float32)).cuda()
        got.append(_batch(lib, lib.tll_loglike_batch_noalloc, lens, p))
        assert _footprint(lib, lens) == before
    for P, g in zip(batches, got):
        p = torch.from_numpy(np.ascontiguousarray(P, np.float32)).cuda()
        ref = _batch(lib, lib.tll_loglike_batch, lens, p)
        assert np.all(np.isfinite(g[np.isfinite(ref)]))
        assert np.array_equal(g, ref)
    # a batch over the stated maximum is refused with a clear error
    big = torch.zeros((tll.NOALLOC_MAX_B + 1, tll.NPARAM), dtype=torch.float32,
                      device="cuda")
    out = torch.zeros(tll.NOALLOC_MAX_B + 1, dtype=torch.float64, device="cuda")
    rc = lib.tll_loglike_batch_noalloc(lens.handle, ctypes.c_void_p(big.data_ptr()),
                                       big.shape[0], ctypes.c_void_p(out.data_ptr()),
                                       None)
    assert rc == tll.EINVAL and b"no-allocation limit" in lib.tll_last_error()
    lens.close()
