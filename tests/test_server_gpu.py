"""The continuous-batching server (tll_server_*): each request's result is
the same alone and when merged with other jobs' requests into shared
launches, and equals the job's own one-lens evaluation; admission by
device-memory budget; error codes."""
import threading

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
from paper_2503_08586_gb300 import build, tll
from paper_2503_08586_gb300 import workloads as W

pytestmark = pytest.mark.gpu

SHAPES = [(64, 64, 0.05, 4, 11), (100, 100, 0.074, 4, 21), (80, 60, 0.06, 5, 15),
          (48, 48, 0.05, 2, 9)]


@pytest.fixture(scope="module")
def lenses():
    build.build()
    tll.load()
    assert torch.cuda.is_available()
    out = []
    for k, (ny, nx, dpix, sub, ks) in enumerate(SHAPES):
        psf = W.gaussian_psf(ks, 1.9)
        rng = np.random.Generator(np.random.PCG64(900 + k))
        render = oracle.columns_renderer(dpix, sub, psf, ny, nx)
        sl = W.synth_lens(rng, ny, nx, dpix, sub, psf, render, "sky+poisson")
        batches = [W.shrinking_draws(rng, sl.truth, int(rng.integers(50, 400)))
                   for _ in range(4)]
        out.append((sl, batches))
    return out


def _open(S, sl):
    return S.open_job(sl.data, sl.noise, sl.psf, sl.pixel_scale, sl.sub, sl.x0, sl.y0)


def _reference(sl, P):
    g = tll.Lens(sl.data, sl.noise, sl.psf, sl.pixel_scale, sl.sub, sl.x0, sl.y0)
    o = g.loglike_batch(torch.from_numpy(P).cuda())
    torch.cuda.synchronize()
    r = o.cpu().numpy()
    g.close()
    return r


@pytest.mark.parametrize("coalesce,graph", [(True, True), (True, False), (False, False)])
def test_same_alone_and_in_the_mix(lenses, coalesce, graph):
    # alone: one job at a time, one request at a time
    alone = []
    for sl, batches in lenses:
        S = tll.Server(max_jobs=4, coalesce=coalesce, use_graph=graph)
        j = _open(S, sl)
        res = []
        for P in batches:
            out, _ = S.wait(S.submit(j, P))
            res.append(out.copy())
        assert S.close_job(j)
        S.close()
        alone.append(res)
    # mix: all jobs open, every job submitting from its own thread
    S = tll.Server(max_jobs=8, coalesce=coalesce, use_graph=graph, max_inflight=2)
    jobs = [_open(S, sl) for sl, _ in lenses]
    mixed = [None] * len(lenses)
    errors = []

    def run(k):
        try:
            rids = [S.submit(jobs[k], P) for P in lenses[k][1]]
            mixed[k] = [S.wait(r)[0].copy() for r in rids]
        except Exception as e:  # pragma: no cover
            errors.append(e)

    th = [threading.Thread(target=run, args=(k,)) for k in range(len(lenses))]
    for t in th:
        t.start()
    for t in th:
        t.join()
    assert not errors, errors
    st = S.stats()
    assert st["requests"] == sum(len(b) for _, b in lenses)
    if coalesce:
        assert st["launches"] <= st["requests"]
    for k, (sl, batches) in enumerate(lenses):
        for b, P in enumerate(batches):
            a, m = alone[k][b], mixed[k][b]
            fin = np.isfinite(a)
            assert np.array_equal(np.isneginf(a), np.isneginf(m))
            assert np.allclose(m[fin], a[fin], rtol=1e-12, atol=1e-9)
        ref = _reference(sl, batches[0])
        assert np.allclose(alone[k][0], ref, rtol=1e-12, atol=1e-9)
    for j in jobs:
        assert S.close_job(j)
    S.close()


def test_admission_by_footprint(lenses):
    sl0, _ = lenses[0]
    g = tll.Lens(sl0.data, sl0.noise, sl0.psf, sl0.pixel_scale, sl0.sub, sl0.x0, sl0.y0)
    import ctypes
    b = ctypes.c_size_t()
    assert tll.load().tll_lens_footprint(g.handle, ctypes.byref(b)) == tll.OK
    g.close()
    one = b.value
    assert one > 16 * 64 * 64
    S = tll.Server(hbm_budget_bytes=int(one * 1.5), max_jobs=4)
    j1 = _open(S, sl0)
    assert j1 is not None
    assert _open(S, sl0) is None                     # over budget: EBUSY
    assert S.stats()["admissions_refused"] == 1
    assert S.close_job(j1)
    j2 = _open(S, sl0)                               # memory freed: admitted
    assert j2 is not None
    assert S.stats()["hbm_used_bytes"] == one
    S.close()


def test_errors_and_timeouts(lenses):
    sl, batches = lenses[1]
    S = tll.Server(max_jobs=2, max_vectors_per_launch=1024)
    j = _open(S, sl)
    with pytest.raises(tll.TLLError) as e:
        S.submit(j + 1, batches[0])                  # no such job
    assert e.value.code == tll.EINVAL
    with pytest.raises(tll.TLLError) as e:
        S.submit(j, np.zeros((2000, 21), np.float32))  # over the launch cap
    assert e.value.code == tll.EINVAL
    big = W.shrinking_draws(np.random.default_rng(1), sl.truth, 1024)
    rid = S.submit(j, big)
    closed_early = S.close_job(j)                    # outstanding -> False
    try:
        out, lat = S.wait(rid, timeout_ms=0)
    except tll.TLLError as ex:
        assert ex.code == tll.ETIMEOUT
        out, lat = S.wait(rid)
    assert np.all(np.isfinite(out)) and lat > 0
    if not closed_early:
        assert S.close_job(j)
    S.close()


def test_autotune_at_admission(lenses):
    # the first job of a signature is tuned at admission; results match the
    # job's own one-lens evaluation up to FP64 summation order
    S = tll.Server(max_jobs=4, autotune=True)
    for sl, batches in lenses[:2]:
        j = _open(S, sl)
        assert j is not None
        out, _ = S.wait(S.submit(j, batches[0]))
        ref = _reference(sl, batches[0])
        fin = np.isfinite(ref)
        assert np.array_equal(fin, np.isfinite(out))
        assert np.allclose(out[fin], ref[fin], rtol=1e-10, atol=1e-8)
        assert S.close_job(j)
    S.close()


# Jobs at the wide end of the request-stream recipe (0.074 arcsec pixels,
# sides up to 200: 11-15 arcsec fields, where a coherent FP32 stretch of the
# image-plane grid would move log L by more than 1e-3): side, PSF side.
WIDE = [(200, 31), (176, 25), (148, 17), (154, 27)]


def test_served_wide_fields_against_oracle():
    """Jobs of 148-200 px at 0.074 arcsec through the server (host buffers,
    requests coalesced into shared launches) against the FP64 oracle: every
    vector within the parity gates, and |dlogL| <= 1e-3 on each job's
    posterior bulk (chi^2 within 50 of the truth's)."""
    from test_parity_gpu import BULK_DCHI2, LL_ABS, _chi2_truth, _lens_consts, _ll_ok
    build.build()
    tll.load()
    rng = np.random.Generator(np.random.PCG64(W.SEED_BASE + 77))
    items = []
    for side, k in WIDE:
        psf = W.gaussian_psf(k, k / 7.0)
        render = oracle.columns_renderer(W.f32(0.074), 4, psf, side, side)
        sl = W.synth_lens(rng, side, side, 0.074, 4, psf, render, "sky+poisson")
        # vectors converging on the truth (the second half sits in the bulk)
        P = W.shrinking_draws(rng, sl.truth, 48, lo_frac=1e-6)[16:]
        items.append((sl, np.ascontiguousarray(P, np.float32)))
    S = tll.Server(max_jobs=8)
    ids = [_open(S, sl) for sl, _ in items]
    assert all(j is not None for j in ids)
    reqs = [S.submit(j, P) for j, (_, P) in zip(ids, items)]
    outs = [S.wait(r)[0].copy() for r in reqs]
    for j in ids:
        assert S.close_job(j)
    S.close()
    worst = 0.0
    for (sl, P), got in zip(items, outs):
        o = oracle.Lens(sl.data, sl.noise, sl.psf, sl.pixel_scale, sl.sub, sl.x0, sl.y0)
        ref = o.loglike_batch(P.astype(np.float64))
        _ll_ok(got, ref, sl)
        _, lognorm, _ = _lens_consts(sl)
        bulk = np.isfinite(ref) & (-2.0 * (ref - lognorm) <= _chi2_truth(sl) + BULK_DCHI2)
        assert bulk.sum() >= 8, f"{sl.ny} px: only {bulk.sum()} vectors in the bulk"
        worst = max(worst, float(np.abs(got - ref)[bulk].max()))
    assert worst <= LL_ABS, f"bulk |dlogL| {worst:.3e}"
