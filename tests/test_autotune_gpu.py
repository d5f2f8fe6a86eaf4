"""Launch shapes and the autotuner: every candidate shape (1 x 1024, 2 x 512,
4 x 256 threads per SM, with the placement its shared-memory share allows)
gives the same log-likelihoods as the FP64 oracle within the parity gates
and as each other to FP64 summation order; the tuner picks the fastest of
what it timed; the batcher groups lenses of different shapes correctly."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
from paper_2503_08586_gb300 import build, tll
from paper_2503_08586_gb300 import workloads as W

from test_parity_gpu import _ll_ok

pytestmark = pytest.mark.gpu

SHAPES = [(1024, 1), (512, 2), (256, 4)]
# (ny, nx, pixel scale, s, PSF side, PSF kind): padded at every shape; padded
# at 1 x 1024 only; banded at every shape; generic (PSF side above 31)
LENSES = [(48, 40, 0.05, 4, 11, "gaussian"), (100, 100, 0.074, 4, 21, "gaussian"),
          (200, 180, 0.05, 5, 15, "moffat"), (40, 36, 0.06, 2, 33, "gaussian")]


def _make(k, ny, nx, dpix, sub, ks, kind):
    psf = W.moffat_psf(ks, 2.0, 3.0) if kind == "moffat" else W.gaussian_psf(ks, ks / 7.0)
    rng = np.random.Generator(np.random.PCG64(4100 + k))
    render = oracle.columns_renderer(dpix, sub, psf, ny, nx)
    sl = W.synth_lens(rng, ny, nx, dpix, sub, psf, render, "sky+poisson")
    P = W.shrinking_draws(rng, sl.truth, 120)
    return sl, P


@pytest.fixture(scope="module")
def cases():
    build.build()
    tll.load()
    assert torch.cuda.is_available()
    out = []
    for k, spec in enumerate(LENSES):
        sl, P = _make(k, *spec)
        ora = oracle.Lens(sl.data, sl.noise, sl.psf, sl.pixel_scale, sl.sub, sl.x0, sl.y0)
        out.append((sl, P, ora.loglike_batch(P)))
    return out


def _lens(sl, **kw):
    return tll.Lens(sl.data, sl.noise, sl.psf, sl.pixel_scale, sl.sub, sl.x0, sl.y0, **kw)


@pytest.mark.parametrize("idx", range(len(LENSES)))
def test_every_shape_matches_oracle(cases, idx):
    sl, P, ref = cases[idx]
    g = _lens(sl)
    Pd = torch.from_numpy(P).cuda()
    first = None
    seen = set()
    for threads, per_sm in SHAPES:
        sh = g.set_shape(threads, per_sm)
        assert sh["threads"] == threads and sh["ctas_per_sm"] >= 1
        seen.add(sh["placement"])
        out = g.loglike_batch(Pd)
        torch.cuda.synchronize()
        o = out.cpu().numpy()
        _ll_ok(o, ref, sl)
        if first is None:
            first = o
        else:
            fin = np.isfinite(first)
            assert np.array_equal(fin, np.isfinite(o))
            assert np.allclose(o[fin], first[fin], rtol=1e-10, atol=1e-8)
    if idx == 2:
        assert "banded" in seen
    if idx == 3:
        assert seen <= {"smem", "global"}
    g.close()


def test_autotune_picks_fastest_and_caches(cases):
    sl, P, ref = cases[1]
    g = _lens(sl)
    Pd = torch.from_numpy(P).cuda()
    r = g.autotune(Pd)
    tried = r["tried"]
    assert len(tried) >= 2 and all(t["ms"] > 0 for t in tried)
    best = min(tried, key=lambda t: t["ms"])
    assert r["chosen"]["threads"] == best["threads"]
    assert g.shape()["threads"] == best["threads"]
    out = g.loglike_batch(Pd)
    torch.cuda.synchronize()
    _ll_ok(out.cpu().numpy(), ref, sl)
    # a new lens with the same signature starts with the tuned shape
    g2 = _lens(sl)
    assert g2.shape()["threads"] == best["threads"]
    # the built-in tuning set works too
    r2 = g2.autotune()
    assert r2["chosen"]["ms"] > 0
    g.close()
    g2.close()


def test_batcher_groups_by_shape(cases):
    lenses, params, refs = [], [], []
    for k, (sl, P, ref) in enumerate(cases[:3]):
        for threads, per_sm in SHAPES[: 2 if k == 1 else 3]:
            g = _lens(sl, batch_only=True)
            g.set_shape(threads, per_sm)
            lenses.append(g)
            params.append(torch.from_numpy(P).cuda())
            refs.append((ref, sl))
    outs = [torch.empty(p.shape[0], dtype=torch.float64, device="cuda") for p in params]
    for graph in (False, True):
        b = tll.Batcher(use_graph=graph)
        stream = torch.cuda.Stream()
        with torch.cuda.stream(stream):
            for _ in range(2):
                for o in outs:
                    o.fill_(0.0)
                b.run(lenses, params, outs, stream=stream)
            stream.synchronize()
        for o, (ref, sl) in zip(outs, refs):
            _ll_ok(o.cpu().numpy(), ref, sl)
        b.close()
    for g in lenses:
        g.close()


def test_autotune_cache_file_roundtrip(cases, tmp_path):
    """A tuned shape saved to the cache file, forgotten, and loaded again:
    a lens created after the load starts with it (marked tuned)."""
    sl, P, ref = cases[0]
    g = tll.Lens(sl.data, sl.noise, sl.psf, sl.pixel_scale, sl.sub, sl.x0, sl.y0)
    chosen = g.autotune(torch.from_numpy(P).cuda())["chosen"]
    g.close()
    path = str(tmp_path / "tune.txt")
    tll.autotune_save(path)
    lines = open(path).read().splitlines()
    assert lines[0] == "tll-autotune 1" and len(lines) >= 2
    tll.autotune_clear()
    g = tll.Lens(sl.data, sl.noise, sl.psf, sl.pixel_scale, sl.sub, sl.x0, sl.y0)
    assert not g.shape()["tuned"]
    g.close()
    tll.autotune_load(path)
    g = tll.Lens(sl.data, sl.noise, sl.psf, sl.pixel_scale, sl.sub, sl.x0, sl.y0)
    sh = g.shape()
    assert sh["tuned"] and sh["threads"] == chosen["threads"]
    assert sh["ctas_per_sm"] == chosen["ctas_per_sm"]
    g.close()
