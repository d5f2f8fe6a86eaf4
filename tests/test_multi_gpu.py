"""Ragged multi-lens launches (tll_batcher) against one-lens launches and
the FP64 oracle: lenses of different sizes, supersampling factors, PSF sides
and image placements in one persistent launch, plain and graph-replayed."""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
from paper_2503_08586_gb300 import build, tll
from paper_2503_08586_gb300 import workloads as W

pytestmark = pytest.mark.gpu

# (ny, nx, dpix, sub, psf kind, psf side, vectors)
LENSES = [
    (64, 64, 0.05, 4, "gauss", 11, 37),
    (100, 100, 0.074, 4, "gauss", 21, 130),
    (48, 70, 0.06, 5, "gauss", 15, 20),
    (33, 41, 0.07, 2, "moffat", 9, 25),      # direct PSF, unpadded shared memory
    (200, 200, 0.05, 1, "moffat", 13, 6),    # global scratch placement
    (64, 64, 0.05, 3, "gauss", 31, 9),
]


@pytest.fixture(scope="module")
def setup():
    build.build()
    tll.load()
    assert torch.cuda.is_available()
    out = []
    for k, (ny, nx, dpix, sub, kind, ks, nv) in enumerate(LENSES):
        psf = W.gaussian_psf(ks, 1.8) if kind == "gauss" else W.moffat_psf(ks, 2.0, 3.0)
        rng = np.random.Generator(np.random.PCG64(500 + k))
        render = oracle.columns_renderer(dpix, sub, psf, ny, nx)
        sl = W.synth_lens(rng, ny, nx, dpix, sub, psf, render, "sky+poisson")
        P = np.concatenate([sl.truth[None], W.shrinking_draws(rng, sl.truth, nv - 1)])
        P[min(3, nv - 1), 8] = -1.0        # one invalid vector per lens
        g = tll.Lens(sl.data, sl.noise, sl.psf, sl.pixel_scale, sl.sub, sl.x0, sl.y0)
        out.append((sl, g, P))
    return out


def _single(g, P):
    o = g.loglike_batch(torch.from_numpy(P).cuda())
    torch.cuda.synchronize()
    return o.cpu().numpy()


@pytest.mark.parametrize("use_graph", [False, True])
def test_multi_equals_single(setup, use_graph):
    b = tll.Batcher(use_graph=use_graph)
    stream = torch.cuda.Stream()
    lenses = [g for _, g, _ in setup]
    params = [torch.from_numpy(P).cuda() for _, _, P in setup]
    torch.cuda.synchronize()
    for rep in range(3):          # replays reuse the captured graph
        with torch.cuda.stream(stream):
            outs = b.run(lenses, params, stream=stream)
        stream.synchronize()
        for (sl, g, P), o in zip(setup, outs):
            got = o.cpu().numpy()
            ref = _single(g, P)
            assert np.array_equal(np.isneginf(got), np.isneginf(ref))
            fin = np.isfinite(ref)
            assert np.allclose(got[fin], ref[fin], rtol=1e-12, atol=1e-9)
    b.close()


def test_multi_against_oracle(setup):
    b = tll.Batcher(use_graph=False)
    lenses = [g for _, g, _ in setup]
    params = [torch.from_numpy(P).cuda() for _, _, P in setup]
    outs = b.run(lenses, params)
    torch.cuda.synchronize()
    for (sl, g, P), o in zip(setup, outs):
        got = o.cpu().numpy()
        idx = np.arange(min(4, len(P)))
        ol = oracle.Lens(sl.data, sl.noise, sl.psf, sl.pixel_scale, sl.sub, sl.x0, sl.y0)
        ref = ol.loglike_batch(P[idx].astype(np.float64))
        fin = np.isfinite(ref)
        assert np.array_equal(np.isneginf(got[idx]), np.isneginf(ref))
        d = np.abs(got[idx][fin] - ref[fin])
        assert np.all(d <= np.maximum(1e-3, 1e-6 * np.abs(ref[fin]))), d
    b.close()


def test_multi_repeated_lens_and_empty_entries(setup):
    """The same lens twice in one launch and zero-length entries."""
    sl, g, P = setup[0]
    b = tll.Batcher(use_graph=False)
    p1 = torch.from_numpy(P[:10]).cuda()
    p2 = torch.from_numpy(P[10:]).cuda()
    p0 = torch.empty((0, 21), dtype=torch.float32, device="cuda")
    outs = b.run([g, g, g], [p1, p0, p2])
    torch.cuda.synchronize()
    got = np.concatenate([outs[0].cpu().numpy(), outs[2].cpu().numpy()])
    ref = _single(g, P)
    fin = np.isfinite(ref)
    assert np.allclose(got[fin], ref[fin], rtol=1e-12, atol=1e-9)
    b.close()


@pytest.mark.parametrize("use_graph", [False, True])
def test_multi_lens_slots_split_and_update(use_graph):
    """Nine two-column lenses of one shape class: a launch group holds at
    most five (their descriptors in the launch parameters), so the sixth
    starts a second group; one lens appears in two non-adjacent entries.
    Runs with other lens sets (in graph form: the captured graph updated in
    place, or instantiated again when the groups change) must again equal
    the one-lens launches."""
    build.build()
    tll.load()
    psf = W.gaussian_psf(11, 1.8)
    render = oracle.columns_renderer(0.05, 4, psf, 40, 44)
    items = []
    for k in range(9):
        rng = np.random.Generator(np.random.PCG64(900 + k))
        sl = W.synth_lens(rng, 40, 44, 0.05, 4, psf, render, "sky")
        P = np.concatenate([sl.truth[None], W.shrinking_draws(rng, sl.truth, 11 + 7 * k)])
        g = tll.Lens(sl.data, sl.noise, sl.psf, sl.pixel_scale, sl.sub, sl.x0, sl.y0)
        items.append((g, P.astype(np.float32)))
    b = tll.Batcher(use_graph=use_graph)
    stream = torch.cuda.Stream()
    # the second run keeps the group launches (graph updated in place), the
    # third has one group fewer (graph instantiated again)
    runs = [list(range(9)) + [2], [8, 7, 6, 5, 4, 3, 1, 0, 2, 6], [8, 5, 1, 7, 3]]
    for sel in runs:
        lenses = [items[k][0] for k in sel]
        parts = []
        for j, k in enumerate(sel):
            P = items[k][1]
            parts.append(P[: len(P) // 2] if sel.count(k) > 1 and j == sel.index(k) else
                         P[len(P) // 2:] if sel.count(k) > 1 else P)
        params = [torch.from_numpy(np.ascontiguousarray(p)).cuda() for p in parts]
        torch.cuda.synchronize()
        with torch.cuda.stream(stream):
            outs = b.run(lenses, params, stream=stream)
        stream.synchronize()
        for k, p, o in zip(sel, parts, outs):
            ref = _single(items[k][0], p)
            got = o.cpu().numpy()
            assert np.array_equal(np.isneginf(got), np.isneginf(ref))
            fin = np.isfinite(ref)
            assert np.allclose(got[fin], ref[fin], rtol=1e-12, atol=1e-9), k
    b.close()
    for g, _ in items:
        g.close()
