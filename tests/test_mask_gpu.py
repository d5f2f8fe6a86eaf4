"""Masked pixels (an infinite sigma or a non-finite datum, the paper's fitting
regions of Appendix A) through the C ABI: the batched kernels trace only
the pixels within the PSF's reach of an unmasked pixel, and log L must still
equal the FP64 oracle's (which traces every pixel and gives masked pixels
zero weight) in every placement, in the batcher, the multi-column kernel
and the split pipeline."""
import numpy as np
import pytest
from scipy import ndimage

torch = pytest.importorskip("torch")

import oracle
from paper_2503_08586_gb300 import build, tll
from paper_2503_08586_gb300 import workloads as W

from test_parity_gpu import _CHI2_TRUTH, _lens_consts, _ll_ok

pytestmark = pytest.mark.gpu


def _masked(k, ny, nx, dpix, sub, ks, kind, r_in, r_out, holes=0):
    psf = W.moffat_psf(ks, 2.0, 3.0) if kind == "moffat" else W.gaussian_psf(ks, ks / 7.0)
    rng = np.random.Generator(np.random.PCG64(7600 + k))
    sl = W.synth_lens(rng, ny, nx, dpix, sub, psf,
                      oracle.columns_renderer(W.f32(dpix), sub, psf, ny, nx), "sky+poisson")
    keep = W.annulus_mask(ny, nx, W.f32(dpix), r_in, r_out, sl.x0, sl.y0)
    W.apply_mask(sl, keep)
    if holes:   # scattered bad data values inside the annulus
        idx = rng.choice(ny * nx, holes, replace=False)
        d = sl.data.copy().ravel()
        d[idx] = np.nan
        sl.data = d.reshape(ny, nx)
    P = np.concatenate([W.shrinking_draws(rng, sl.truth, 40, lo_frac=1e-6),
                        W.draw_prior(rng, 24)]).astype(np.float32)
    o = oracle.Lens(sl.data, sl.noise, sl.psf, sl.pixel_scale, sl.sub, sl.x0, sl.y0)
    return sl, P, o, o.loglike_batch(P.astype(np.float64))


@pytest.fixture(scope="module")
def cases():
    build.build()
    tll.load()
    assert torch.cuda.is_available()
    return [_masked(0, 100, 100, 0.074, 4, 21, "gaussian", 0.3, 2.2, holes=25),
            _masked(1, 72, 60, 0.06, 5, 13, "moffat", 0.5, 1.6),
            _masked(2, 72, 64, 0.08, 3, 35, "moffat", 0.2, 0.8)]   # generic convolution


def _gpu(sl, **kw):
    return tll.Lens(sl.data, sl.noise, sl.psf, sl.pixel_scale, sl.sub, sl.x0, sl.y0, **kw)


def _run(g, P):
    out = g.loglike_batch(torch.from_numpy(P).cuda())
    torch.cuda.synchronize()
    return out.cpu().numpy()


def test_traced_set_is_the_dilated_mask(cases):
    """The traced pixels are the unmasked ones dilated by the PSF box."""
    for sl, P, o, ref in cases:
        used = np.isfinite(sl.noise) & (sl.noise > 0) & np.isfinite(sl.data)
        k = sl.psf.shape[0]
        want = ndimage.binary_dilation(used, structure=np.ones((k, k), bool)).sum()
        g = _gpu(sl)
        assert 0 < g.ntrace() == want < sl.ny * sl.nx
        g.close()


@pytest.mark.parametrize("idx", range(3))
def test_masked_loglike_every_placement(cases, idx):
    sl, P, o, ref = cases[idx]
    g = _gpu(sl)
    _ll_ok(_run(g, P), ref, sl)
    for threads, per_sm in ((512, 2), (256, 4)):
        g.set_shape(threads, per_sm)
        _ll_ok(_run(g, P), ref, sl)
    g.close()
    g = _gpu(sl, direct_conv=True)
    _ll_ok(_run(g, P), ref, sl)
    # the model image traces every pixel: it equals the oracle's model there too
    for j in (0, 39):
        img, amps, ll = g.model_image(P[j])
        oll, _, _, omod, _ = o.model(P[j].astype(np.float64))
        _ll_ok(np.array([ll]), np.array([oll]), sl)
        assert np.max(np.abs(img - omod)) <= 1e-4 * np.abs(omod).max()
    g.close()


def test_masked_in_batcher_and_split(cases):
    (s0, P0, _, r0), (s1, P1, _, r1) = cases[0], cases[1]
    rng = np.random.Generator(np.random.PCG64(7700))
    psf = W.gaussian_psf(9, 1.8)
    su = W.synth_lens(rng, 48, 40, 0.05, 4, psf, oracle.columns_renderer(0.05, 4, psf, 48, 40))
    Pu = W.shrinking_draws(rng, su.truth, 40, lo_frac=1e-6)
    ru = oracle.Lens(su.data, su.noise, su.psf, su.pixel_scale, su.sub, su.x0,
                     su.y0).loglike_batch(Pu.astype(np.float64))
    lenses = [_gpu(s0, batch_only=True), _gpu(su, batch_only=True), _gpu(s1, batch_only=True)]
    params = [torch.from_numpy(p).cuda() for p in (P0, Pu, P1)]
    for graph in (False, True):
        b = tll.Batcher(use_graph=graph)
        st = torch.cuda.Stream()
        with torch.cuda.stream(st):
            outs = b.run(lenses, params, stream=st)
            st.synchronize()
        for out, r, sl in zip(outs, (r0, ru, r1), (s0, su, s1)):
            _ll_ok(out.cpu().numpy(), r, sl)
        b.close()
    for L in lenses:
        L.close()
    g = _gpu(s1)
    g.set_conv(tll.CONV_SPLIT_DIRECT, chunk=16)
    _ll_ok(_run(g, P1), r1, s1)
    g.close()


def test_masked_multi_component(cases):
    sl0 = cases[0][0]
    comps = W.SLACS_COMPS
    rng = np.random.Generator(np.random.PCG64(7800))
    render = oracle.multi_columns_renderer(sl0.pixel_scale, sl0.sub, sl0.psf, sl0.ny, sl0.nx,
                                           comps)
    sl = W.synth_multi_lens(rng, sl0.ny, sl0.nx, sl0.pixel_scale, sl0.sub, sl0.psf, render,
                            comps)
    W.apply_mask(sl, W.annulus_mask(sl.ny, sl.nx, sl.pixel_scale, 0.3, 2.2, sl.x0, sl.y0))
    P = np.concatenate([sl.truth[None], W.shrinking_draws_multi(rng, sl.truth, 30, comps,
                                                                lo_frac=1e-6),
                        W.draw_prior_multi(rng, 9, comps)]).astype(np.float32)
    o = oracle.MultiLens(sl.data, sl.noise, sl.psf, sl.pixel_scale, sl.sub, comps, sl.x0, sl.y0)
    ref = o.loglike_batch(P.astype(np.float64))
    _, lognorm, _ = _lens_consts(sl)
    _CHI2_TRUTH[id(sl)] = (sl, max(-2.0 * (ref[0] - lognorm), 0.0))
    g = _gpu(sl)
    g.set_light([tll.comp(c["type"], c["plane"], index=c["index"]) for c in comps])
    _ll_ok(_run(g, P), ref, sl)
    cols = g.model_columns_n(P[0], blurred=True)   # every pixel, as the oracle
    assert np.max(np.abs(cols - o.model(P[0].astype(np.float64))[1])) <= 1e-4 * np.abs(cols).max()
    g.close()


def test_fully_masked_lens(cases):
    sl, P, o, ref = cases[1]
    noise = np.full_like(sl.noise, np.inf)
    g = tll.Lens(sl.data, noise, sl.psf, sl.pixel_scale, sl.sub, sl.x0, sl.y0)
    assert g.ntrace() == 0
    Q = P[:6].copy()
    Q[5, 8] = -1.0      # an invalid vector stays -inf
    out = _run(g, Q)
    assert np.all(out[:5] == 0.0) and np.isneginf(out[5])
    g.close()
