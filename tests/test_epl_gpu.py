"""The elliptical power-law mass (Eq. 12 at any slope; lenses created with
TLL_MASS_EPL, 22 parameters): model columns and log L against the FP64
oracle, validity of the slope, and the batcher, server and split pipeline
with EPL and SIE lenses together."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
from paper_2503_08586_gb300 import build, tll
from paper_2503_08586_gb300 import workloads as W

from test_parity_gpu import _ll_ok, _pix_allowance, _pix_ok

pytestmark = pytest.mark.gpu

# (ny, nx, pixel scale, s, PSF side, PSF kind)
SHAPES = [(100, 100, 0.074, 4, 21, "gaussian"), (37, 53, 0.06, 3, 7, "moffat"),
          (64, 64, 0.05, 5, 11, "gaussian")]


def _epl_lens(k, ny, nx, dpix, sub, ks, kind):
    psf = W.moffat_psf(ks, 2.0, 3.0) if kind == "moffat" else W.gaussian_psf(ks, ks / 7.0)
    rng = np.random.Generator(np.random.PCG64(6100 + k))
    render = oracle.columns_renderer(dpix, sub, psf, ny, nx, mass="epl")
    sl = W.synth_lens(rng, ny, nx, dpix, sub, psf, render, "sky+poisson", mass="epl")
    P = np.concatenate([W.shrinking_draws(rng, sl.truth, 48, lo_frac=1e-6),
                        W.draw_prior(rng, 24, "epl")]).astype(np.float32)
    # prior draws with steeper / shallower slopes and flatter ellipses
    P[48:54, 21] = [1.15, 1.4, 2.6, 2.9, 2.0, 1.05]
    P[54:58, 1] = [0.5, -0.45, 0.3, 0.58]
    return sl, P


@pytest.fixture(scope="module")
def cases():
    build.build()
    tll.load()
    assert torch.cuda.is_available()
    out = []
    for k, spec in enumerate(SHAPES):
        sl, P = _epl_lens(k, *spec)
        o = oracle.Lens(sl.data, sl.noise, sl.psf, sl.pixel_scale, sl.sub, sl.x0, sl.y0,
                        mass="epl")
        out.append((sl, P, o, o.loglike_batch(P.astype(np.float64))))
    return out


def _gpu(sl, **kw):
    return tll.Lens(sl.data, sl.noise, sl.psf, sl.pixel_scale, sl.sub, sl.x0, sl.y0,
                    mass="epl", **kw)


@pytest.mark.parametrize("idx", range(len(SHAPES)))
def test_epl_columns_and_loglike(cases, idx):
    sl, P, o, ref = cases[idx]
    g = _gpu(sl)
    assert g.nparam == 22
    for j in (0, 10, 47, 50, 55):
        il, is_ = o.unblurred(P[j].astype(np.float64))
        gl, gs = g.model_columns(P[j], blurred=False)
        au = _pix_allowance(o, P[j], blurred=False)
        for gg, oo, aa, nm in ((gl, il, au[0], "lens"), (gs, is_, au[1], "source")):
            ok, worst = _pix_ok(np.asarray(gg).reshape(oo.shape), oo, aa)
            assert ok, f"vector {j} unblurred {nm}: worst error / tol {worst:.3f}"
    out = g.loglike_batch(torch.from_numpy(P).cuda())
    torch.cuda.synchronize()
    _ll_ok(out.cpu().numpy(), ref, sl)
    g.close()


def test_epl_table_switch(cases):
    """Either side of the switch between the per-vector table of the
    deflection's series and the per-subpixel recurrence ((1-q)/(1+q) = |eps|
    = 0.35), at two position angles: columns within the pixel gate and log L
    within the gates."""
    sl, P, o, ref = cases[1]
    g = _gpu(sl)
    Q = np.repeat(P[:1], 4, axis=0)
    for i, (e, phi) in enumerate(((0.3499, 0.4), (0.3501, 0.4), (0.3499, 2.0), (0.3501, 2.0))):
        Q[i, 1], Q[i, 2] = e * np.cos(2 * phi), e * np.sin(2 * phi)
    for p in Q:
        il, is_ = o.unblurred(p.astype(np.float64))
        gl, gs = g.model_columns(p, blurred=False)
        au = _pix_allowance(o, p, blurred=False)
        for gg, oo, aa, nm in ((gl, il, au[0], "lens"), (gs, is_, au[1], "source")):
            ok, worst = _pix_ok(np.asarray(gg).reshape(oo.shape), oo, aa)
            assert ok, f"|eps| {np.hypot(p[1], p[2]):.4f} {nm}: worst error / tol {worst:.3f}"
    out = g.loglike_batch(torch.from_numpy(Q).cuda())
    torch.cuda.synchronize()
    _ll_ok(out.cpu().numpy(), o.loglike_batch(Q.astype(np.float64)), sl)
    g.close()


def test_epl_slope_validity(cases):
    sl, P, o, ref = cases[1]
    Q = P[:8].copy()
    Q[:, 21] = [1.0, 3.0, np.nan, 0.5, 1.01, 2.99, 2.0, 1.5]
    g = _gpu(sl)
    got = g.loglike_batch(torch.from_numpy(Q).cuda())
    torch.cuda.synchronize()
    got = got.cpu().numpy()
    assert np.isneginf(got[:4]).all() and np.isfinite(got[4:]).all()
    _ll_ok(got, o.loglike_batch(Q.astype(np.float64)), sl)
    g.close()


def test_epl_at_slope_two_is_the_sie(cases):
    sl, P, _, _ = cases[0]
    Q = P[:32].copy()
    Q[:, 21] = 2.0
    ge, gs = _gpu(sl), tll.Lens(sl.data, sl.noise, sl.psf, sl.pixel_scale, sl.sub, sl.x0, sl.y0)
    a = ge.loglike_batch(torch.from_numpy(Q).cuda())
    b = gs.loglike_batch(torch.from_numpy(np.ascontiguousarray(Q[:, :21])).cuda())
    torch.cuda.synchronize()
    os_ = oracle.Lens(sl.data, sl.noise, sl.psf, sl.pixel_scale, sl.sub, sl.x0, sl.y0)
    ref = os_.loglike_batch(Q[:, :21].astype(np.float64))
    _ll_ok(a.cpu().numpy(), ref, sl)
    _ll_ok(b.cpu().numpy(), ref, sl)
    ge.close()
    gs.close()


def test_epl_in_batcher_server_and_split(cases):
    (sl0, P0, _, ref0), (sl1, P1, _, ref1) = cases[0], cases[1]
    # an SIE lens in the same batches
    rng = np.random.Generator(np.random.PCG64(6200))
    psf = W.gaussian_psf(9, 1.8)
    sls = W.synth_lens(rng, 48, 40, 0.05, 4, psf,
                       oracle.columns_renderer(0.05, 4, psf, 48, 40), "sky")
    Ps = W.shrinking_draws(rng, sls.truth, 40, lo_frac=1e-6)
    refs = oracle.Lens(sls.data, sls.noise, sls.psf, sls.pixel_scale, sls.sub, sls.x0,
                       sls.y0).loglike_batch(Ps.astype(np.float64))
    lenses = [_gpu(sl0, batch_only=True), _gpu(sl1, batch_only=True),
              tll.Lens(sls.data, sls.noise, sls.psf, sls.pixel_scale, sls.sub, sls.x0,
                       sls.y0, batch_only=True)]
    params = [torch.from_numpy(p).cuda() for p in (P0, P1, Ps)]
    for graph in (False, True):
        b = tll.Batcher(use_graph=graph)
        st = torch.cuda.Stream()
        with torch.cuda.stream(st):
            outs = b.run(lenses, params, stream=st)
            st.synchronize()
        for o, r, sl in zip(outs, (ref0, ref1, refs), (sl0, sl1, sls)):
            _ll_ok(o.cpu().numpy(), r, sl)
        b.close()
    # the server, an EPL job beside an SIE job
    S = tll.Server(max_jobs=4)
    je = S.open_job(sl1.data, sl1.noise, sl1.psf, sl1.pixel_scale, sl1.sub, sl1.x0, sl1.y0,
                    mass="epl")
    js = S.open_job(sls.data, sls.noise, sls.psf, sls.pixel_scale, sls.sub, sls.x0, sls.y0)
    r1, r2 = S.submit(je, P1), S.submit(js, Ps)
    _ll_ok(S.wait(r1)[0], ref1, sl1)
    _ll_ok(S.wait(r2)[0], refs, sls)
    assert S.close_job(je) and S.close_job(js)
    S.close()
    # the split pipeline (both convolutions)
    for v in (tll.CONV_SPLIT_DIRECT, tll.CONV_SPLIT_TOEPLITZ_TC):
        g = _gpu(sl0)
        g.set_conv(v, chunk=32)
        out = g.loglike_batch(torch.from_numpy(P0).cuda())
        torch.cuda.synchronize()
        g.conv_check()
        _ll_ok(out.cpu().numpy(), ref0, sl0)
        g.close()
    for L in lenses:
        L.close()
