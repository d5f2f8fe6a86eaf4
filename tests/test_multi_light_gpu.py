"""Multi-component light with N-column FNNLS (Sec. 2.3, Eq. 7; Sec. 3.2's
double Sersic; Gaussian components), through the C ABI, against the FP64
oracle: unblurred and blurred columns per pixel, log L per vector (the
parity gates of test_parity_gpu), model images, invalid vectors, the
no-allocation entry point, and the calls that refuse such lenses (launch
shapes, the autotuner, the split convolutions; the batcher and the server
take them, tests/test_multi_batch_gpu.py)."""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
from paper_2503_08586_gb300 import build, tll
from paper_2503_08586_gb300 import workloads as W

from test_parity_gpu import (PIX_FLOOR, PIX_REL, POS_ERR, POS_ERR_SRC, _CHI2_TRUTH,
                             _lens_consts, _ll_ok, _pix_ok)

pytestmark = pytest.mark.gpu

MIXED = [dict(type="sersic", plane="lens", free_index=True),
         dict(type="gauss", plane="lens", free_scale=False, scale=0.3),
         dict(type="sersic", plane="lens", index=4.0),
         dict(type="gauss", plane="lens"),
         dict(type="sersic", plane="lens", index=1.0, free_scale=False, scale=0.6),
         dict(type="sersic", plane="source", free_index=True),
         dict(type="gauss", plane="source")]     # 7 columns, two lens passes

# 20 columns: 3 Sersic passes per plane mixed with Gaussian passes
MANY = ([dict(type="sersic", plane="lens", index=float(n)) for n in (0.7, 1.0, 1.6, 2.5, 4.0, 6.0)]
        + [dict(type="gauss", plane="lens", free_scale=False, scale=float(sg))
           for sg in np.geomspace(0.05, 1.5, 5)]
        + [dict(type="sersic", plane="source", index=float(n), free_index=(n == 1.0))
           for n in (0.8, 1.0, 2.0, 3.0, 4.5)]
        + [dict(type="gauss", plane="source") for _ in range(4)])

# (name, ny, nx, pixel scale, s, PSF side, PSF kind, components, mass)
CASES = [
    ("slacs_direct", 48, 40, 0.05, 4, 9, "moffat", W.SLACS_COMPS, "sie"),
    ("slacs_sep", 44, 52, 0.06, 5, 11, "gaussian", W.SLACS_COMPS, "sie"),
    ("mixed_odd", 36, 36, 0.07, 3, 7, "moffat", MIXED, "sie"),
    ("mge_generic", 30, 34, 0.08, 4, 33, "moffat", W.MGE_COMPS, "sie"),
    ("slacs_epl", 40, 40, 0.06, 4, 13, "gaussian", W.SLACS_COMPS, "epl"),
    ("mge32", 40, 36, 0.07, 3, 9, "gaussian", W.MGE32_COMPS, "sie"),
    ("many20_generic", 34, 30, 0.08, 2, 33, "moffat", MANY, "sie"),
    ("tiny_1x1", 1, 1, 0.1, 1, 1, "gaussian", W.SLACS_COMPS, "sie"),
    ("tiny_3x2", 3, 2, 0.2, 4, 5, "moffat", MIXED, "sie"),
    ("column_7x1", 7, 1, 0.1, 3, 5, "gaussian", MIXED, "sie"),
]


def _to_tll(comps):
    return [tll.comp(c["type"], c["plane"], c.get("free_scale", True),
                     c.get("free_index", False), c.get("scale", 1.0), c.get("index", 1.0))
            for c in comps]


def _case(k, name, ny, nx, dpix, sub, ks, kind, comps, mass):
    psf = W.moffat_psf(ks, 2.2, 3.0) if kind == "moffat" else W.gaussian_psf(ks, ks / 6.0)
    rng = np.random.Generator(np.random.PCG64(7300 + k))
    render = oracle.multi_columns_renderer(W.f32(dpix), sub, psf, ny, nx, comps, mass=mass)
    sl = W.synth_multi_lens(rng, ny, nx, dpix, sub, psf, render, comps, mass=mass)
    P = np.concatenate([sl.truth[None],
                        W.shrinking_draws_multi(rng, sl.truth, 40, comps, lo_frac=1e-6),
                        W.draw_prior_multi(rng, 23, comps, mass)]).astype(np.float32)
    o = oracle.MultiLens(sl.data, sl.noise, sl.psf, sl.pixel_scale, sl.sub, comps,
                         sl.x0, sl.y0, mass=mass)
    ref = o.loglike_batch(P.astype(np.float64))
    _, lognorm, _ = _lens_consts(sl)
    _CHI2_TRUTH[id(sl)] = (sl, max(-2.0 * (ref[0] - lognorm), 0.0))
    return sl, P, o, ref


@pytest.fixture(scope="module")
def cases():
    build.build()
    tll.load()
    assert torch.cuda.is_available()
    return [_case(k, *c) for k, c in enumerate(CASES)]


def _gpu(sl, comps, mass="sie", **kw):
    g = tll.Lens(sl.data, sl.noise, sl.psf, sl.pixel_scale, sl.sub, sl.x0, sl.y0,
                 mass=mass, **kw)
    g.set_light(_to_tll(comps))
    return g


def _allowance(o, p, blurred):
    """Per-pixel allowance per column: the oracle column's change when both
    planes' centres ([9], [10] by +-POS_ERR and [13], [14] by +-POS_ERR_SRC)
    move."""
    def cols(q):
        return o.model(q)[1] if blurred else o.unblurred(q)
    p0 = np.asarray(p, np.float64)
    base = cols(p0)
    allow = np.zeros_like(base)
    for sx, sy in ((1, 0), (-1, 0), (0, 1), (0, -1)):
        q = p0.copy()
        q[9] += sx * POS_ERR; q[10] += sy * POS_ERR
        q[13] += sx * POS_ERR_SRC; q[14] += sy * POS_ERR_SRC
        allow = np.maximum(allow, np.abs(cols(q) - base))
    return allow


@pytest.mark.parametrize("idx", range(len(CASES)))
def test_multi_columns_and_loglike(cases, idx):
    sl, P, o, ref = cases[idx]
    comps, mass = CASES[idx][7], CASES[idx][8]
    g = _gpu(sl, comps, mass)
    assert g.nparam == o.nparam and g.ncols == len(comps)
    for j in (0, 7, 40, 45, 60):
        for blurred in (False, True):
            gc = g.model_columns_n(P[j], blurred=blurred)
            oc = o.model(P[j].astype(np.float64))[1] if blurred else o.unblurred(
                P[j].astype(np.float64))
            al = _allowance(o, P[j], blurred)
            for c in range(len(comps)):
                ok, worst = _pix_ok(gc[c], oc[c], al[c])
                assert ok, f"vector {j} column {c} blurred={blurred}: worst/tol {worst:.3f}"
    out = g.loglike_batch(torch.from_numpy(P).cuda())
    torch.cuda.synchronize()
    _ll_ok(out.cpu().numpy(), ref, sl)
    g.close()


def test_multi_model_image_and_amplitudes(cases):
    """The model image (sum_k s_k M_k) is unique; amplitudes of the truth
    vector (well separated columns) agree to 1e-4 relative; model_image's
    log L is the batch's."""
    for idx in (0, 2):
        sl, P, o, ref = cases[idx]
        g = _gpu(sl, CASES[idx][7])
        for j in (0, 20):
            img, amps, ll = g.model_image(P[j])
            oll, _, omod, oamps = o.model(P[j].astype(np.float64))
            assert abs(ll - oll) <= 1e-3
            assert np.max(np.abs(img - omod)) <= 1e-4 * np.abs(omod).max()
            big = oamps > 1e-3 * oamps.max()
            assert np.all(np.abs(amps[big] - oamps[big]) <= 1e-4 * oamps[big] + 1e-6 * oamps.max())
        g.close()


def test_multi_sie_form_boundaries(cases):
    """The multi-column kernel's SIE closed forms (fast for q >= sqrt(3)/2,
    mid for 1/sqrt(2) <= q < sqrt(3)/2, general below) on both sides of each
    switch, at two position angles: blurred columns within the pixel gate
    and log L within the gates."""
    sl, P, o, ref = cases[1]
    comps = CASES[1][7]
    g = _gpu(sl, comps)
    vecs = []
    for q in (0.99, 0.8662, 0.8659, 0.7072, 0.7070, 0.55):
        for phi in (0.3, 1.9):
            p = np.array(P[0], np.float64)
            e = (1.0 - q) / (1.0 + q)
            p[1], p[2] = e * np.cos(2 * phi), e * np.sin(2 * phi)
            vecs.append(p.astype(np.float32))
    Q = np.stack(vecs)
    for p in Q:
        gc = g.model_columns_n(p, blurred=True)
        oc = o.model(p.astype(np.float64))[1]
        al = _allowance(o, p, True)
        for c in range(len(comps)):
            ok, worst = _pix_ok(gc[c], oc[c], al[c])
            assert ok, f"column {c}: worst/tol {worst:.3f}"
    got = g.loglike_batch(torch.from_numpy(Q).cuda())
    torch.cuda.synchronize()
    _ll_ok(got.cpu().numpy(), o.loglike_batch(Q.astype(np.float64)), sl)
    g.close()


def test_multi_invalid_vectors(cases):
    sl, P, o, ref = cases[2]      # MIXED: slots 15 r_e, 16 n, 17 sigma, 18 r_e, 19 r_e, 20 n, 21 sigma
    Q = np.repeat(P[:1], 9, axis=0)
    Q[1, 15] = 0.0        # r_e = 0
    Q[2, 16] = 0.1        # index below 0.2
    Q[3, 20] = 10.5       # index above 10
    Q[4, 17] = -0.2       # sigma < 0
    Q[5, 21] = np.nan
    Q[6, 7], Q[6, 8] = 0.8, 0.7   # |eps_L| >= 1
    Q[7, 0] = -0.1        # theta_E < 0
    g = _gpu(sl, CASES[2][7])
    got = g.loglike_batch(torch.from_numpy(Q).cuda())
    torch.cuda.synchronize()
    got = got.cpu().numpy()
    oref = o.loglike_batch(Q.astype(np.float64))
    assert np.isneginf(oref[1:8]).all() and np.isneginf(got[1:8]).all()
    _ll_ok(got, oref, sl)
    with pytest.raises(tll.TLLError):
        g.model_image(Q[1])
    g.close()


def test_multi_noalloc_host_and_revert(cases):
    sl, P, o, ref = cases[1]
    g = _gpu(sl, CASES[1][7])
    p = torch.from_numpy(P).cuda()
    a = g.loglike_batch(p)
    b = torch.empty_like(a)
    g.loglike_batch_noalloc(p, b)
    torch.cuda.synchronize()
    assert torch.equal(a, b)
    h = g.loglike_batch_host(P)
    assert np.array_equal(h, a.cpu().numpy())
    # back to the two-column model: 21 parameters again
    g.set_light([])
    assert g.nparam == 21 and g.ncols == 2
    g.close()


def test_multi_refused_by_shape_and_conv_variants(cases):
    sl, P, o, ref = cases[0]
    g = _gpu(sl, CASES[0][7])
    for call in (lambda: g.set_conv(tll.CONV_SPLIT_DIRECT),
                 lambda: g.set_shape(512, 2), lambda: g.autotune(),
                 lambda: g.model_columns(P[0])):
        with pytest.raises(tll.TLLError) as e:
            call()
        assert e.value.code == tll.EINVAL
    # bad component lists
    lib = tll.load()
    bad = [tll.Comp(7, 0, 1, 1.0, 1.0)]
    arr = (tll.Comp * 1)(*bad)
    assert lib.tll_set_light(g.handle, arr, 1) == tll.EINVAL
    arr = (tll.Comp * 1)(tll.Comp(0, 0, 0, 0.5, 12.0))   # fixed index out of range
    assert lib.tll_set_light(g.handle, arr, 1) == tll.EINVAL
    arr = (tll.Comp * 33)(*[tll.comp("gauss", "lens")] * 33)
    assert lib.tll_set_light(g.handle, arr, 33) == tll.EINVAL
    assert g.nparam == o.nparam          # the lens kept its model
    g.close()


@pytest.mark.parametrize("name", ["slacs120", "mge120", "mge32"])
def test_multi_full_size_sampled(name):
    """The bench workloads at full size, in the launch configuration the
    bench times (the whole batch in one call): 48 sampled vectors (the
    truth, a converging chain, prior draws) against the oracle."""
    build.build()
    sl, P = W.multi_workload(name, oracle.multi_columns_renderer)
    comps = W.MULTI_WORKLOADS[name].comps
    rng = np.random.Generator(np.random.PCG64(7400))
    P = np.concatenate([sl.truth[None], W.shrinking_draws_multi(rng, sl.truth, 300, comps,
                                                                lo_frac=1e-5), P])
    g = _gpu(sl, comps)
    out = g.loglike_batch(torch.from_numpy(np.ascontiguousarray(P)).cuda())
    torch.cuda.synchronize()
    out = out.cpu().numpy()
    pick = np.r_[0, 1:300:20, 280:300:4, 301 + rng.choice(P.shape[0] - 301, 27, replace=False)]
    o = oracle.MultiLens(sl.data, sl.noise, sl.psf, sl.pixel_scale, sl.sub, comps, sl.x0, sl.y0)
    ref = o.loglike_batch(P[pick].astype(np.float64))
    _, lognorm, _ = _lens_consts(sl)
    _CHI2_TRUTH[id(sl)] = (sl, max(-2.0 * (ref[0] - lognorm), 0.0))
    _ll_ok(out[pick], ref, sl)
    g.close()
