"""Edge cases of the multi-column and sampler paths against the FP64 oracle:
component lists confined to one plane (lens light only, lensed source
only), the largest supersampling factor (s = 8, the generic subpixel loop),
s = 1 with an odd column count, images convolved band by band (bands of
odd height included), an image
wider than 256 pixels (generic convolution), and the device sampler on a
masked power-law multi-component lens."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
from paper_2503_08586_gb300 import build, tll
from paper_2503_08586_gb300 import workloads as W

from test_multi_light_gpu import _case, _to_tll
from test_parity_gpu import POS_ERR, POS_ERR_SRC, _CHI2_TRUTH, _lens_consts, _ll_ok

pytestmark = pytest.mark.gpu

LENS_ONLY = [dict(type="sersic", plane="lens", index=1.0),
             dict(type="sersic", plane="lens", index=4.0),
             dict(type="gauss", plane="lens", free_scale=False, scale=0.2)]
SOURCE_ONLY = [dict(type="sersic", plane="source", free_index=True),
               dict(type="gauss", plane="source")]

EDGE = [
    ("lens_only", 30, 28, 0.07, 4, 9, "moffat", LENS_ONLY, "sie"),
    ("source_only", 32, 30, 0.07, 4, 11, "gaussian", SOURCE_ONLY, "epl"),
    ("sub8", 20, 18, 0.1, 8, 7, "gaussian", W.SLACS_COMPS, "sie"),
    ("sub1_odd", 40, 44, 0.06, 1, 13, "moffat", LENS_ONLY[:1] + SOURCE_ONLY, "sie"),
    # the compiled convolution band by band (the padded image exceeds shared memory)
    ("banded_160x150", 160, 150, 0.05, 3, 31, "moffat", W.SLACS_COMPS, "sie"),
    # the direct convolution two output rows per item (K <= 21) on bands of
    # odd height (the lower row of the last pair is not stored)
    ("banded_k21_163x150", 163, 150, 0.05, 3, 21, "moffat", W.SLACS_COMPS, "sie"),
    # nx > 256: the generic convolution on the global slots
    ("wide_10x300", 10, 300, 0.03, 2, 5, "gaussian", W.SLACS_COMPS, "sie"),
]


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    tll.load()
    assert torch.cuda.is_available()


def _grid_shift_allowance(sl, P, ref, comps, mass):
    """The oracle's |dlogL| per vector when the image grid moves by
    POS_ERR in x or in y (the FP32 position rounding; test_parity_gpu)."""
    allow = np.zeros_like(ref)
    for dx, dy in ((POS_ERR, 0.0), (0.0, POS_ERR)):
        o = oracle.MultiLens(sl.data, sl.noise, sl.psf, sl.pixel_scale, sl.sub, comps,
                             float(sl.x0) + dx, float(sl.y0) + dy, mass=mass)
        r = o.loglike_batch(P.astype(np.float64))
        fin = np.isfinite(ref)
        allow[fin] = np.maximum(allow[fin], np.abs(r[fin] - ref[fin]))
    return allow


def _multi_pix_allowance(o, p0):
    """The pixel gates' a_i for every blurred column of a multi-component
    model: the largest change of the oracle's column when the lens-light
    centre ([9], [10]) moves by +-POS_ERR and the source centre ([13], [14])
    by +-POS_ERR_SRC, in x and in y (test_parity_gpu._pix_allowance for the
    two-column layout)."""
    base = o.model(p0)[1]
    allow = np.zeros_like(base)
    for sx, sy in ((1, 0), (-1, 0), (0, 1), (0, -1)):
        q = p0.copy()
        q[9] += sx * POS_ERR; q[10] += sy * POS_ERR
        q[13] += sx * POS_ERR_SRC; q[14] += sy * POS_ERR_SRC
        allow = np.maximum(allow, np.abs(o.model(q)[1] - base))
    return allow


@pytest.mark.parametrize("spec", EDGE, ids=[e[0] for e in EDGE])
def test_edge_multi_loglike(spec):
    sl, P, o, ref = _case(90 + EDGE.index(spec), *spec)
    comps, mass = spec[7], spec[8]
    g = tll.Lens(sl.data, sl.noise, sl.psf, sl.pixel_scale, sl.sub, sl.x0, sl.y0, mass=mass)
    g.set_light(_to_tll(comps))
    if spec[0].startswith("banded"):
        sh = g.shape()
        assert sh["placement"] == "banded" and 0 < sh["band_rows"] < sl.ny
    out = g.loglike_batch(torch.from_numpy(np.ascontiguousarray(P)).cuda())
    torch.cuda.synchronize()
    _ll_ok(out.cpu().numpy(), ref, sl, allow=_grid_shift_allowance(sl, P, ref, comps, mass))
    # every blurred column of the true vector within the pixel gate, with its
    # per-pixel position allowance a_i
    p0 = P[0].astype(np.float64)
    gc = g.model_columns_n(P[0], blurred=True).astype(np.float64)
    oc = o.model(p0)[1]
    allow = _multi_pix_allowance(o, p0)
    for c in range(len(comps)):
        tol = 1e-5 * np.abs(oc[c]) + 1e-7 * np.abs(oc[c]).max() + allow[c]
        err = np.abs(gc[c] - oc[c])
        assert np.all(err <= tol), (
            f"column {c}: worst error / tol = {(err / np.maximum(tol, 1e-300)).max():.3f}")
    g.close()


def test_sampler_on_masked_epl_multi_lens():
    spec = ("slacs_epl_mask", 40, 40, 0.06, 4, 13, "gaussian", W.SLACS_COMPS, "epl")
    sl, P, o, ref = _case(95, *spec)
    W.apply_mask(sl, W.annulus_mask(sl.ny, sl.nx, sl.pixel_scale, 0.3, 1.1, sl.x0, sl.y0))
    comps = W.SLACS_COMPS
    om = oracle.MultiLens(sl.data, sl.noise, sl.psf, sl.pixel_scale, sl.sub, comps, sl.x0, sl.y0,
                          mass="epl")
    _, lognorm, _ = _lens_consts(sl)
    _CHI2_TRUTH[id(sl)] = (sl, max(-2.0 * (om.loglike(sl.truth) - lognorm), 0.0))
    g = tll.Lens(sl.data, sl.noise, sl.psf, sl.pixel_scale, sl.sub, sl.x0, sl.y0, mass="epl")
    g.set_light(_to_tll(comps))
    assert g.ntrace() < sl.ny * sl.nx
    lo = np.asarray(sl.truth, np.float32) - 0.2
    hi = np.asarray(sl.truth, np.float32) + 0.2
    lo[15:19], hi[15:19] = 0.03, 3.0
    lo[19], hi[19] = 1.5, 2.5
    rng = np.random.Generator(np.random.PCG64(9600))
    x0 = np.clip(sl.truth[None] + rng.normal(scale=0.005, size=(24, g.nparam)), lo, hi)
    S = tll.Sampler(g, 24, lo, hi, seed=3)
    S.set_walkers(torch.from_numpy(x0.astype(np.float32)).cuda())
    chain, lpc, _ = S.run(5)
    torch.cuda.synchronize()
    last = chain[-1].cpu().numpy()
    _ll_ok(lpc[-1].cpu().numpy(), om.loglike_batch(last.astype(np.float64)), sl)
    _, _, steps, nacc, nprop = S.state()
    assert steps == 5 and nprop == 5 * 24 and 0 < nacc <= nprop
    S.close()
    g.close()
