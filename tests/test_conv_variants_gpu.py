"""The PSF convolution (Eq. 3) four ways on the same lens and vectors: the
fused kernel (default), the split pipeline with a direct FP32 convolution, and
the split pipeline with the banded-Toeplitz GEMM on the tensor cores, in TF32
(three products per term) and in split BF16 (three parts per operand, six
products).  Each against the FP64 oracle: blurred model columns within the
pixel gate, log L within the parity gates."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
from paper_2503_08586_gb300 import build, tll
from paper_2503_08586_gb300 import workloads as W

from test_parity_gpu import _ll_ok, _pix_allowance, _pix_ok

pytestmark = pytest.mark.gpu

VARIANTS = [tll.CONV_FUSED, tll.CONV_SPLIT_DIRECT, tll.CONV_SPLIT_TOEPLITZ_TC,
            tll.CONV_SPLIT_TOEPLITZ_BF16]
# (ny, nx, pixel scale, s, PSF side, kind): the hst200 geometry at a smaller
# batch; ragged sizes with a small PSF; a PSF side the compiled split kernel
# does not cover; the largest side the Toeplitz tiles hold
LENSES = [(200, 200, 0.05, 5, 31, "moffat"), (37, 53, 0.06, 3, 7, "moffat"),
          (130, 70, 0.05, 2, 15, "gaussian"), (64, 64, 0.05, 2, 33, "moffat")]


@pytest.fixture(scope="module")
def cases():
    build.build()
    tll.load()
    assert torch.cuda.is_available()
    out = []
    for k, (ny, nx, dpix, sub, ks, kind) in enumerate(LENSES):
        psf = W.moffat_psf(ks, 2.0, 3.0) if kind == "moffat" else W.gaussian_psf(ks, ks / 7.0)
        rng = np.random.Generator(np.random.PCG64(5200 + k))
        render = oracle.columns_renderer(dpix, sub, psf, ny, nx)
        sl = W.synth_lens(rng, ny, nx, dpix, sub, psf, render, "sky+poisson")
        P = np.concatenate([W.shrinking_draws(rng, sl.truth, 40, lo_frac=1e-5),
                            W.draw_prior(rng, 20)]).astype(np.float32)
        P[3, 1], P[3, 2] = 0.9, 0.5        # |eps| >= 1: invalid
        o = oracle.Lens(sl.data, sl.noise, sl.psf, sl.pixel_scale, sl.sub, sl.x0, sl.y0)
        ref = o.loglike_batch(P.astype(np.float64))
        cols = [o.model(P[j].astype(np.float64), mode=1)[1:3] for j in (0, 25, 45)]
        allows = [_pix_allowance(o, P[j], blurred=True) for j in (0, 25, 45)]
        out.append((sl, P, ref, cols, allows))
    return out


@pytest.mark.parametrize("variant", VARIANTS,
                         ids=["fused", "split_direct", "split_tc", "split_bf16"])
@pytest.mark.parametrize("idx", range(len(LENSES)))
def test_variant_against_oracle(cases, idx, variant):
    sl, P, ref, cols, allows = cases[idx]
    g = tll.Lens(sl.data, sl.noise, sl.psf, sl.pixel_scale, sl.sub, sl.x0, sl.y0,
                 direct_conv=True)
    g.set_conv(variant, chunk=16)      # several passes of the split pipeline
    out = g.loglike_batch(torch.from_numpy(P).cuda())
    torch.cuda.synchronize()
    g.conv_check()
    got = out.cpu().numpy()
    assert np.isneginf(got[3])
    _ll_ok(got, ref, sl)
    for j, (ml, ms), ab in zip((0, 25, 45), cols, allows):
        bl, bs = g.model_columns(P[j], blurred=True)
        for gg, oo, aa, nm in ((bl, ml, ab[0], "lens"), (bs, ms, ab[1], "source")):
            ok, worst = _pix_ok(np.asarray(gg).reshape(oo.shape), oo, aa)
            assert ok, f"vector {j} {nm}: worst pixel error / tol = {worst:.3f}"
    g.conv_check()
    g.close()


def test_variants_agree(cases):
    sl, P, ref, _, _ = cases[0]
    g = tll.Lens(sl.data, sl.noise, sl.psf, sl.pixel_scale, sl.sub, sl.x0, sl.y0)
    Pd = torch.from_numpy(P).cuda()
    res = []
    for v in VARIANTS:
        g.set_conv(v)
        o = g.loglike_batch(Pd)
        torch.cuda.synchronize()
        res.append(o.cpu().numpy())
    g.conv_check()
    fin = np.isfinite(res[0])
    for r in res[1:]:
        assert np.array_equal(fin, np.isfinite(r))
        assert np.allclose(r[fin], res[0][fin], rtol=1e-6, atol=1e-2)
    g.close()


def test_bad_variant(cases):
    sl = cases[1][0]
    g = tll.Lens(sl.data, sl.noise, sl.psf, sl.pixel_scale, sl.sub, sl.x0, sl.y0)
    with pytest.raises(tll.TLLError) as e:
        g.set_conv(7)
    assert e.value.code == tll.EINVAL
    g.close()
