"""The device-side sampler loop (tll_sampler: the stretch move with
Philox4x32-10, the paper's Sec. 4.2 proposal of a GPU-resident sampler)
through the C ABI.  The oracle replays every half step from the same walkers:
its proposals (the same generator and the same once-rounded FP64
arithmetic) must reproduce the GPU's walker states bit for bit, its accept /
reject decisions -- taken in FP64 from the GPU's proposal log posteriors --
must match, and those log posteriors must match the oracle's likelihood."""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
from paper_2503_08586_gb300 import build, tll
from paper_2503_08586_gb300 import workloads as W

from test_parity_gpu import POS_ERR, _CHI2_TRUTH, _lens_consts, _ll_ok

pytestmark = pytest.mark.gpu

SEED = 0x5DEECE66D2503
A = 2.0


def _lens(k=0):
    rng = np.random.Generator(np.random.PCG64(7900 + k))
    psf = W.gaussian_psf(9, 1.8)
    sl = W.synth_lens(rng, 40, 44, 0.06, 4, psf, oracle.columns_renderer(W.f32(0.06), 4, psf,
                                                                          40, 44), "sky")
    return sl, rng


def _box(truth):
    """Uniform box prior around the truth; the amplitude slots and the tied
    lens-light centre are fixed (lo == hi) or move with the mass centre."""
    lo = np.asarray(truth, np.float32) - np.float32(0.5)
    hi = np.asarray(truth, np.float32) + np.float32(0.5)
    lo[[7, 14]] = hi[[7, 14]] = 1.0
    lo[[9, 16]], hi[[9, 16]] = 0.5, 6.0
    lo[[8, 15]], hi[[8, 15]] = 0.02, 3.0
    return lo, hi


def _shift_allowance(sl, P, ref):
    """The oracle's |dlogL| per vector when the image grid moves by POS_ERR
    in x or in y (the FP32 position rounding, as in the parity tests): the
    log L gates' allowance away from the posterior bulk, where a cusp of the
    light or the deflection makes log L sensitive to the coordinates'
    rounding."""
    allow = np.zeros_like(ref)
    fin = np.isfinite(ref)
    for dx, dy in ((POS_ERR, 0.0), (0.0, POS_ERR)):
        o = oracle.Lens(sl.data, sl.noise, sl.psf, sl.pixel_scale, sl.sub,
                        float(sl.x0) + dx, float(sl.y0) + dy)
        r = o.loglike_batch(np.asarray(P, np.float64))
        allow[fin] = np.maximum(allow[fin], np.abs(r[fin] - ref[fin]))
    return allow


def _start(rng, truth, nw, lo, hi):
    x = np.repeat(np.asarray(truth, np.float32)[None], nw, axis=0)
    x[:, [7, 14]] = 1.0
    free = np.where(lo < hi)[0]
    x[:, free] += rng.normal(scale=0.02, size=(nw, free.size)).astype(np.float32)
    x[:, 12], x[:, 13] = x[:, 3], x[:, 4]
    return np.clip(x, lo, hi).astype(np.float32)


# 48 walkers: each half step is one likelihood launch with the proposals and
# the accept / reject fused in (halves within the grid); 640: the separate
# proposal and accept kernels around the batched likelihood (halves beyond
# the grid of 152 SMs x up to 2 CTAs)
@pytest.mark.parametrize("nw,nsteps", [(48, 12), (640, 3)], ids=["fused", "separate"])
def test_sampler_chain_replays_in_the_oracle(nw, nsteps):
    build.build()
    sl, rng = _lens()
    g = tll.Lens(sl.data, sl.noise, sl.psf, sl.pixel_scale, sl.sub, sl.x0, sl.y0)
    o = oracle.Lens(sl.data, sl.noise, sl.psf, sl.pixel_scale, sl.sub, sl.x0, sl.y0)
    lo, hi = _box(sl.truth)
    x0 = _start(rng, sl.truth, nw, lo, hi)
    ndim = int(np.sum(lo < hi)) - 2     # x_L, y_L follow x_m, y_m
    S = tll.Sampler(g, nw, lo, hi, a=A, ndim=ndim, seed=SEED)
    S.set_walkers(torch.from_numpy(x0).cuda())
    _, lp0, step0, acc0, _ = S.state()
    lp0 = lp0.cpu().numpy()
    ref0 = o.loglike_batch(x0.astype(np.float64))
    _ll_ok(lp0, ref0, sl, allow=_shift_allowance(sl, x0, ref0))
    chain, lpc, lpp = S.run(nsteps, keep_proposals=True)
    xf, lpf, steps, nacc, nprop = S.state()
    torch.cuda.synchronize()
    chain, lpc, lpp = chain.cpu().numpy(), lpc.cpu().numpy(), lpp.cpu().numpy()
    assert steps == nsteps and nprop == nsteps * nw and step0 == 0 and acc0 == 0
    # replay
    x, lp = x0.copy(), lp0.copy()
    total = 0
    for s in range(nsteps):
        for h in (0, 1):
            Y, z, j = oracle.stretch_propose(x, h, s, SEED, A)
            half = slice(h * nw // 2, (h + 1) * nw // 2)
            if s < 2:   # the GPU's proposal log posteriors against the oracle's likelihood
                inside = np.all((Y >= lo) | (lo == hi), axis=1) & np.all((Y <= hi) | (lo == hi),
                                                                          axis=1)
                ref = o.loglike_batch(Y[inside].astype(np.float64))
                _ll_ok(lpp[s, half][inside], ref, sl, allow=_shift_allowance(sl, Y[inside], ref))
                assert np.all(np.isneginf(lpp[s, half][~inside]))
            acc = oracle.stretch_accept(x, lp, h, s, SEED, ndim, Y, z, lpp[s, half], lo, hi)
            total += int(acc.sum())
        assert np.array_equal(chain[s], x), f"walkers differ after step {s}"
        assert np.array_equal(lpc[s], lp)
    assert total == nacc > 0
    assert np.array_equal(xf.cpu().numpy(), x)
    # lo == hi entries never moved; the tied centre still follows the mass centre
    assert np.all(chain[..., 7] == 1.0) and np.all(chain[..., 14] == 1.0)
    S.close()
    g.close()


def test_sampler_determinism_and_continuation():
    """Same seed: the same chain; one run of 6 steps equals runs of 2 + 4;
    another seed: another chain."""
    sl, rng = _lens(1)
    g = tll.Lens(sl.data, sl.noise, sl.psf, sl.pixel_scale, sl.sub, sl.x0, sl.y0)
    lo, hi = _box(sl.truth)
    x0 = torch.from_numpy(_start(rng, sl.truth, 32, lo, hi)).cuda()
    chains = []
    for seed, split in ((5, None), (5, 2), (6, None)):
        S = tll.Sampler(g, 32, lo, hi, seed=seed)
        S.set_walkers(x0)
        if split:
            a, _, _ = S.run(split)
            b, _, _ = S.run(6 - split)
            c = torch.cat([a, b])
        else:
            c, _, _ = S.run(6)
        torch.cuda.synchronize()
        chains.append(c.cpu().numpy())
        S.close()
    assert np.array_equal(chains[0], chains[1])
    assert not np.array_equal(chains[0], chains[2])
    g.close()


def test_sampler_on_a_multi_component_lens_and_errors():
    comps = W.SLACS_COMPS
    rng = np.random.Generator(np.random.PCG64(7950))
    psf = W.gaussian_psf(9, 1.8)
    render = oracle.multi_columns_renderer(W.f32(0.06), 4, psf, 36, 36, comps)
    sl = W.synth_multi_lens(rng, 36, 36, 0.06, 4, psf, render, comps)
    g = tll.Lens(sl.data, sl.noise, sl.psf, sl.pixel_scale, sl.sub, sl.x0, sl.y0)
    g.set_light([tll.comp(c["type"], c["plane"], index=c["index"]) for c in comps])
    P = g.nparam
    lo = np.asarray(sl.truth, np.float32) - 0.3
    hi = np.asarray(sl.truth, np.float32) + 0.3
    lo[15:], hi[15:] = 0.03, 3.0
    x0 = np.clip(sl.truth[None] + rng.normal(scale=0.01, size=(16, P)), lo, hi).astype(np.float32)
    S = tll.Sampler(g, 16, lo, hi, seed=9)
    S.set_walkers(torch.from_numpy(x0).cuda())
    chain, lpc, _ = S.run(4)
    torch.cuda.synchronize()
    o = oracle.MultiLens(sl.data, sl.noise, sl.psf, sl.pixel_scale, sl.sub, comps, sl.x0, sl.y0)
    last = chain[-1].cpu().numpy()
    ref = o.loglike_batch(last.astype(np.float64))
    _, lognorm, _ = _lens_consts(sl)
    _CHI2_TRUTH[id(sl)] = (sl, max(-2.0 * (o.loglike(sl.truth) - lognorm), 0.0))
    _ll_ok(lpc[-1].cpu().numpy(), ref, sl)
    S.close()
    lib = tll.load()
    h = ctypes.c_void_p()
    bad = np.zeros(P, np.float32)
    assert lib.tll_sampler_create(g.handle, 7, bad.ctypes.data, bad.ctypes.data, 2.0, 0, 1,
                                  ctypes.byref(h)) == tll.EINVAL   # odd W
    assert lib.tll_sampler_create(g.handle, 8, hi.ctypes.data, lo.ctypes.data, 2.0, 0, 1,
                                  ctypes.byref(h)) == tll.EINVAL   # lo > hi
    with pytest.raises(tll.TLLError):
        S2 = tll.Sampler(g, 8, lo, hi)
        S2.run(1)          # walkers not set
    g.close()
