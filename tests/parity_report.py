"""Error of the CUDA path against the FP64 oracle, per workload (run on a GPU):

    python tests/parity_report.py > parity.md

For each workload: the worst per-pixel error of the model columns (lens and
source light, before and after the PSF) relative to the pixel gate
1e-5 |m| + 1e-7 max|m|, over the true vector and prior draws; and |dlogL| by
region -- the posterior bulk (chi^2 within 50 of the truth's), the rest of
chi^2 <= 2N, and prior draws -- plus the error of log L differences between
bulk vectors (what a sampler compares).  hst200 is reported again with the
split pipeline's two convolutions (direct FP32, and the banded-Toeplitz GEMM
on the tensor cores); csst100_mask is csst100 fitted in an annulus; the
multi-component workloads report every column.  Inputs are the seeded synthetic workloads; nothing is
stored.
"""
import os
import sys

import numpy as np

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, os.path.dirname(os.path.abspath(__file__)))

import torch  # noqa: E402

import oracle  # noqa: E402
from paper_2503_08586_gb300 import build, tll  # noqa: E402
from paper_2503_08586_gb300 import workloads as W  # noqa: E402
from test_parity_gpu import (BULK_DCHI2, POS_ERR, POS_ERR_SRC, _chi2_truth,  # noqa: E402
                             _lens_consts, _pix_allowance)


def pix_ratio(gpu, ora, allow):
    ora = np.asarray(ora, np.float64)
    tol = 1e-5 * np.abs(ora) + 1e-7 * np.abs(ora).max() + allow
    return float((np.abs(np.asarray(gpu, np.float64) - ora) / np.maximum(tol, 1e-300)).max())


def report(name, n_prior=24, n_conv=64, conv=None):
    lens, prior = W.workload(name, oracle.columns_renderer, batch=n_prior)
    mass = W.WORKLOADS[name].mass
    g = tll.Lens(lens.data, lens.noise, lens.psf, lens.pixel_scale, lens.sub, lens.x0, lens.y0,
                 mass=mass)
    label = name
    if conv is not None:
        g.set_conv(conv[1])
        label = f"{name} ({conv[0]})"
    o = oracle.Lens(lens.data, lens.noise, lens.psf, lens.pixel_scale, lens.sub, lens.x0, lens.y0,
                    mass=mass)
    worst = 0.0
    for p in np.concatenate([lens.truth[None], prior[:4]]):
        il, is_ = o.unblurred(p.astype(np.float64))
        _, ml, ms, _, _ = o.model(p.astype(np.float64), mode=1)
        for blurred, refs in ((False, (il, is_)), (True, (ml, ms))):
            cols = g.model_columns(p, blurred=blurred)
            allow = _pix_allowance(o, p, blurred)
            for c, r, a in zip(cols, refs, allow):
                worst = max(worst, pix_ratio(np.asarray(c).reshape(r.shape), r, a))
    rng = np.random.Generator(np.random.PCG64(2024))
    conv = W.shrinking_draws(rng, lens.truth, n_conv, lo_frac=1e-6)
    P = np.concatenate([conv, prior]).astype(np.float32)
    ref = o.loglike_batch(P.astype(np.float64))
    got = g.loglike_batch(torch.from_numpy(P).cuda())
    torch.cuda.synchronize()
    g.conv_check()
    got = got.cpu().numpy()
    _, lognorm, nun = _lens_consts(lens)
    fin = np.isfinite(ref)
    chi2 = -2.0 * (ref - lognorm)
    bulk = fin & (chi2 <= _chi2_truth(lens) + BULK_DCHI2)
    near = fin & ~bulk & (chi2 <= 2 * nun)
    far = fin & ~bulk & ~near
    d = np.abs(got - ref)

    def mx(m):
        return f"{d[m].max():.2e} ({int(m.sum())})" if m.any() else "-"
    pair = "-"
    if bulk.sum() >= 2:
        gb, rb = got[bulk], ref[bulk]
        pair = f"{np.abs((gb[:, None] - gb[None]) - (rb[:, None] - rb[None])).max():.2e}"
    g.close()
    return (f"| {label} | {lens.ny}x{lens.nx}, s={lens.sub}, K={lens.psf.shape[0]} | {worst:.3f} | "
            f"{mx(bulk)} | {pair} | {mx(near)} | {mx(far)} |")


def report_multi(name, n_prior=16, n_conv=48):
    """The same columns for a multi-component workload (every column before
    and after the PSF; light centres at [9], [10] and [13], [14])."""
    lens, prior = W.multi_workload(name, oracle.multi_columns_renderer, batch=n_prior)
    comps = W.MULTI_WORKLOADS[name].comps
    g = tll.Lens(lens.data, lens.noise, lens.psf, lens.pixel_scale, lens.sub, lens.x0, lens.y0)
    g.set_light([tll.comp(c["type"], c["plane"], c.get("free_scale", True),
                          c.get("free_index", False), c.get("scale", 1.0), c.get("index", 1.0))
                 for c in comps])
    o = oracle.MultiLens(lens.data, lens.noise, lens.psf, lens.pixel_scale, lens.sub, comps,
                         lens.x0, lens.y0)

    def cols(p, blurred):
        return o.model(p)[1] if blurred else o.unblurred(p)
    worst = 0.0
    for p in np.concatenate([lens.truth[None], prior[:2]]).astype(np.float64):
        for blurred in (False, True):
            base = cols(p, blurred)
            allow = np.zeros_like(base)
            for sx, sy in ((1, 0), (-1, 0), (0, 1), (0, -1)):
                q = p.copy()
                q[9] += sx * POS_ERR; q[10] += sy * POS_ERR
                q[13] += sx * POS_ERR_SRC; q[14] += sy * POS_ERR_SRC
                allow = np.maximum(allow, np.abs(cols(q, blurred) - base))
            gc = g.model_columns_n(p.astype(np.float32), blurred=blurred)
            for c in range(len(comps)):
                worst = max(worst, pix_ratio(gc[c], base[c], allow[c]))
    rng = np.random.Generator(np.random.PCG64(2025))
    conv = W.shrinking_draws_multi(rng, lens.truth, n_conv, comps, lo_frac=1e-6)
    P = np.concatenate([conv, prior]).astype(np.float32)
    ref = o.loglike_batch(P.astype(np.float64))
    got = g.loglike_batch(torch.from_numpy(P).cuda())
    torch.cuda.synchronize()
    got = got.cpu().numpy()
    _, lognorm, nun = _lens_consts(lens)
    fin = np.isfinite(ref)
    chi2 = -2.0 * (ref - lognorm)
    chi2_t = -2.0 * (o.loglike(lens.truth) - lognorm)
    bulk = fin & (chi2 <= chi2_t + BULK_DCHI2)
    near = fin & ~bulk & (chi2 <= 2 * nun)
    far = fin & ~bulk & ~near
    d = np.abs(got - ref)

    def mx(m):
        return f"{d[m].max():.2e} ({int(m.sum())})" if m.any() else "-"
    pair = "-"
    if bulk.sum() >= 2:
        gb, rb = got[bulk], ref[bulk]
        pair = f"{np.abs((gb[:, None] - gb[None]) - (rb[:, None] - rb[None])).max():.2e}"
    g.close()
    return (f"| {name} ({len(comps)} columns, FNNLS) | {lens.ny}x{lens.nx}, s={lens.sub}, "
            f"K={lens.psf.shape[0]} | {worst:.3f} | {mx(bulk)} | {pair} | {mx(near)} | "
            f"{mx(far)} |")


def main():
    build.build()
    tll.load()
    print("| workload | image | worst pixel error / gate | bulk max abs dlogL (n) | "
          "bulk pairwise d(dlogL) | near max (n) | prior max (n) |")
    print("|---|---|---|---|---|---|---|")
    for name in ("plain64", "csst100", "hst200", "csst100_epl", "csst100_mask"):
        print(report(name), flush=True)
    for name in ("slacs120", "mge120", "mge32"):
        print(report_multi(name), flush=True)
    # the hst200 convolution (Eq. 3) run three ways
    for conv in (("split, direct FP32", tll.CONV_SPLIT_DIRECT),
                 ("split, Toeplitz 3xTF32 tensor cores", tll.CONV_SPLIT_TOEPLITZ_TC)):
        print(report("hst200", conv=conv), flush=True)


if __name__ == "__main__":
    main()
