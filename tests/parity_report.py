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
multi-component workloads report every column; the ragged and served rows
are a few lenses of those recipes through the batcher and the server (log L
only: their columns are the one-lens kernels').  Inputs are the seeded synthetic workloads; nothing is
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


def _regions(got, ref, which, lenses, chi2_truths):
    """max |dlogL| (count) per region over several lenses: got and ref are
    concatenated, which[i] is the index of entry i's lens in lenses, and
    chi2_truths[k] is lens k's chi^2 at its true parameters."""
    got, ref = np.asarray(got), np.asarray(ref)
    fin = np.isfinite(ref)
    bulk = np.zeros(len(ref), bool)
    near = np.zeros(len(ref), bool)
    pair = 0.0
    for k, lens in enumerate(lenses):
        m = which == k
        _, lognorm, nun = _lens_consts(lens)
        chi2 = -2.0 * (ref[m] - lognorm)
        b = fin[m] & (chi2 <= chi2_truths[k] + BULK_DCHI2)
        bulk[m] = b
        near[m] = fin[m] & ~b & (chi2 <= 2 * nun)
        if b.sum() >= 2:
            gb, rb = got[m][b], ref[m][b]
            pair = max(pair, float(np.abs((gb[:, None] - gb[None])
                                          - (rb[:, None] - rb[None])).max()))
    far = fin & ~bulk & ~near
    d = np.abs(got - ref)

    def mx(m):
        return f"{d[m].max():.2e} ({int(m.sum())})" if m.any() else "-"
    return mx(bulk), f"{pair:.2e}", mx(near), mx(far)


def _against_oracle(items, outs):
    """Concatenated GPU and oracle log L of (lens, params) items, the lens
    index of each entry and each lens's chi^2 at its truth."""
    got, ref, which, chi2_t = [], [], [], []
    for k, ((sl, P), out) in enumerate(zip(items, outs)):
        o = oracle.Lens(sl.data, sl.noise, sl.psf, sl.pixel_scale, sl.sub, sl.x0, sl.y0)
        got.append(np.asarray(out))
        ref.append(o.loglike_batch(np.asarray(P, np.float64)))
        which.append(np.full(len(P), k))
        _, lognorm, _ = _lens_consts(sl)
        chi2_t.append(-2.0 * (o.loglike(sl.truth) - lognorm))
    return np.concatenate(got), np.concatenate(ref), np.concatenate(which), chi2_t


def report_ragged(n_lenses=6, per_lens=48):
    """A few lenses of the ragged recipe (sides 64..200, PSF 11..31, 4 x 4
    subpixels, vectors shrinking around each truth) in one multi-lens
    launch replayed as a CUDA graph (tll_batcher), against the oracle."""
    items = W.ragged_workload(n_lenses, per_lens, oracle.columns_renderer, seed_offset=40)
    lenses = [tll.Lens(sl.data, sl.noise, sl.psf, sl.pixel_scale, sl.sub, sl.x0, sl.y0,
                       batch_only=True) for sl, _ in items]
    params = [torch.from_numpy(np.ascontiguousarray(P, np.float32)).cuda() for _, P in items]
    b = tll.Batcher(use_graph=True)
    b.run(lenses, params)            # the capture; the second run replays it
    outs = b.run(lenses, params)
    torch.cuda.synchronize()
    outs = [o.cpu().numpy() for o in outs]
    b.close()
    for L in lenses:
        L.close()
    got, ref, which, chi2_t = _against_oracle(items, outs)
    cols = _regions(got, ref, which, [sl for sl, _ in items], chi2_t)
    sides = sorted({sl.ny for sl, _ in items})
    ks = sorted({sl.psf.shape[0] for sl, _ in items})
    return (f"| ragged ({n_lenses} lenses, one graph-replayed multi-lens launch) | sides "
            f"{sides}, s=4, K {ks} | - | " + " | ".join(cols) + " |")


def report_served(n_jobs=4, per_job=48):
    """Jobs of the request-stream recipe (sides 64..200, PSF 11..31) through
    the server (tll_server: host buffers, their requests coalesced per
    launch), against the oracle."""
    jobs = W.request_stream(n_jobs, iters=1, seed_offset=50)
    rng = np.random.Generator(np.random.PCG64(W.SEED_BASE + 51))
    items = []
    for jd in jobs:
        psf = W.gaussian_psf(jd["psf"], jd["psf"] / 7.0)
        render = oracle.columns_renderer(W.f32(0.074), 4, psf, jd["side"], jd["side"])
        sl = W.synth_lens(rng, jd["side"], jd["side"], 0.074, 4, psf, render, "sky+poisson")
        items.append((sl, W.shrinking_draws(rng, sl.truth, per_job).astype(np.float32)))
    S = tll.Server(max_jobs=2 * n_jobs)
    ids = [S.open_job(sl.data, sl.noise, sl.psf, sl.pixel_scale, sl.sub, sl.x0, sl.y0)
           for sl, _ in items]
    reqs = [S.submit(j, P) for j, (_, P) in zip(ids, items)]
    outs = [S.wait(r)[0] for r in reqs]
    for j in ids:
        S.close_job(j)
    S.close()
    got, ref, which, chi2_t = _against_oracle(items, outs)
    cols = _regions(got, ref, which, [sl for sl, _ in items], chi2_t)
    sides = sorted({sl.ny for sl, _ in items})
    ks = sorted({sl.psf.shape[0] for sl, _ in items})
    return (f"| served ({n_jobs} jobs through tll_server, host buffers) | sides {sides}, "
            f"s=4, K {ks} | - | " + " | ".join(cols) + " |")


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
    print(report_ragged(), flush=True)
    print(report_served(), flush=True)
    # the hst200 convolution (Eq. 3) run three ways
    for conv in (("split, direct FP32", tll.CONV_SPLIT_DIRECT),
                 ("split, Toeplitz 3xTF32 tensor cores", tll.CONV_SPLIT_TOEPLITZ_TC),
                 ("split, Toeplitz split-BF16 tensor cores", tll.CONV_SPLIT_TOEPLITZ_BF16)):
        print(report("hst200", conv=conv), flush=True)


if __name__ == "__main__":
    main()
