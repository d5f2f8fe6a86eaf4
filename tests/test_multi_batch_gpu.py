"""Multi-component lenses in the multi-lens launches: the batcher (their own
k_loglike_nc_multi groups beside the two-column groups, with and without
CUDA-graph replay) and the server (tll_server_set_light).  Each result must
equal the lens's own one-lens evaluation bit for bit (the same arithmetic)
and pass the parity gates against the FP64 oracle."""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
from paper_2503_08586_gb300 import build, tll
from paper_2503_08586_gb300 import workloads as W

from test_multi_light_gpu import CASES, _case, _to_tll
from test_parity_gpu import _CHI2_TRUTH, _lens_consts, _ll_ok

pytestmark = pytest.mark.gpu

PICK = (0, 3, 4, 5)   # SLACS direct, 8 Gaussians on the generic convolution, SLACS + EPL, 32 Gaussians


@pytest.fixture(scope="module")
def setups():
    build.build()
    tll.load()
    assert torch.cuda.is_available()
    out = []
    for idx in PICK:
        sl, P, o, ref = _case(idx, *CASES[idx])
        out.append((idx, sl, P, ref))
    # a masked multi-component lens
    idx = 1
    sl, P, o, ref = _case(idx, *CASES[idx])
    W.apply_mask(sl, W.annulus_mask(sl.ny, sl.nx, sl.pixel_scale, 0.2, 1.0, sl.x0, sl.y0))
    om = oracle.MultiLens(sl.data, sl.noise, sl.psf, sl.pixel_scale, sl.sub, CASES[idx][7],
                          sl.x0, sl.y0)
    refm = om.loglike_batch(P.astype(np.float64))
    _, lognorm, _ = _lens_consts(sl)
    _CHI2_TRUTH[id(sl)] = (sl, max(-2.0 * (refm[0] - lognorm), 0.0))   # P[0] is the truth
    out.append((idx, sl, P, refm))
    # a two-column lens in the same launches
    rng = np.random.Generator(np.random.PCG64(8100))
    psf = W.gaussian_psf(9, 1.8)
    s2 = W.synth_lens(rng, 44, 40, 0.05, 4, psf, oracle.columns_renderer(0.05, 4, psf, 44, 40))
    P2 = W.shrinking_draws(rng, s2.truth, 40, lo_frac=1e-6)
    r2 = oracle.Lens(s2.data, s2.noise, s2.psf, s2.pixel_scale, s2.sub, s2.x0,
                     s2.y0).loglike_batch(P2.astype(np.float64))
    out.append((None, s2, P2, r2))
    return out


def _lens(idx, sl, batch_only):
    mass = CASES[idx][8] if idx is not None else "sie"
    g = tll.Lens(sl.data, sl.noise, sl.psf, sl.pixel_scale, sl.sub, sl.x0, sl.y0, mass=mass,
                 batch_only=batch_only)
    if idx is not None:
        g.set_light(_to_tll(CASES[idx][7]))
    return g


def test_batcher_mixes_multi_and_two_column_lenses(setups):
    lenses = [_lens(idx, sl, True) for idx, sl, _, _ in setups]
    params = [torch.from_numpy(np.ascontiguousarray(P)).cuda() for _, _, P, _ in setups]
    alone = []
    for (idx, sl, P, _), p in zip(setups, params):
        g = _lens(idx, sl, False)
        out = g.loglike_batch(p)
        torch.cuda.synchronize()
        alone.append(out.cpu().numpy())
        g.close()
    for graph in (False, True):
        b = tll.Batcher(use_graph=graph)
        st = torch.cuda.Stream()
        for _ in range(2):   # the second run replays the graph
            with torch.cuda.stream(st):
                outs = b.run(lenses, params, stream=st)
                st.synchronize()
            for out, a, (idx, sl, P, ref) in zip(outs, alone, setups):
                got = out.cpu().numpy()
                assert np.array_equal(got, a), f"lens {idx}: batcher differs from one-lens"
                _ll_ok(got, ref, sl)
        b.close()
    for L in lenses:
        L.close()


def test_server_serves_multi_component_jobs(setups):
    S = tll.Server(max_jobs=8)
    jobs = []
    for idx, sl, P, ref in setups[:2] + setups[-1:]:
        mass = CASES[idx][8] if idx is not None else "sie"
        j = S.open_job(sl.data, sl.noise, sl.psf, sl.pixel_scale, sl.sub, sl.x0, sl.y0, mass=mass)
        if idx is not None:
            S.set_light(j, _to_tll(CASES[idx][7]))
        jobs.append((j, P, ref, sl))
    reqs = [(S.submit(j, P), ref, sl) for j, P, ref, sl in jobs]
    for r, ref, sl in reqs:
        _ll_ok(S.wait(r)[0], ref, sl)
    for j, _, _, _ in jobs:
        assert S.close_job(j)
    S.close()


def test_batch_only_multi_lens_defers_its_slots(setups):
    idx, sl, P, ref = setups[0]
    g = _lens(idx, sl, True)
    lib = tll.load()
    n = ctypes.c_size_t()
    assert lib.tll_lens_footprint(g.handle, ctypes.byref(n)) == tll.OK
    before = n.value
    p = torch.from_numpy(np.ascontiguousarray(P)).cuda()
    out = torch.empty(P.shape[0], dtype=torch.float64, device="cuda")
    with pytest.raises(tll.TLLError):       # no one-lens slots yet, and no allocation here
        g.loglike_batch_noalloc(p, out)
    a = g.loglike_batch(p)                   # allocates them
    torch.cuda.synchronize()
    assert lib.tll_lens_footprint(g.handle, ctypes.byref(n)) == tll.OK
    g_bytes = n.value
    assert g_bytes > before
    g.loglike_batch_noalloc(p, out)
    torch.cuda.synchronize()
    assert torch.equal(a, out)
    g.close()


def test_multi_column_lens_slots_split_and_update():
    """Seven multi-component lenses of one shape class (the SLACS direct
    case's geometry, each with its own data): a launch group holds at most
    five lens slots (their descriptors and component lists in the launch
    parameters), so the sixth starts a second group; one lens appears in two
    non-adjacent entries.  Later runs keep the group launches (graph updated
    in place) or drop one (graph instantiated again); every result must equal
    the lens's own one-lens evaluation bit for bit."""
    build.build()
    tll.load()
    name, ny, nx, dpix, sub, ks, kind, comps, mass = CASES[0]
    psf = W.moffat_psf(ks, 2.2, 3.0)
    render = oracle.multi_columns_renderer(W.f32(dpix), sub, psf, ny, nx, comps, mass=mass)
    items = []
    for k in range(7):
        rng = np.random.Generator(np.random.PCG64(9100 + k))
        sl = W.synth_multi_lens(rng, ny, nx, dpix, sub, psf, render, comps, mass=mass)
        P = np.concatenate([sl.truth[None],
                            W.shrinking_draws_multi(rng, sl.truth, 9 + 6 * k, comps,
                                                    lo_frac=1e-6)]).astype(np.float32)
        g = tll.Lens(sl.data, sl.noise, sl.psf, sl.pixel_scale, sl.sub, sl.x0, sl.y0,
                     mass=mass)
        g.set_light(_to_tll(comps))
        items.append((g, P))
    alone = {}
    b = tll.Batcher(use_graph=True)
    st = torch.cuda.Stream()
    runs = [list(range(7)) + [3], [6, 5, 4, 3, 1, 0, 2, 5], [6, 2, 4]]
    for sel in runs:
        parts = []
        for j, k in enumerate(sel):
            P = items[k][1]
            h = len(P) // 2
            parts.append((k, P[:h] if sel.count(k) > 1 and j == sel.index(k) else
                          P[h:] if sel.count(k) > 1 else P))
        params = [torch.from_numpy(np.ascontiguousarray(p)).cuda() for _, p in parts]
        for (k, p), t in zip(parts, params):
            key = (k, p.shape[0], float(p[0, 0]))
            if key not in alone:
                out = items[k][0].loglike_batch(t)
                torch.cuda.synchronize()
                alone[key] = out.cpu().numpy()
        torch.cuda.synchronize()
        with torch.cuda.stream(st):
            outs = b.run([items[k][0] for k, _ in parts], params, stream=st)
        st.synchronize()
        for (k, p), o in zip(parts, outs):
            got = o.cpu().numpy()
            assert np.array_equal(got, alone[(k, p.shape[0], float(p[0, 0]))]), (sel, k)
    b.close()
    for g, _ in items:
        g.close()
