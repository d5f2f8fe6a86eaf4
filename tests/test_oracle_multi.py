"""Pins for the oracle's multi-component light model and its N-column FNNLS
(arXiv:2503.08586 Sec. 2.3, Eq. 7 and the non-negative penalty after it;
Sec. 3.2's double Sersic; Sec. 4.3's Gaussian expansion), against library
routines, brute force, closed forms and the pinned two-column oracle --
never the oracle's own formulas retyped.  CPU only."""
import itertools
import math

import numpy as np
import pytest
from scipy import optimize

import oracle

rng0 = np.random.default_rng(20250311)


# ------------------------------------------------------------- FNNLS
def _random_problem(r, n, m=40, collinear=False):
    Z = r.normal(size=(m, n))
    if collinear and n >= 2:
        Z[:, 1] = Z[:, 0] * 1.7 + 1e-6 * r.normal(size=m)
    y = r.normal(size=m) + Z @ r.uniform(-1.0, 1.0, n)
    return Z, y


def _brute_force(Z, y):
    """Global NNLS optimum by enumerating every face: the unconstrained
    least-squares minimiser on each subset of free columns, kept when all of
    its entries are positive; the smallest residual wins."""
    n = Z.shape[1]
    best, bestx = float(y @ y), np.zeros(n)
    for k in range(1, n + 1):
        for S in itertools.combinations(range(n), k):
            S = list(S)
            zs, *_ = np.linalg.lstsq(Z[:, S], y, rcond=None)
            if np.all(zs > 0):
                x = np.zeros(n)
                x[S] = zs
                r = y - Z @ x
                if r @ r < best - 1e-12:
                    best, bestx = float(r @ r), x
    return bestx, best


@pytest.mark.parametrize("n", [1, 2, 3, 4, 5, 6, 8])
def test_fnnls_vs_brute_force(n):
    r = np.random.default_rng(100 + n)
    for _ in range(40):
        Z, y = _random_problem(r, n)
        x, steps = oracle.fnnls(Z.T @ Z, Z.T @ y)
        assert steps >= 0
        xb, rb = _brute_force(Z, y)
        res = y - Z @ x
        assert abs(res @ res - rb) <= 1e-9 * max(rb, 1.0)
        assert np.max(np.abs(x - xb)) <= 1e-7 * max(1.0, np.max(np.abs(xb)))


@pytest.mark.parametrize("n", [2, 4, 8, 12, 16, 32, 48])
def test_fnnls_vs_library_nnls_and_kkt(n):
    """scipy.optimize.nnls (Lawson-Hanson on Z itself) gives the same
    optimum; the KKT conditions hold: x >= 0, gradient b - A x <= 0 on the
    zero set and = 0 on the support."""
    r = np.random.default_rng(200 + n)
    for _ in range(30):
        Z, y = _random_problem(r, n, m=3 * n + 10)
        A, b = Z.T @ Z, Z.T @ y
        x, steps = oracle.fnnls(A, b)
        assert steps >= 0
        xs, _ = optimize.nnls(Z, y)
        assert np.max(np.abs(x - xs)) <= 1e-8 * max(1.0, np.max(np.abs(xs)))
        g = b - A @ x
        scale = np.max(np.abs(A)) * max(1.0, np.max(np.abs(x)))
        assert np.all(x >= 0)
        assert np.all(g[x == 0] <= 1e-10 * scale)
        assert np.all(np.abs(g[x > 0]) <= 1e-10 * scale)


def test_fnnls_special_cases():
    """b <= 0 gives x = 0; a diagonal A gives x = max(b / diag, 0); an
    unconstrained optimum that is already positive is returned unchanged."""
    r = np.random.default_rng(3)
    A = np.diag(r.uniform(0.5, 3.0, 6))
    x, _ = oracle.fnnls(A, -r.uniform(0.1, 1.0, 6))
    assert np.all(x == 0)
    b = r.normal(size=6)
    x, _ = oracle.fnnls(A, b)
    assert np.allclose(x, np.maximum(b / np.diag(A), 0), rtol=1e-14, atol=0)
    Z = r.normal(size=(30, 5))
    xt = r.uniform(0.5, 2.0, 5)
    x, _ = oracle.fnnls(Z.T @ Z, Z.T @ (Z @ xt))
    assert np.max(np.abs(x - xt)) < 1e-10


def test_fnnls_nearly_collinear_columns():
    """Two columns equal to 1e-6: the residual still matches brute force
    (the optimum may sit on either face)."""
    r = np.random.default_rng(4)
    for _ in range(30):
        Z, y = _random_problem(r, 4, collinear=True)
        x, steps = oracle.fnnls(Z.T @ Z, Z.T @ y)
        _, rb = _brute_force(Z, y)
        res = y - Z @ x
        assert np.all(x >= 0)
        assert abs(res @ res - rb) <= 1e-7 * max(rb, 1.0)


def test_cholesky_solve_vs_library():
    r = np.random.default_rng(5)
    for k in (1, 2, 5, 9, 16):
        Z = r.normal(size=(k + 5, k))
        G = Z.T @ Z
        rhs = r.normal(size=k)
        z = oracle.chol_solve(G, rhs)
        assert np.allclose(z, np.linalg.solve(G, rhs), rtol=1e-10, atol=1e-12)
    assert oracle.chol_solve(np.array([[1.0, 2.0], [2.0, 1.0]]), np.ones(2)) is None


# ------------------------------------------------- component profiles
def test_gaussian_is_half_sersic_one_half():
    """R13 against Eq. (8): a Sersic of index 1/2 has b = ln 2 exactly
    (P(1, b) = 1 - e^{-b}), so I = 2 exp(-ln2 R^2/r_e^2): the unit Gaussian of
    sigma = r_e / sqrt(2 ln 2) is half of it everywhere."""
    r = np.random.default_rng(6)
    for _ in range(200):
        re = r.uniform(0.05, 2.0)
        q, phi = r.uniform(0.2, 1.0), r.uniform(-3, 3)
        cx, cy, x, y = r.normal(0, 0.5, 4)
        sig = re / math.sqrt(2 * math.log(2))
        if oracle.sersic(x, y, cx, cy, q, phi, re, 0.5, math.log(2)) == 0.0:
            continue
        g = oracle.gauss(x, y, cx, cy, q, phi, sig)
        s = oracle.sersic(x, y, cx, cy, q, phi, re, 0.5, math.log(2))
        # exp's rounding grows with its argument: |d ln I| <= few eps |ln I|
        assert abs(g - 0.5 * s) <= 1e-15 * (8 + abs(math.log(s))) * s


def _comps_slacs():
    """Sec. 3.2's SLACS model: two Sersics per galaxy, indices fixed at 1
    and 4, free effective radii, shared centre and ellipticity per plane."""
    return [dict(type="sersic", plane="lens", index=1.0),
            dict(type="sersic", plane="lens", index=4.0),
            dict(type="sersic", plane="source", index=1.0),
            dict(type="sersic", plane="source", index=4.0)]


def _mvec(r_es, **kw):
    head = dict(theta_E=1.1, eps1_m=0.1, eps2_m=-0.05, x_m=0.02, y_m=-0.03,
                gamma_1=0.03, gamma_2=-0.02, eps1_L=0.08, eps2_L=0.02, x_L=0.02,
                y_L=-0.03, eps1_S=-0.1, eps2_S=0.15, x_S=0.1, y_S=-0.05)
    head.update(kw)
    names = ["theta_E", "eps1_m", "eps2_m", "x_m", "y_m", "gamma_1", "gamma_2",
             "eps1_L", "eps2_L", "x_L", "y_L", "eps1_S", "eps2_S", "x_S", "y_S"]
    return np.array([head[k] for k in names] + list(r_es), dtype=np.float64)


def test_gaussian_flux_on_grid():
    """A lens-plane Gaussian column, finely supersampled, sums (x pixel area)
    to 2 pi sigma^2 for any axis ratio (the Eq. 10 radius keeps the area of
    an isophote at pi R^2)."""
    comps = [dict(type="gauss", plane="lens"), dict(type="gauss", plane="source")]
    dpix, npx, sub = 0.05, 140, 3
    lens = oracle.MultiLens(np.zeros((npx, npx)), np.ones((npx, npx)),
                            np.ones((1, 1)), dpix, sub, comps)
    sig = 0.35
    p = _mvec([sig, 0.2], eps1_L=0.25, eps2_L=-0.1, x_L=0.11, y_L=-0.04)
    cols = lens.unblurred(p)
    assert abs(cols[0].sum() * dpix ** 2 - 2 * math.pi * sig ** 2) < 1e-7 * 2 * math.pi * sig ** 2


def test_two_component_model_is_the_pinned_two_column_oracle():
    """One free-index Sersic per plane is the paper's Table-1 model: the
    multi-component oracle must give the pinned two-column oracle's log L,
    columns and amplitudes when the parameter slots are mapped across."""
    comps = [dict(type="sersic", plane="lens", free_index=True),
             dict(type="sersic", plane="source", free_index=True)]
    r = np.random.default_rng(9)
    ny = nx = 24
    psf = np.exp(-0.5 * (np.arange(7) - 3.0) ** 2)[None, :] * np.exp(
        -0.5 * (np.arange(7) - 3.0) ** 2 / 1.5)[:, None]
    data = r.normal(size=(ny, nx)) + 3.0
    noise = r.uniform(0.5, 1.5, (ny, nx))
    two = oracle.Lens(data, noise, psf, 0.08, 3)
    multi = oracle.MultiLens(data, noise, psf, 0.08, 3, comps)
    assert multi.nparam == 19
    for _ in range(6):
        v = np.array([r.uniform(0.5, 1.5), *r.uniform(-0.2, 0.2, 2), *r.normal(0, 0.05, 2),
                      *r.normal(0, 0.05, 2), 1.0, r.uniform(0.2, 1.0), r.uniform(1, 4),
                      *r.uniform(-0.2, 0.2, 2), *r.normal(0, 0.05, 2), 1.0,
                      r.uniform(0.1, 0.8), r.uniform(1, 4), *r.uniform(-0.2, 0.2, 2),
                      *r.normal(0, 0.2, 2)])
        m = np.concatenate([v[0:7], v[10:14], v[17:21], [v[8], v[9], v[15], v[16]]])
        ll2, ml, ms, mod2, amps2 = two.model(v)
        llm, cols, modm, ampsm = multi.model(m)
        assert abs(llm - ll2) <= 1e-9 * abs(ll2)
        assert np.allclose(cols[0], ml, rtol=1e-13, atol=1e-300)
        assert np.allclose(cols[1], ms, rtol=1e-13, atol=1e-300)
        assert np.allclose(ampsm, amps2, rtol=1e-8, atol=1e-12)


def test_source_component_without_deflection_equals_lens_component():
    """theta_E = 0 and no shear make beta = theta (Eq. 1): a source-plane
    component with the lens-plane geometry equals the lens-plane one."""
    comps = [dict(type="sersic", plane="lens", index=2.5),
             dict(type="sersic", plane="source", index=2.5),
             dict(type="gauss", plane="lens"), dict(type="gauss", plane="source")]
    lens = oracle.MultiLens(np.zeros((20, 20)), np.ones((20, 20)), np.ones((1, 1)),
                            0.07, 2, comps)
    g = dict(eps1_L=0.12, eps2_L=-0.07, x_L=0.05, y_L=0.02)
    p = _mvec([0.3, 0.3, 0.2, 0.2], theta_E=0.0, gamma_1=0.0, gamma_2=0.0,
              eps1_S=g["eps1_L"], eps2_S=g["eps2_L"], x_S=g["x_L"], y_S=g["y_L"], **g)
    c = lens.unblurred(p)
    assert np.array_equal(c[0], c[1]) and np.array_equal(c[2], c[3])


def test_fixed_and_free_slots_agree():
    """A component's fixed value (from the list) and the same value read
    from its free slot give the same column; slots follow component order."""
    free = [dict(type="sersic", plane="lens", index=1.0),
            dict(type="gauss", plane="source"),
            dict(type="sersic", plane="source", free_index=True)]
    fixed = [dict(type="sersic", plane="lens", index=1.0, free_scale=False, scale=0.45),
             dict(type="gauss", plane="source", free_scale=False, scale=0.12),
             dict(type="sersic", plane="source", free_scale=False, scale=0.2,
                  free_index=False, index=3.3)]
    args = (np.zeros((16, 16)), np.ones((16, 16)), np.ones((3, 3)), 0.1, 2)
    a = oracle.MultiLens(*args, free)
    b = oracle.MultiLens(*args, fixed)
    assert a.nparam == 15 + 4 and b.nparam == 15
    ca = a.unblurred(_mvec([0.45, 0.12, 0.2, 3.3]))
    cb = b.unblurred(_mvec([]))
    assert np.array_equal(ca, cb)


def test_exact_multi_model_recovers_amplitudes():
    """Noiseless data built from the columns with known amplitudes (one of
    them zero): FNNLS recovers them and log L = -sum log(2 pi sigma^2)/2
    (chi^2 = 0 when m = d, Eq. 5)."""
    comps = _comps_slacs()
    ny = nx = 30
    psf = np.exp(-0.5 * ((np.arange(9) - 4.0)[:, None] ** 2 + (np.arange(9) - 4.0)[None, :] ** 2) / 2.0)
    render = oracle.multi_columns_renderer(0.06, 3, psf, ny, nx, comps)
    p = _mvec([0.5, 0.9, 0.12, 0.3])
    cols = render(p)
    s_true = np.array([3.0, 0.0, 7.0, 2.0])
    data = np.tensordot(s_true, cols, axes=1)
    sigma = np.full((ny, nx), 0.7)
    lens = oracle.MultiLens(data, sigma, psf, 0.06, 3, comps)
    ll, _, mod, amps = lens.model(p)
    assert np.max(np.abs(amps - s_true)) < 1e-7 * s_true.max()
    C = -0.5 * ny * nx * math.log(2 * math.pi * 0.49)
    assert abs(ll - C) < 1e-9 * abs(C)



def test_multi_masked_pixels_leave_the_fit():
    """Masked pixels (sigma <= 0, non-finite sigma or data) drop out of Eq. 5
    and of the N-column FNNLS: with noisy data, the oracle equals a library
    NNLS fit (scipy) of its blurred columns to the unmasked pixels alone.
    The masked pixels hold +-1e6 or NaN, so a leak would show at once."""
    r = np.random.default_rng(32)
    comps = _comps_slacs()
    ny, nx = 26, 24
    psf = np.exp(-0.5 * ((np.arange(7) - 3.0)[:, None] ** 2 + (np.arange(7) - 3.0)[None, :] ** 2) / 1.8)
    p = _mvec([0.5, 0.9, 0.12, 0.3])
    cols = oracle.multi_columns_renderer(0.06, 3, psf, ny, nx, comps)(p)
    sig = r.uniform(0.4, 1.6, (ny, nx))
    d = np.tensordot(np.array([3.0, 1.0, 7.0, 2.0]), cols, axes=1) + r.normal(0.0, 1.0, (ny, nx)) * sig
    for (i, j), (sv, dv) in zip([(0, 0), (3, 7), (ny // 2, nx // 2), (ny - 1, nx - 1), (5, 5)],
                                [(0.0, 1e6), (-2.0, -1e6), (np.inf, 5e5), (np.nan, 1e6),
                                 (1.0, np.nan)]):
        sig[i, j], d[i, j] = sv, dv
    ok = np.isfinite(sig) & (sig > 0) & np.isfinite(d)
    assert ok.sum() == ny * nx - 5
    w = 1.0 / sig[ok]
    A = np.stack([c[ok] * w for c in cols], axis=1)
    x_ref, rnorm = optimize.nnls(A, d[ok] * w)
    ll_ref = -0.5 * rnorm ** 2 - 0.5 * np.sum(np.log(2 * math.pi * sig[ok] ** 2))
    ll, _, _, amps = oracle.MultiLens(d, sig, psf, 0.06, 3, comps).model(p)
    assert abs(ll - ll_ref) <= 1e-9 * abs(ll_ref)
    assert np.allclose(amps, x_ref, rtol=1e-7, atol=1e-9 * x_ref.max())


def test_zero_column_and_component_order():
    """Structure of the amplitude fit (Eq. 7 with the non-negative
    penalty): a component whose column is identically zero (a fixed
    Gaussian of width 1e-6 arcsec off every subpixel centre) gets amplitude
    0 and leaves log L and the other amplitudes exactly as without it,
    wherever it sits in the list; reordering the components permutes the
    amplitudes and leaves log L unchanged up to rounding."""
    r = np.random.default_rng(33)
    ny, nx = 24, 22
    psf = np.exp(-0.5 * ((np.arange(5) - 2.0)[:, None] ** 2 + (np.arange(5) - 2.0)[None, :] ** 2) / 1.2)
    base = _comps_slacs()
    p = _mvec([0.5, 0.9, 0.12, 0.3], x_L=0.0123, y_L=-0.0171)
    cols = oracle.multi_columns_renderer(0.06, 3, psf, ny, nx, base)(p)
    sig = r.uniform(0.5, 1.5, (ny, nx))
    d = np.tensordot(np.array([3.0, 1.0, 7.0, 2.0]), cols, axes=1) + r.normal(0, 1, (ny, nx)) * sig
    ll0, _, _, a0 = oracle.MultiLens(d, sig, psf, 0.06, 3, base).model(p)
    assert np.all(a0 > 0)
    tiny = dict(type="gauss", plane="lens", free_scale=False, scale=1e-6)
    for pos in (0, 2, 4):
        comps = base[:pos] + [tiny] + base[pos:]
        ll1, c1, _, a1 = oracle.MultiLens(d, sig, psf, 0.06, 3, comps).model(p)
        assert not np.any(c1[pos])
        assert ll1 == ll0
        assert a1[pos] == 0.0 and np.array_equal(np.delete(a1, pos), a0)
    # the free radii follow their components: slots 15..18 are the four
    # components' r_e in list order
    perm = [2, 0, 3, 1]
    q = np.concatenate([p[:15], p[15:][perm]])
    llp, _, _, ap = oracle.MultiLens(d, sig, psf, 0.06, 3, [base[k] for k in perm]).model(q)
    assert abs(llp - ll0) <= 1e-10 * abs(ll0)
    assert np.allclose(ap, a0[perm], rtol=1e-9)

def test_multi_invalid_vectors():
    comps = _comps_slacs() + [dict(type="sersic", plane="lens", free_index=True)]
    lens = oracle.MultiLens(np.zeros((8, 8)), np.ones((8, 8)), np.ones((1, 1)), 0.1, 1, comps)
    good = _mvec([0.5, 0.9, 0.12, 0.3, 0.4, 2.0])
    assert np.isfinite(lens.loglike(good))
    for k, v in ((15, 0.0), (16, -1.0), (20, 0.1), (20, 10.5), (0, -0.1),
                 (7, 0.9), (11, 1.2), (3, np.nan)):
        bad = good.copy()
        if k == 7:
            bad[7], bad[8] = 0.8, 0.7
        else:
            bad[k] = v
        assert lens.loglike(bad) == -np.inf, k


def test_multi_batch_equals_single():
    comps = _comps_slacs()
    r = np.random.default_rng(10)
    lens = oracle.MultiLens(r.normal(size=(12, 12)), np.ones((12, 12)), np.ones((3, 3)),
                            0.1, 2, comps)
    P = np.stack([_mvec(r.uniform(0.1, 1.0, 4), theta_E=r.uniform(0.5, 1.5)) for _ in range(5)])
    out = lens.loglike_batch(P, nthreads=2)
    assert np.array_equal(out, np.array([lens.loglike(p) for p in P]))
