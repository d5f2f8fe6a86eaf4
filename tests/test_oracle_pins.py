"""Pins for the FP64 oracle: closed forms, library routines, brute force and
independent quadratures -- never the oracle's own formulas retyped.

Each test names the part of arXiv:2503.08586 it pins (section / equation).
All run on the CPU (not marked gpu).
"""
import math

import numpy as np
import pytest
from scipy import integrate, optimize, signal, special

import oracle
from paper_2503_08586_gb300 import workloads as W

rng_global = np.random.default_rng(12345)


def _vec(**kw):
    """A valid parameter vector with overrides (names as in the layout)."""
    names = ["theta_E", "eps1_m", "eps2_m", "x_m", "y_m", "gamma_1", "gamma_2",
             "Ie_L", "re_L", "n_L", "eps1_L", "eps2_L", "x_L", "y_L",
             "Ie_S", "re_S", "n_S", "eps1_S", "eps2_S", "x_S", "y_S"]
    base = dict(theta_E=1.0, eps1_m=0.0, eps2_m=0.0, x_m=0.0, y_m=0.0,
                gamma_1=0.0, gamma_2=0.0, Ie_L=1.0, re_L=0.5, n_L=2.0,
                eps1_L=0.0, eps2_L=0.0, x_L=0.0, y_L=0.0, Ie_S=1.0, re_S=0.2,
                n_S=1.0, eps1_S=0.0, eps2_S=0.0, x_S=0.0, y_S=0.0)
    base.update(kw)
    return np.array([base[k] for k in names], dtype=np.float64)


# ------------------------------------------------------------ Eq. (11)
def test_ellipse_special_values():
    """Eq. (11): eps = 0 is round; eps = ((1-q)/(1+q), 0) has angle 0; the
    second component alone gives angle pi/4; |eps| >= 1 is no ellipse."""
    q, phi = oracle.ellipse(0.0, 0.0)
    assert q == 1.0 and phi == 0.0
    q, phi = oracle.ellipse(1.0 / 3.0, 0.0)
    assert abs(q - 0.5) < 1e-15 and abs(phi) < 1e-15
    q, phi = oracle.ellipse(0.0, 1.0 / 3.0)
    assert abs(q - 0.5) < 1e-15 and abs(phi - math.pi / 4) < 1e-15
    q, phi = oracle.ellipse(-0.2, 0.0)
    assert abs(abs(phi) - math.pi / 2) < 1e-15
    assert oracle.ellipse(1.0, 0.0) is None
    assert oracle.ellipse(0.8, 0.7) is None


def test_ellipse_roundtrip():
    """(q, theta) -> Eq. (11) -> oracle -> (q, theta mod pi)."""
    r = np.random.default_rng(1)
    for _ in range(200):
        q0 = r.uniform(0.05, 1.0)
        th0 = r.uniform(-math.pi / 2, math.pi / 2)
        e = (1 - q0) / (1 + q0)
        q, phi = oracle.ellipse(e * math.cos(2 * th0), e * math.sin(2 * th0))
        assert abs(q - q0) < 1e-13
        if q0 < 0.999:
            d = (phi - th0) % math.pi
            assert min(d, math.pi - d) < 1e-10


# ------------------------------------------------------------- Eq. (9)
def test_gammainc_matches_library():
    for a in (0.4, 0.6, 1.0, 2.0, 3.3, 8.0, 15.0, 20.0):
        for x in (1e-3, 0.1, 0.5, 1.0, a - 0.3, a, a + 2, 2 * a + 5):
            if x <= 0:
                continue
            ref = special.gammainc(a, x)
            assert abs(oracle.gammainc_P(a, x) - ref) <= 1e-13 * max(ref, 1e-300) + 1e-15


@pytest.mark.parametrize("n", [0.2, 0.3, 0.5, 0.8, 1.0, 1.5, 2.0, 2.5, 3.0,
                               4.0, 5.5, 8.0, 10.0])
def test_bn_root(n):
    """Eq. (9): Gamma(2n) = 2 gamma(2n, b_n) <=> P(2n, b_n) = 1/2, checked
    with the library's incomplete gamma and its inverse."""
    b = oracle.sersic_bn(n)
    assert abs(special.gammainc(2 * n, b) - 0.5) < 1e-14
    ref = special.gammaincinv(2 * n, 0.5)
    assert abs(b - ref) < 1e-12 * ref


def test_bn_closed_forms():
    """n = 1/2: P(1, b) = 1 - e^{-b} = 1/2 => b = ln 2 exactly.
    n >= 1: the leading terms of the Ciotti & Bertin (1999) asymptotic
    series, 2n - 1/3 + 4/(405 n) + 46/(25515 n^2), whose remainder is
    O(n^-3)."""
    assert abs(oracle.sersic_bn(0.5) - math.log(2.0)) < 1e-15
    for n in (1.0, 2.0, 4.0, 8.0, 16.0):
        cb = 2 * n - 1 / 3 + 4 / (405 * n) + 46 / (25515 * n ** 2)
        assert abs(oracle.sersic_bn(n) - cb) < 1.5e-4 / n ** 3


# ---------------------------------------------------- Eqs. (8), (10)
def test_sersic_unit_amplitude_and_centre():
    """Eq. (8) with I_e = 1: I = 1 on the isophote R_p = r_e and e^{b_n} at
    the centre; the major axis lies along theta_p (Eq. 10 with q < 1)."""
    for n in (0.5, 1.0, 4.0):
        b = special.gammaincinv(2 * n, 0.5)
        q, phi, re = 0.6, 0.4, 0.7
        assert abs(oracle.sersic(0.3, -0.2, 0.3, -0.2, q, phi, re, n, b)
                   - math.exp(b)) < 1e-12 * math.exp(b)
        # point on the major axis at distance re/sqrt(q): R_p = re
        x = 0.3 + re / math.sqrt(q) * math.cos(phi)
        y = -0.2 + re / math.sqrt(q) * math.sin(phi)
        assert abs(oracle.sersic(x, y, 0.3, -0.2, q, phi, re, n, b) - 1) < 1e-12
        # the same distance along the minor axis is fainter
        x2 = 0.3 - re / math.sqrt(q) * math.sin(phi)
        y2 = -0.2 + re / math.sqrt(q) * math.cos(phi)
        assert oracle.sersic(x2, y2, 0.3, -0.2, q, phi, re, n, b) < 0.5


@pytest.mark.parametrize("n,q,phi", [(0.5, 1.0, 0.0), (1.0, 0.55, 0.3),
                                     (2.5, 0.8, -1.1), (4.0, 0.7, 2.0)])
def test_sersic_half_light(n, q, phi):
    """Eq. (9)'s purpose: the flux inside R_p = r_e is half the total.  With
    R_p of Eq. (10) the isophote R_p = R encloses area pi R^2 for every q, so
    flux(<R) = int_0^R I(R') 2 pi R' dR'; I is read off the oracle along the
    rotated major axis and integrated by quadrature; the total must equal the
    closed form 2 pi n r_e^2 e^{b} Gamma(2n) / b^{2n}."""
    b = special.gammaincinv(2 * n, 0.5)
    re = 0.37

    def I_of_R(R):
        x = R / math.sqrt(q) * math.cos(phi)
        y = R / math.sqrt(q) * math.sin(phi)
        return oracle.sersic(x, y, 0.0, 0.0, q, phi, re, n, b)

    f = lambda R: I_of_R(R) * 2 * math.pi * R
    inner = integrate.quad(f, 0, re, epsabs=0, epsrel=1e-12, limit=400)[0]
    total = inner + integrate.quad(f, re, np.inf, epsabs=0, epsrel=1e-12,
                                   limit=400)[0]
    closed = 2 * math.pi * n * re ** 2 * math.exp(b) * math.gamma(2 * n) / b ** (2 * n)
    assert abs(total - closed) < 1e-8 * closed
    assert abs(inner / total - 0.5) < 1e-8


def test_sersic_flux_on_grid():
    """A finely supersampled, unblurred oracle image of the lens light sums
    (x pixel area) to the closed-form total flux: pins the grid (R1), the
    mean binning (R2) and the elliptical area of Eq. (10)."""
    n, re = 0.5, 0.4
    p = _vec(n_L=n, re_L=re, eps1_L=0.2, eps2_L=-0.1, x_L=0.13, y_L=-0.07)
    dpix, npx, sub = 0.05, 120, 3
    lens = oracle.Lens(np.zeros((npx, npx)), np.ones((npx, npx)),
                       np.ones((1, 1)), dpix, sub)
    il, _ = lens.unblurred(p)
    b = special.gammaincinv(2 * n, 0.5)
    closed = 2 * math.pi * n * re ** 2 * math.exp(b) * math.gamma(2 * n) / b ** (2 * n)
    assert abs(il.sum() * dpix ** 2 - closed) < 1e-6 * closed


# ---------------------------------------------- Eq. (12), gamma = 2
def _alpha_homoeoid(x, y, thE, q):
    """Independent SIE deflection (frame aligned with the ellipse) from the
    homoeoid integrals of an elliptical convergence kappa(xi),
    xi^2 = x^2 + y^2/q^2 (Schramm 1990; Keeton 2001):
      alpha_x = q x int_0^1 kappa(xi(u)) / (1-(1-q^2)u)^{1/2} du
      alpha_y = q y int_0^1 kappa(xi(u)) / (1-(1-q^2)u)^{3/2} du
      xi(u)^2 = u (x^2 + y^2 / (1-(1-q^2)u)).
    Eq. (12) at gamma = 2 with the Eq. (10) radius:
    kappa = thE / (2 sqrt(q x^2 + y^2/q)) = thE / (2 sqrt(q) xi)."""
    def kap(xi):
        return thE / (2 * math.sqrt(q) * xi)

    def xi(u):
        return math.sqrt(u * (x * x + y * y / (1 - (1 - q * q) * u)))

    jx = integrate.quad(lambda t: 2 * t * kap(xi(t * t))
                        / math.sqrt(1 - (1 - q * q) * t * t), 0, 1,
                        epsabs=1e-15, epsrel=1e-13, limit=200)[0]
    jy = integrate.quad(lambda t: 2 * t * kap(xi(t * t))
                        / (1 - (1 - q * q) * t * t) ** 1.5, 0, 1,
                        epsabs=1e-15, epsrel=1e-13, limit=200)[0]
    return q * x * jx, q * y * jy


def test_sie_vs_homoeoid_quadrature():
    r = np.random.default_rng(7)
    for _ in range(100):
        thE = r.uniform(0.3, 2.0)
        q = r.uniform(0.3, 0.999)
        phi = r.uniform(-math.pi / 2, math.pi / 2)
        xc, yc = r.normal(0, 0.1, 2)
        x, y = r.uniform(-2.5, 2.5, 2)
        ax, ay = oracle.sie_alpha(x, y, thE, q, phi, xc, yc)
        c, s = math.cos(phi), math.sin(phi)
        xp = (x - xc) * c + (y - yc) * s
        yp = -(x - xc) * s + (y - yc) * c
        hx, hy = _alpha_homoeoid(xp, yp, thE, q)
        rx, ry = hx * c - hy * s, hx * s + hy * c
        assert abs(ax - rx) < 1e-10 * thE and abs(ay - ry) < 1e-10 * thE


def test_sie_divergence_and_curl():
    """div alpha = 2 kappa (Poisson) and curl alpha = 0, by finite
    differences, with kappa from Eq. (12) at gamma = 2 and the Eq. (10)
    radius."""
    r = np.random.default_rng(8)
    h = 1e-5
    for _ in range(50):
        thE, q = r.uniform(0.5, 1.5), r.uniform(0.4, 0.98)
        phi = r.uniform(0, math.pi)
        x, y = r.uniform(-2, 2, 2)
        if math.hypot(x, y) < 0.2:
            continue
        f = lambda a, b: oracle.sie_alpha(a, b, thE, q, phi)
        dax = (f(x + h, y)[0] - f(x - h, y)[0]) / (2 * h)
        day = (f(x, y + h)[1] - f(x, y - h)[1]) / (2 * h)
        curl = (f(x + h, y)[1] - f(x - h, y)[1]) / (2 * h) - (
            f(x, y + h)[0] - f(x, y - h)[0]) / (2 * h)
        c, s = math.cos(phi), math.sin(phi)
        xp, yp = x * c + y * s, -x * s + y * c
        kappa = thE / (2 * math.sqrt(q * xp * xp + yp * yp / q))
        assert abs(dax + day - 2 * kappa) < 1e-6 * (1 + kappa)
        assert abs(curl) < 1e-6


def test_sie_sis_limit():
    """q = 1: the singular isothermal sphere, alpha = theta_E theta/|theta|;
    and continuity for q -> 1."""
    for (x, y) in [(0.3, 0.4), (-1.2, 0.5), (2.0, -2.0)]:
        r = math.hypot(x, y)
        ax, ay = oracle.sie_alpha(x, y, 1.3, 1.0, 0.7)
        assert abs(ax - 1.3 * x / r) < 1e-15 and abs(ay - 1.3 * y / r) < 1e-15
        q = (1 - 1e-9) / (1 + 1e-9)
        ax, ay = oracle.sie_alpha(x, y, 1.3, q, 0.7)
        assert abs(ax - 1.3 * x / r) < 1e-8 and abs(ay - 1.3 * y / r) < 1e-8


# ---------------------------------------------- Eq. (12), any gamma (EPL)
def _alpha_homoeoid_kappa(x, y, q, kap):
    """The homoeoid integrals above for any elliptical convergence kappa(xi),
    xi^2 = x^2 + y^2/q^2, with u = s^4 so that kappa ~ u^(-t/2) (t < 2) leaves
    a smooth integrand."""
    def xi(u):
        return math.sqrt(u * (x * x + y * y / (1 - (1 - q * q) * u)))

    def jx_f(s_):
        u = s_ ** 4
        return 4 * s_ ** 3 * kap(xi(u)) / math.sqrt(1 - (1 - q * q) * u)

    def jy_f(s_):
        u = s_ ** 4
        return 4 * s_ ** 3 * kap(xi(u)) / (1 - (1 - q * q) * u) ** 1.5

    jx = integrate.quad(jx_f, 0, 1, epsabs=1e-15, epsrel=1e-13, limit=400)[0]
    jy = integrate.quad(jy_f, 0, 1, epsabs=1e-15, epsrel=1e-13, limit=400)[0]
    return q * x * jx, q * y * jy


def _kappa_epl(thE, q, gamma):
    """Eq. (12) with the Eq. (10) radius R_p = sqrt(q) xi."""
    return lambda xi: (3 - gamma) / 2 * (thE / (math.sqrt(q) * xi)) ** (gamma - 1)


def test_epl_vs_homoeoid_quadrature():
    r = np.random.default_rng(17)
    for _ in range(60):
        thE = r.uniform(0.3, 2.0)
        q = r.uniform(0.3, 0.999)
        gamma = r.uniform(1.3, 2.7)
        phi = r.uniform(-math.pi / 2, math.pi / 2)
        xc, yc = r.normal(0, 0.1, 2)
        x, y = r.uniform(-2.5, 2.5, 2)
        ax, ay = oracle.epl_alpha(x, y, thE, q, phi, gamma, xc, yc)
        c, s = math.cos(phi), math.sin(phi)
        xp = (x - xc) * c + (y - yc) * s
        yp = -(x - xc) * s + (y - yc) * c
        hx, hy = _alpha_homoeoid_kappa(xp, yp, q, _kappa_epl(thE, q, gamma))
        rx, ry = hx * c - hy * s, hx * s + hy * c
        scale = thE + math.hypot(rx, ry)
        assert abs(ax - rx) < 1e-9 * scale and abs(ay - ry) < 1e-9 * scale, (gamma, q)


def test_epl_circular_closed_form():
    """q = 1: alpha = theta_E (theta_E/r)^(gamma-2) theta/|theta| (the
    enclosed convergence of Eq. 12), so |theta| = theta_E maps to beta = 0."""
    for gamma in (1.4, 2.0, 2.6):
        for (x, y) in [(0.3, 0.4), (-1.2, 0.5), (2.0, -2.0)]:
            r = math.hypot(x, y)
            ax, ay = oracle.epl_alpha(x, y, 1.3, 1.0, 0.7, gamma)
            a = 1.3 * (1.3 / r) ** (gamma - 2)
            assert abs(ax - a * x / r) < 1e-13 and abs(ay - a * y / r) < 1e-13
        ax, ay = oracle.epl_alpha(1.3 * 0.6, 1.3 * 0.8, 1.3, 1.0, 0.0, gamma)
        assert abs(ax - 1.3 * 0.6) < 1e-13 and abs(ay - 1.3 * 0.8) < 1e-13


def test_epl_is_sie_at_gamma_2():
    r = np.random.default_rng(18)
    for _ in range(50):
        thE, q, phi = r.uniform(0.3, 2.0), r.uniform(0.3, 0.999), r.uniform(0, math.pi)
        x, y = r.uniform(-2.5, 2.5, 2)
        a = oracle.epl_alpha(x, y, thE, q, phi, 2.0)
        b = oracle.sie_alpha(x, y, thE, q, phi)
        assert abs(a[0] - b[0]) < 1e-12 * thE and abs(a[1] - b[1]) < 1e-12 * thE


def test_epl_divergence_and_curl():
    """div alpha = 2 kappa (Eq. 12, any gamma) and curl alpha = 0."""
    r = np.random.default_rng(19)
    h = 1e-5
    for _ in range(50):
        thE, q, gamma = r.uniform(0.5, 1.5), r.uniform(0.4, 0.98), r.uniform(1.4, 2.6)
        phi = r.uniform(0, math.pi)
        x, y = r.uniform(-2, 2, 2)
        if math.hypot(x, y) < 0.2:
            continue
        f = lambda a, b: oracle.epl_alpha(a, b, thE, q, phi, gamma)
        dax = (f(x + h, y)[0] - f(x - h, y)[0]) / (2 * h)
        day = (f(x, y + h)[1] - f(x, y - h)[1]) / (2 * h)
        curl = (f(x + h, y)[1] - f(x - h, y)[1]) / (2 * h) - (
            f(x, y + h)[0] - f(x, y - h)[0]) / (2 * h)
        c, s = math.cos(phi), math.sin(phi)
        xp, yp = x * c + y * s, -x * s + y * c
        kappa = (3 - gamma) / 2 * (thE / math.sqrt(q * xp * xp + yp * yp / q)) ** (gamma - 1)
        assert abs(dax + day - 2 * kappa) < 1e-6 * (1 + kappa)
        assert abs(curl) < 1e-6


def test_epl_lens_validity_and_batch():
    """EPL lenses take 22 entries (gamma last, valid in (1, 3)); the batch
    equals single evaluations; gamma = 2 gives the SIE lens's log L."""
    rng = np.random.default_rng(20)
    ny = nx = 12
    psf = W.gaussian_psf(5, 1.5)
    data = rng.normal(size=(ny, nx))
    sig = np.ones((ny, nx))
    le = oracle.Lens(data, sig, psf, 0.1, 2, mass="epl")
    ls = oracle.Lens(data, sig, psf, 0.1, 2)
    P = W.draw_prior(rng, 6).astype(np.float64)
    Pe = np.concatenate([P, np.full((6, 1), 2.0)], axis=1)
    assert np.allclose(le.loglike_batch(Pe), ls.loglike_batch(P), rtol=1e-11, atol=1e-9)
    Pe[:, 21] = [1.5, 2.5, 1.0, 3.0, np.nan, 2.2]
    out = le.loglike_batch(Pe)
    assert np.isneginf(out[[2, 3, 4]]).all() and np.isfinite(out[[0, 1, 5]]).all()
    single = [le.loglike(Pe[k]) for k in range(6)]
    assert np.array_equal(np.asarray(single), out)


def test_einstein_ring():
    """Circular SIS, no shear: every point on |theta| = theta_E maps to
    beta = 0 (Eq. 1)."""
    p = _vec(theta_E=1.17)
    for t in np.linspace(0, 2 * math.pi, 37):
        bx, by = oracle.trace_point(p, 1.17 * math.cos(t), 1.17 * math.sin(t))
        assert abs(bx) < 1e-14 and abs(by) < 1e-14
    bx, by = oracle.trace_point(p, 2.0, 0.0)  # outside: beta = (2 - 1.17, 0)
    assert abs(bx - 0.83) < 1e-14 and abs(by) < 1e-15


# ----------------------------------------------------- Eqs. (13), (14)
def test_shear_is_gradient_of_potential():
    r = np.random.default_rng(9)
    h = 1e-6
    for _ in range(20):
        g1, g2 = r.normal(0, 0.1, 2)
        x, y = r.uniform(-2, 2, 2)
        ax, ay = oracle.shear_alpha(x, y, g1, g2)
        px = (oracle.shear_potential(x + h, y, g1, g2)
              - oracle.shear_potential(x - h, y, g1, g2)) / (2 * h)
        py = (oracle.shear_potential(x, y + h, g1, g2)
              - oracle.shear_potential(x, y - h, g1, g2)) / (2 * h)
        assert abs(ax - px) < 1e-8 and abs(ay - py) < 1e-8


def test_shear_components_and_polar_form():
    """Cartesian components: (psi_11 - psi_22)/2 = gamma_1, psi_12 = gamma_2,
    psi_11 + psi_22 = 0 (no convergence), alpha(0) = 0; and the potential is
    Eq. (13)'s polar form with gamma_ext = |gamma| (Eq. 14) at the angle
    whose tan 2phi = gamma_2/gamma_1 (Eq. 14) on the branch
    gamma_1 = -gamma cos 2phi."""
    g1, g2 = 0.031, -0.047
    h = 1e-3
    a = lambda x, y: oracle.shear_alpha(x, y, g1, g2)
    psi11 = (a(h, 0)[0] - a(-h, 0)[0]) / (2 * h)
    psi22 = (a(0, h)[1] - a(0, -h)[1]) / (2 * h)
    psi12 = (a(0, h)[0] - a(0, -h)[0]) / (2 * h)
    assert abs(0.5 * (psi11 - psi22) - g1) < 1e-14
    assert abs(psi12 - g2) < 1e-14
    assert abs(psi11 + psi22) < 1e-14
    assert oracle.shear_alpha(0.0, 0.0, g1, g2) == (0.0, 0.0)
    gam = math.hypot(g1, g2)
    phi_ext = 0.5 * math.atan2(-g2, -g1)
    assert abs(math.tan(2 * phi_ext) - g2 / g1) < 1e-12
    for (x, y) in [(0.4, 0.9), (-1.3, 0.2), (0.7, -0.8)]:
        th, vphi = math.hypot(x, y), math.atan2(y, x)
        polar = -0.5 * gam * th * th * math.cos(2 * (vphi - phi_ext))
        assert abs(oracle.shear_potential(x, y, g1, g2) - polar) < 1e-15


def test_lens_equation_composition():
    """Eq. (1) with SIE + shear: beta = theta - alpha_SIE - alpha_shear
    (each pinned above), checked on random points."""
    r = np.random.default_rng(10)
    for _ in range(20):
        p = _vec(theta_E=r.uniform(0.5, 1.5), eps1_m=r.normal(0, 0.1),
                 eps2_m=r.normal(0, 0.1), x_m=r.normal(0, 0.05),
                 y_m=r.normal(0, 0.05), gamma_1=r.normal(0, 0.05),
                 gamma_2=r.normal(0, 0.05))
        x, y = r.uniform(-2, 2, 2)
        q, phi = oracle.ellipse(p[1], p[2])
        ax, ay = oracle.sie_alpha(x, y, p[0], q, phi, p[3], p[4])
        sx, sy = oracle.shear_alpha(x, y, p[5], p[6])
        bx, by = oracle.trace_point(p, x, y)
        assert abs(bx - (x - ax - sx)) < 1e-14 and abs(by - (y - ay - sy)) < 1e-14


# -------------------------------------------------------------- Eq. (3)
def test_convolution_vs_library():
    r = np.random.default_rng(11)
    for (ny, nx, k) in [(7, 9, 3), (16, 13, 5), (20, 20, 11), (5, 4, 7)]:
        img = r.random((ny, nx))
        psf = r.random((k, k))
        psf /= psf.sum()
        ref = signal.convolve2d(img, psf, mode="same", boundary="fill")
        assert np.allclose(oracle.convolve(img, psf), ref, rtol=1e-13, atol=1e-15)


def test_convolution_orientation_and_identity():
    """A point source reproduces the (asymmetric) kernel centred on it, the
    true-convolution orientation; a delta kernel is the identity; a unit-sum
    kernel conserves the flux of a source away from the edges."""
    k = 5
    psf = np.arange(1, k * k + 1, dtype=float).reshape(k, k)
    psf /= psf.sum()
    img = np.zeros((15, 15))
    img[6, 8] = 1.0
    out = oracle.convolve(img, psf)
    assert np.allclose(out[4:9, 6:11], psf, rtol=0, atol=1e-16)
    r = np.random.default_rng(12)
    im = r.random((9, 11))
    assert np.array_equal(oracle.convolve(im, np.ones((1, 1))), im)
    d3 = np.zeros((3, 3)); d3[1, 1] = 1.0
    assert np.array_equal(oracle.convolve(im, d3), im)
    src = np.zeros((30, 30)); src[12:18, 13:16] = r.random((6, 3))
    g = np.exp(-0.5 * ((np.arange(7) - 3) / 1.2) ** 2)
    gk = np.outer(g, g); gk /= gk.sum()
    assert abs(oracle.convolve(src, gk).sum() - src.sum()) < 1e-13


def test_psf_normalise():
    psf = np.random.default_rng(3).random((7, 7)) * 5
    out = oracle.psf_normalise(psf)
    assert abs(out.sum() - 1) < 1e-15
    with pytest.raises(ValueError):
        oracle.psf_normalise(np.zeros((3, 3)))


# ----------------------------------------------------- Sec. 2.3 NNLS
def _weighted_nnls_lib(ml, ms, d, w):
    sw = np.sqrt(w)
    M = np.stack([ml * sw, ms * sw], axis=1)
    s, _ = optimize.nnls(M, d * sw)
    return s


def test_nnls2_vs_library_and_kkt():
    r = np.random.default_rng(13)
    for trial in range(300):
        n = r.integers(3, 40)
        ml, ms = r.random(n), r.random(n)
        if trial % 5 == 0:
            ms = ml * 0.9 + 0.1 * r.random(n)      # nearly collinear
        d = r.normal(0, 1, n) + r.uniform(-1, 2) * ml + r.uniform(-1, 2) * ms
        w = r.uniform(0.2, 3.0, n)
        w[r.random(n) < 0.1] = 0.0
        s = oracle.nnls2(ml, ms, d, w)
        assert s[0] >= 0 and s[1] >= 0
        lib = _weighted_nnls_lib(ml, ms, d, w)
        c_or = oracle.chi2(ml, ms, d, w, s[0], s[1])
        c_lib = oracle.chi2(ml, ms, d, w, lib[0], lib[1])
        assert c_or <= c_lib * (1 + 1e-12) + 1e-12
        # KKT: gradient g = A s - b >= 0, s_k g_k = 0
        A = np.array([[np.sum(w * ml * ml), np.sum(w * ml * ms)],
                      [np.sum(w * ml * ms), np.sum(w * ms * ms)]])
        b = np.array([np.sum(w * ml * d), np.sum(w * ms * d)])
        g = A @ s - b
        scale = np.abs(A).max() * (np.abs(s).max() + 1) + np.abs(b).max()
        assert np.all(g >= -1e-9 * scale)
        assert np.all(np.abs(s * g) <= 1e-9 * scale * (np.abs(s).max() + 1))


def test_nnls2_brute_force():
    r = np.random.default_rng(14)
    for _ in range(20):
        n = 12
        ml, ms = r.random(n), r.random(n)
        d = r.normal(0, 1, n) + r.uniform(-1, 2) * ml + r.uniform(-1, 2) * ms
        w = r.uniform(0.5, 2.0, n)
        s = oracle.nnls2(ml, ms, d, w)
        grid = np.linspace(0, 4, 401)
        best = min(oracle.chi2(ml, ms, d, w, a, c) for a in grid[::4] for c in grid[::4])
        assert oracle.chi2(ml, ms, d, w, s[0], s[1]) <= best + 1e-12


# -------------------------------------------- Sec. 2.1 grid, Eq. (5)
def test_tiny_grid_by_hand():
    """2x2 pixels, 2x2 subpixels, delta PSF, fixed amplitudes: each pixel is
    the mean of the lens-light Sersic at the four subpixel centres computed
    here by hand (R1, R2); the grid's +x runs along columns, +y along rows."""
    n, re = 1.0, 0.3
    b = special.gammaincinv(2 * n, 0.5)
    p = _vec(n_L=n, re_L=re, x_L=0.05, y_L=-0.02, Ie_S=0.0)
    dpix = 0.1
    lens = oracle.Lens(np.zeros((2, 2)), np.ones((2, 2)), np.ones((1, 1)), dpix, 2)
    il, _ = lens.unblurred(p)
    for i in range(2):
        for j in range(2):
            xc = -0.05 + j * dpix
            yc = -0.05 + i * dpix
            vals = []
            for a in range(2):
                for c in range(2):
                    x = xc + ((c + 0.5) / 2 - 0.5) * dpix
                    y = yc + ((a + 0.5) / 2 - 0.5) * dpix
                    R = math.hypot(x - 0.05, y + 0.02)
                    vals.append(math.exp(-b * ((R / re) ** (1 / n) - 1)))
            assert abs(il[i, j] - np.mean(vals)) < 1e-14


def test_single_pixel_loglike_by_hand():
    """1x1 image, 1 subpixel, delta PSF, lens light centred on the pixel so
    the model is I_e e^{b_n}; Eq. (5): log L = -(d - m)^2/(2 s^2)
    - log(2 pi s^2)/2, in fixed-amplitude mode and with NNLS (which then
    fits d exactly: m = d)."""
    n = 2.0
    b = special.gammaincinv(2 * n, 0.5)
    Ie, d, s = 0.7, 3.1, 0.4
    p = _vec(n_L=n, Ie_L=Ie, Ie_S=0.0, theta_E=0.0, x_S=50.0)
    lens = oracle.Lens(np.array([[d]]), np.array([[s]]), np.ones((1, 1)), 0.1, 1)
    m = Ie * math.exp(b)
    expect = -0.5 * (d - m) ** 2 / s ** 2 - 0.5 * math.log(2 * math.pi * s * s)
    assert abs(lens.loglike(p, mode=1) - expect) < 1e-13 * abs(expect)
    assert abs(lens.loglike(p, mode=0) + 0.5 * math.log(2 * math.pi * s * s)) < 1e-12


def test_exact_model_recovers_amplitudes():
    """Noiseless data built from the oracle's own columns at the truth:
    NNLS returns the true amplitudes and chi^2 = 0, so log L is the
    normalisation alone; masked pixels (sigma <= 0, non-finite sigma or
    data) drop out of both terms (Eq. 5 over unmasked pixels)."""
    r = np.random.default_rng(15)
    ny, nx = 24, 20
    psf = np.exp(-0.5 * ((np.arange(5) - 2) / 0.9) ** 2)
    psf = np.outer(psf, psf)
    p = _vec(theta_E=0.6, eps1_m=0.1, x_S=0.05, y_S=0.02, re_S=0.15, re_L=0.3)
    lens0 = oracle.Lens(np.zeros((ny, nx)), np.ones((ny, nx)), psf, 0.05, 2)
    _, ml, ms, _, _ = lens0.model(p, mode=1)
    d = 3.0 * ml + 7.0 * ms
    sig = r.uniform(0.5, 2.0, (ny, nx))
    sig[0, 0] = 0.0
    sig[1, 3] = np.inf
    sig[2, 5] = -1.0
    d[4, 4] = np.nan
    lens = oracle.Lens(d, sig, psf, 0.05, 2)
    ll, _, _, _, amps = lens.model(p, mode=0)
    assert abs(amps[0] - 3.0) < 1e-9 and abs(amps[1] - 7.0) < 1e-9
    ok = np.isfinite(sig) & (sig > 0) & np.isfinite(d)
    norm = -0.5 * np.sum(np.log(2 * math.pi * sig[ok] ** 2))
    assert abs(ll - norm) < 1e-9



def _masked_noisy(r, ml_cols, amps, ny, nx):
    """Noisy data from the columns, then five masked pixels whose values
    would dominate any fit that used them: sigma 0, negative, infinite or
    NaN, and a NaN datum under a valid sigma."""
    sig = r.uniform(0.4, 1.6, (ny, nx))
    d = np.tensordot(amps, ml_cols, axes=1) + r.normal(0.0, 1.0, (ny, nx)) * sig
    spots = [(0, 0), (3, 7), (ny // 2, nx // 2), (ny - 1, nx - 1), (5, 5)]
    vals = [(0.0, 1e6), (-2.0, -1e6), (np.inf, 5e5), (np.nan, 1e6), (1.0, np.nan)]
    for (i, j), (sv, dv) in zip(spots, vals):
        sig[i, j], d[i, j] = sv, dv
    ok = np.isfinite(sig) & (sig > 0) & np.isfinite(d)
    assert ok.sum() == ny * nx - 5
    return d, sig, ok


def _library_fit(cols, d, sig, ok):
    """Eq. 5 over the unmasked pixels at the NNLS amplitudes, with the NNLS
    taken from scipy on the sigma-weighted columns."""
    w = 1.0 / sig[ok]
    A = np.stack([c[ok] * w for c in cols], axis=1)
    x, rnorm = optimize.nnls(A, d[ok] * w)
    return -0.5 * rnorm ** 2 - 0.5 * np.sum(np.log(2 * math.pi * sig[ok] ** 2)), x


def test_masked_pixels_leave_the_fit():
    """Masked pixels drop out of Eq. 5 and of the amplitudes' NNLS: with
    noisy data, the oracle's log L and amplitudes equal a library NNLS fit of
    its blurred unit columns to the unmasked pixels alone.  A masked pixel
    that reached the normal equations or either term of Eq. 5 would move the
    result by orders of magnitude (their data are +-1e6 or NaN)."""
    r = np.random.default_rng(31)
    ny, nx = 22, 26
    psf = np.exp(-0.5 * ((np.arange(7) - 3.0)[:, None] ** 2 + (np.arange(7) - 3.0)[None, :] ** 2) / 1.4)
    p = _vec(theta_E=0.7, eps1_m=0.1, eps2_m=-0.05, x_S=0.04, y_S=-0.03, re_S=0.2,
             re_L=0.4, n_L=3.0, eps1_L=0.1)
    lens0 = oracle.Lens(np.zeros((ny, nx)), np.ones((ny, nx)), psf, 0.06, 3)
    _, ml, ms, _, _ = lens0.model(p, mode=1)
    d, sig, ok = _masked_noisy(r, np.stack([ml, ms]), np.array([2.5, 6.0]), ny, nx)
    ll_ref, x_ref = _library_fit([ml, ms], d, sig, ok)
    ll, _, _, _, amps = oracle.Lens(d, sig, psf, 0.06, 3).model(p, mode=0)
    assert abs(ll - ll_ref) <= 1e-9 * abs(ll_ref)
    assert np.allclose(amps, x_ref, rtol=1e-8, atol=1e-10)


def test_fully_masked_lens():
    """No unmasked pixel: both sums of Eq. 5 are empty, so log L = 0 and the
    amplitudes are 0, for either kind of mask and for the multi-component
    model too."""
    ny, nx = 10, 12
    psf = np.ones((3, 3))
    comps = [dict(type="sersic", plane="lens", index=1.0),
             dict(type="gauss", plane="source")]
    mp = np.concatenate([_vec()[:7], [0.0, 0.0, 0.0, 0.0], [0.0, 0.0, 0.0, 0.0], [0.5, 0.2]])
    for d, sig in ((np.full((ny, nx), np.nan), np.ones((ny, nx))),
                   (np.ones((ny, nx)), np.full((ny, nx), np.inf))):
        ll, _, _, _, amps = oracle.Lens(d, sig, psf, 0.1, 2).model(_vec(), mode=0)
        assert ll == 0.0 and not np.any(amps)
        llm, _, _, ampm = oracle.MultiLens(d, sig, psf, 0.1, 2, comps).model(mp)
        assert llm == 0.0 and not np.any(ampm)

def test_invalid_vectors():
    lens = oracle.Lens(np.zeros((4, 4)), np.ones((4, 4)), np.ones((1, 1)), 0.1, 1)
    bad = [dict(eps1_m=0.8, eps2_m=0.7), dict(eps1_L=1.0), dict(eps2_S=-1.2),
           dict(re_L=0.0), dict(re_S=-0.1), dict(n_L=0.1), dict(n_S=12.0),
           dict(theta_E=-0.1), dict(x_S=np.nan), dict(gamma_1=np.inf)]
    for kw in bad:
        assert lens.loglike(_vec(**kw)) == -np.inf
    assert np.isfinite(lens.loglike(_vec()))


def test_lensed_ring_radius():
    """Whole forward model: circular SIS, compact round source at the
    origin; the lensed-source column peaks on the Einstein ring."""
    p = _vec(theta_E=0.8, re_S=0.03, n_S=0.5, Ie_L=0.0)
    npx, dpix = 60, 0.04
    lens = oracle.Lens(np.zeros((npx, npx)), np.ones((npx, npx)),
                       np.ones((1, 1)), dpix, 3)
    _, is_ = lens.unblurred(p)
    yy, xx = np.mgrid[0:npx, 0:npx]
    x = -(npx - 1) * dpix / 2 + xx * dpix
    y = -(npx - 1) * dpix / 2 + yy * dpix
    r = np.hypot(x, y)
    bins = np.arange(0, 1.2, dpix)
    idx = np.digitize(r.ravel(), bins)
    prof = [is_.ravel()[idx == k].mean() for k in range(1, len(bins))]
    peak_r = bins[int(np.argmax(prof))] + dpix / 2
    assert abs(peak_r - 0.8) <= dpix


def test_batch_equals_single():
    r = np.random.default_rng(16)
    lens = oracle.Lens(r.normal(0, 1, (12, 10)), np.ones((12, 10)),
                       np.ones((3, 3)), 0.08, 2)
    P = np.stack([_vec(theta_E=t, x_S=0.02 * t) for t in (0.5, 0.7, 0.9, 1.1)])
    out = lens.loglike_batch(P, nthreads=2)
    for k in range(4):
        assert out[k] == lens.loglike(P[k])
