"""The kernels' table of the EPL deflection series (host-side check of its
design constants, no GPU).

The deflection of the elliptical power law (Eq. 12 at slope gamma) carries
the angular sum sum_n c_n e^{i (2n+1) vphi} with c_0 = 1 and
c_n = c_{n-1} (2n - 2 + t)/(2n + 2 - t) (-(1-q)/(1+q)), t = gamma - 1 (the
hypergeometric series of Tessore & Metcalf 2015).  The kernels write it as
cos(vphi) F1(x) + i sin(vphi) F2(x) with x = cos(2 vphi), and, where the
ratio r = (1-q)/(1+q) is at most kEplTabR, take F1 and F2 from kEplTab
cubic Hermite intervals over x in [-1, 1] built per vector.  This file
checks, in FP64:
  * the factorisation itself against the direct complex sum;
  * that the table's interpolation error stays below 2e-8 of the sum at the
    largest ratio the kernels allow, for slopes 1.2 .. 2.8 (the float sum's
    own rounding is ~6e-8);
  * that the workloads' mass prior (q >= 0.5) lies inside that range.
kEplTab and kEplTabR are read from the kernel header."""
import os
import re

import numpy as np

HDR = os.path.join(os.path.dirname(__file__), "..", "paper_2503_08586_gb300", "csrc",
                   "tll_device.cuh")


def _header_const(name):
    src = open(HDR).read()
    m = re.search(r"constexpr\s+\w+\s+" + name + r"\s*=\s*([0-9.]+)f?;", src)
    assert m, name
    return float(m.group(1))


def _coeffs(r, t, nmax=400):
    c = [1.0]
    for n in range(1, nmax + 1):
        c.append(c[-1] * (-r) * (2 * n - 2 + t) / (2 * n + 2 - t))
        if abs(c[-1]) < 1e-18:
            break
    return np.array(c)


def _sums(c, x):
    """F1, F2 at x and their x-derivatives (Clenshaw in alpha = 2x)."""
    al = 2.0 * x
    b1 = np.zeros_like(x); b2 = np.zeros_like(x)
    d1 = np.zeros_like(x); d2 = np.zeros_like(x)
    for ck in c[::-1]:
        b0 = al * b1 + ck - b2
        d0 = b1 + al * d1 - d2
        b2, b1 = b1, b0
        d2, d1 = d1, d0
    return b1 - b2, b1 + b2, 2 * (d1 - d2), 2 * (d1 + d2)


def test_factorisation_matches_direct_sum():
    rng = np.random.Generator(np.random.PCG64(11))
    for r, t in ((0.1, 0.6), (1 / 3, 1.0), (0.35, 1.8), (0.6, 0.2)):
        c = _coeffs(r, t)
        phi = rng.uniform(-np.pi, np.pi, 200)
        direct = np.array([np.sum(c * np.exp(1j * (2 * np.arange(len(c)) + 1) * p))
                           for p in phi])
        F1, F2, _, _ = _sums(c, np.cos(2 * phi))
        got = np.cos(phi) * F1 + 1j * np.sin(phi) * F2
        assert np.max(np.abs(got - direct)) < 1e-12 * np.max(np.abs(direct))


def test_table_interpolation_bound():
    N = int(_header_const("kEplTab"))
    rmax = _header_const("kEplTabR")
    h = 2.0 / N
    x = np.linspace(-1.0, 1.0, 100001)
    for t in (0.2, 0.6, 1.0, 1.4, 1.8):
        c = _coeffs(rmax, t)
        nodes = -1.0 + (np.arange(N + 3) - 1) * h          # intervals 0 .. N+1
        F1n, F2n, D1n, D2n = _sums(c, nodes)
        U = (x + 1.0) / h + 1.0
        k = np.clip(np.floor(U).astype(int), 0, N + 1)
        s = U - k
        F1x, F2x, _, _ = _sums(c, x)
        for Fn, Dn, ref in ((F1n, D1n, F1x), (F2n, D2n, F2x)):
            a0 = Fn[k]
            a1 = h * Dn[k]
            a2 = 3 * (Fn[k + 1] - Fn[k]) - h * (2 * Dn[k] + Dn[k + 1])
            a3 = 2 * (Fn[k] - Fn[k + 1]) + h * (Dn[k] + Dn[k + 1])
            p = ((a3 * s + a2) * s + a1) * s + a0
            err = np.max(np.abs(p - ref)) / np.max(np.abs(ref))
            assert err < 2e-8, (t, err)


def test_prior_masses_take_the_table():
    rmax = _header_const("kEplTabR")
    q_min = 0.5                       # the workloads' mass prior: q ~ U[0.5, 1]
    assert (1 - q_min) / (1 + q_min) <= rmax
