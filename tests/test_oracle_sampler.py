"""Pins for the oracle's sampler loop (the stretch move of Goodman & Weare
2010 with Philox4x32-10 random numbers; the paper's Sec. 4.2 proposes
moving the sampler to the GPU): published known answers of the generator,
the stretch factor's distribution, the proposal arithmetic, and
stationarity on a target with known moments.  CPU only."""
import math
import os

import numpy as np
import pytest
from scipy import stats

import oracle

HERE = os.path.dirname(os.path.abspath(__file__))


def test_philox_known_answers():
    rows = [l.split() for l in open(os.path.join(HERE, "golden", "philox4x32_10_kat.txt"))
            if l.strip() and not l.startswith("#")]
    assert len(rows) == 3
    for r in rows:
        v = [int(t, 16) for t in r]
        assert oracle.philox4x32_10(v[0:4], v[4:6]) == v[6:10]


def test_philox_uniformity():
    """Outputs over consecutive counters are uniform (chi-square on the top
    byte of each word)."""
    counts = np.zeros(256)
    for c in range(4096):
        for w in oracle.philox4x32_10([c, 7, 0, 0], [123, 456]):
            counts[w >> 24] += 1
    assert stats.chisquare(counts).pvalue > 1e-3


def test_stretch_factor_distribution_and_partners():
    """z has density ~ 1/sqrt(z) on [1/a, a]: CDF (sqrt(a z) - 1)/(a - 1)
    (Kolmogorov-Smirnov); partners lie in the other half, uniformly."""
    W, P, a = 64, 3, 2.0
    x = np.random.default_rng(1).normal(size=(W, P)).astype(np.float32)
    zs, js = [], []
    for step in range(200):
        for h in (0, 1):
            _, z, j = oracle.stretch_propose(x, h, step, 99, a)
            zs.append(z)
            js.append(j if h == 0 else j + W // 2)   # h=0 partners in [W/2, W)
            assert np.all((j >= (1 - h) * W // 2) & (j < (2 - h) * W // 2))
    z = np.concatenate(zs)
    assert z.min() >= 1 / a and z.max() <= a
    cdf = lambda v: (np.sqrt(a * v) - 1) / (a - 1)
    assert stats.kstest(z, cdf).pvalue > 1e-3
    part = np.concatenate(js) % (W // 2)
    assert stats.chisquare(np.bincount(part, minlength=W // 2)).pvalue > 1e-3


def test_proposal_arithmetic_bit_exact():
    """Y = float32(x_j + z (x_k - x_j)) with each FP64 operation rounded once
    (numpy evaluates the same operations without contraction)."""
    W, P = 16, 21
    x = np.random.default_rng(2).normal(size=(W, P)).astype(np.float32)
    for h in (0, 1):
        Y, z, j = oracle.stretch_propose(x, h, 5, 2024, 2.5)
        k = np.arange(W // 2) + h * W // 2
        xj = x[j].astype(np.float64)
        d = x[k].astype(np.float64) - xj
        want = (xj + z[:, None] * d).astype(np.float32)
        assert np.array_equal(Y, want)


def _gauss_target():
    C = np.array([[1.0, 0.6, 0.0], [0.6, 2.0, -0.5], [0.0, -0.5, 0.5]])
    Ci = np.linalg.inv(C)

    def logp(Y):
        Y = np.asarray(Y, np.float64)
        return -0.5 * np.einsum("ni,ij,nj->n", Y, Ci, Y)
    return C, logp


def _moments(ndim):
    C, logp = _gauss_target()
    W = 64
    x0 = np.random.default_rng(3).normal(scale=0.1, size=(W, 3)).astype(np.float32)
    lo, hi = np.full(3, -50.0, np.float32), np.full(3, 50.0, np.float32)
    chain, lpc, rate = oracle.stretch_run(x0, logp, 1500, 7, lo, hi, ndim=ndim)
    s = chain[300:].reshape(-1, 3).astype(np.float64)
    return C, s.mean(axis=0), np.cov(s.T), rate


def test_stretch_move_is_stationary_on_a_gaussian():
    """Goodman & Weare's move with the z^(d-1) factor leaves the target
    invariant: the chain's mean and covariance match a correlated 3-D
    Gaussian's; the same run with the factor's exponent wrong (a planted
    mistake, d taken as 1) misses them."""
    C, m, S, rate = _moments(3)
    assert 0.2 < rate < 0.9
    assert np.all(np.abs(m) < 0.12)
    assert np.max(np.abs(S - C) / np.sqrt(np.outer(np.diag(C), np.diag(C)))) < 0.1
    _, _, Sb, _ = _moments(1)
    assert np.max(np.abs(np.diag(Sb) - np.diag(C)) / np.diag(C)) > 0.2


def test_box_prior_and_fixed_coordinates():
    """A proposal leaving [lo, hi] is rejected; lo == hi coordinates never
    move (every walker starts there and the move is affine)."""
    W, P = 32, 3
    r = np.random.default_rng(4)
    x = r.uniform(-1, 1, (W, P)).astype(np.float32)
    x[:, 2] = 0.25
    lo = np.array([-1, -1, 0.25], np.float32)
    hi = np.array([1, 1, 0.25], np.float32)
    lp = np.zeros(W)
    for step in range(50):
        for h in (0, 1):
            Y, z, _ = oracle.stretch_propose(x, h, step, 11)
            out = np.any((Y[:, :2] < lo[:2]) | (Y[:, :2] > hi[:2]), axis=1)
            acc = oracle.stretch_accept(x, lp, h, step, 11, 2, Y, z, np.zeros(W // 2), lo, hi)
            assert not np.any(acc[out])
    assert np.all(x[:, 2] == np.float32(0.25))
    assert np.all((x[:, :2] >= -1) & (x[:, :2] <= 1))
