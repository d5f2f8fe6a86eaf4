"""The seeded input generator: reproducible, in range, unit-sum PSFs."""
import numpy as np

from paper_2503_08586_gb300 import workloads as W


def test_psfs_unit_sum_and_symmetric():
    for k, fw in ((11, 2.0), (21, 2.03), (31, 2.0)):
        g = W.gaussian_psf(k, fw)
        assert g.dtype == np.float32 and g.shape == (k, k)
        assert abs(float(g.astype(np.float64).sum()) - 1) < 1e-6
        assert np.array_equal(g, g.T) and np.array_equal(g, g[::-1, ::-1])
    m = W.moffat_psf(31, 2.0, 3.0)
    assert abs(float(m.astype(np.float64).sum()) - 1) < 1e-6
    # FWHM of the Moffat: half maximum at r = FWHM/2 along an axis
    r = np.arange(31) - 15
    alpha = 2.0 / (2 * np.sqrt(2 ** (1 / 3) - 1))
    prof = (1 + (1.0 / alpha) ** 2) ** -3
    assert abs(prof - 0.5) < 1e-12


def test_priors_in_range_and_reproducible():
    r1 = np.random.Generator(np.random.PCG64(5))
    r2 = np.random.Generator(np.random.PCG64(5))
    a, b = W.draw_prior(r1, 500), W.draw_prior(r2, 500)
    assert np.array_equal(a, b) and a.shape == (500, 21) and a.dtype == np.float32
    assert a[:, 0].min() >= 0.5 and a[:, 0].max() <= 1.5
    for i, j in ((1, 2), (10, 11), (17, 18)):
        e = np.hypot(a[:, i], a[:, j])
        assert e.max() <= 1 / 3 + 1e-6
    assert np.all((a[:, 9] >= 1) & (a[:, 9] <= 4))
    assert np.all(np.hypot(a[:, 19], a[:, 20]) <= 0.3 + 1e-6)
    assert np.array_equal(a[:, 12], a[:, 3]) and np.array_equal(a[:, 13], a[:, 4])


def test_synth_lens_uses_render_and_noise_model():
    calls = []

    def fac(ps, sub, psf, ny, nx):
        def render(p):
            calls.append(p.copy())
            yy, xx = np.mgrid[0:ny, 0:nx]
            return np.exp(-((xx - nx / 2) ** 2 + (yy - ny / 2) ** 2) / 20.0), \
                np.exp(-((xx - nx / 3) ** 2 + (yy - ny / 3) ** 2) / 10.0)
        return render

    lens, params = W.workload("csst100", fac, batch=16)
    assert len(calls) == 1 and params.shape == (16, 21)
    assert lens.data.shape == (100, 100) and lens.noise.min() >= 1.0
    assert lens.x0 == W.f32(-99 * W.f32(0.074) / 2) and lens.pixel_scale == W.f32(0.074)
    lens2, _ = W.workload("csst100", fac, batch=16)
    assert np.array_equal(lens.data, lens2.data)


def test_ragged_and_stream_descriptors():
    _, specs = W.ragged_specs(50)
    assert all(s in W.RAGGED_SIDES and 11 <= k <= 31 and k % 2 for s, k in specs)
    jobs = W.request_stream(10, iters=5)
    t = [j["arrival"] for j in jobs]
    assert t == sorted(t) and all(500 <= b <= 5000 for j in jobs for b in j["batches"])
