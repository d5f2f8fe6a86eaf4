"""Seeded synthetic lens workloads (inputs only).

This module draws parameter vectors from priors, samples PSFs at pixel
centres, and adds noise.  It holds none of the likelihood's arithmetic: the
noiseless image it needs is produced by a ``render(params) -> (m_lens,
m_source)`` callable that the caller supplies (the FP64 oracle in the tests,
the library's own ``model_columns`` in the benchmark), so the same generator
serves both sides without either importing the other.

Workloads (the paper's datasets -- the 1,000 CSST-like mocks and the SLACS HST
images -- are not available; these seeded stand-ins echo their image sizes,
pixel scales, PSFs and the Sec. 3 / Table 1 model: SIE + external shear,
Sersic lens light tied to the mass centre, Sersic source):

  plain64     64x64 at 0.05"/px, 4x4 subpixels, 11x11 Gaussian PSF FWHM 0.1"
  csst100     100x100 at 0.074"/px, 4x4 subpixels, 21x21 Gaussian PSF FWHM
              0.15", noise = sky + Poisson term
  hst200      200x200 at 0.05"/px, 5x5 subpixels, 31x31 Moffat PSF
              (beta = 3, FWHM 0.1")
  ragged      many lenses, sides in {64,100,128,160,200}, PSF 11..31 px
  stream      Poisson job arrivals for the serving loop
  slacs120    multi-component light (Sec. 3.2's SLACS model: two Sersics per
              galaxy, indices fixed at 1 and 4, one centre and ellipticity
              per galaxy): 120x120 at 0.05"/px, 4x4 subpixels, 21x21 Moffat
              PSF (beta = 3, FWHM 0.1"), 4 columns
  mge120      the same image with a Gaussian expansion: 4 lens-plane and 4
              source-plane Gaussians of fixed, log-spaced widths (8 columns)
  mge32       a full Gaussian expansion on the csst100 image geometry: 20
              lens-plane Gaussians (sigma 0.03" - 2.5") and 12 source-plane
              Gaussians (0.01" - 0.6"), 32 columns

Seeds: workload k uses numpy PCG64 seeded with 2503085860 + k.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

SEED_BASE = 2503085860
NPARAM = 21
NPARAM_EPL = 22          # elliptical power-law mass: the slope gamma appended

PARAM_NAMES = [
    "theta_E", "eps1_m", "eps2_m", "x_m", "y_m", "gamma_1", "gamma_2",
    "Ie_L", "re_L", "n_L", "eps1_L", "eps2_L", "x_L", "y_L",
    "Ie_S", "re_S", "n_S", "eps1_S", "eps2_S", "x_S", "y_S",
]

# Spread used by the shrinking-Gaussian "sampler" draws around a truth.
PRIOR_WIDTH = np.array([
    0.29, 0.10, 0.10, 0.05, 0.05, 0.05, 0.05,
    0.0, 0.26, 0.87, 0.10, 0.10, 0.05, 0.05,
    0.0, 0.26, 0.87, 0.10, 0.10, 0.15, 0.15,
])
PRIOR_WIDTH_EPL = np.append(PRIOR_WIDTH, 0.23)   # gamma ~ U[1.6, 2.4]


@dataclass
class WorkloadSpec:
    name: str
    ny: int
    nx: int
    pixel_scale: float
    sub: int
    psf_size: int
    psf_kind: str          # "gaussian" | "moffat"
    psf_fwhm_arcsec: float
    batch: int
    noise_kind: str        # "sky" | "sky+poisson"
    moffat_beta: float = 3.0
    seed_offset: int = 0
    mass: str = "sie"      # "sie" | "epl"
    mask: tuple | None = None   # ("annulus", r_in, r_out) arcsec about the image centre


WORKLOADS = {
    "plain64": WorkloadSpec("plain64", 64, 64, 0.05, 4, 11, "gaussian", 0.10,
                            256, "sky", seed_offset=1),
    "csst100": WorkloadSpec("csst100", 100, 100, 0.074, 4, 21, "gaussian", 0.15,
                            4096, "sky+poisson", seed_offset=2),
    "hst200": WorkloadSpec("hst200", 200, 200, 0.05, 5, 31, "moffat", 0.10,
                           2048, "sky+poisson", seed_offset=3),
    # csst100 with the elliptical power-law mass of Eq. 12 (slope free)
    "csst100_epl": WorkloadSpec("csst100_epl", 100, 100, 0.074, 4, 21, "gaussian", 0.15,
                                4096, "sky+poisson", seed_offset=6, mass="epl"),
    # csst100 fitted only in an annulus around the Einstein ring (the paper's
    # fitting regions, Appendix A): pixels outside 0.3" - 2.2" are masked
    "csst100_mask": WorkloadSpec("csst100_mask", 100, 100, 0.074, 4, 21, "gaussian", 0.15,
                                 4096, "sky+poisson", seed_offset=2,
                                 mask=("annulus", 0.3, 2.2)),
}


def annulus_mask(ny, nx, pixel_scale, r_in, r_out, x0=None, y0=None) -> np.ndarray:
    """Boolean [ny, nx]: True where the pixel centre lies at r_in <= r <=
    r_out arcsec from the origin (the pixels fitted)."""
    x0 = centred_origin(nx, pixel_scale) if x0 is None else x0
    y0 = centred_origin(ny, pixel_scale) if y0 is None else y0
    x = x0 + pixel_scale * np.arange(nx)
    y = y0 + pixel_scale * np.arange(ny)
    r = np.hypot(x[None, :], y[:, None])
    return (r >= r_in) & (r <= r_out)


def apply_mask(lens, keep: np.ndarray):
    """Mask every pixel outside `keep` by an infinite noise sigma (the
    library's and the oracle's masking rule)."""
    noise = lens.noise.copy()
    noise[~keep] = np.float32(np.inf)
    lens.noise = noise
    return lens


# ------------------------------------------------------------------ PSFs
def gaussian_psf(size: int, fwhm_px: float) -> np.ndarray:
    """Circular Gaussian sampled at pixel centres, unit sum, float32."""
    if size % 2 != 1:
        raise ValueError("PSF size must be odd")
    sig = fwhm_px / (2.0 * math.sqrt(2.0 * math.log(2.0)))
    r = np.arange(size) - (size - 1) / 2
    g = np.exp(-0.5 * (r / sig) ** 2)
    k = np.outer(g, g)
    return (k / k.sum()).astype(np.float32)


def moffat_psf(size: int, fwhm_px: float, beta: float) -> np.ndarray:
    """Circular Moffat sampled at pixel centres, unit sum, float32."""
    if size % 2 != 1:
        raise ValueError("PSF size must be odd")
    alpha = fwhm_px / (2.0 * math.sqrt(2.0 ** (1.0 / beta) - 1.0))
    r = np.arange(size) - (size - 1) / 2
    rr = r[:, None] ** 2 + r[None, :] ** 2
    k = (1.0 + rr / alpha ** 2) ** (-beta)
    return (k / k.sum()).astype(np.float32)


def make_psf(spec: WorkloadSpec) -> np.ndarray:
    fwhm_px = spec.psf_fwhm_arcsec / spec.pixel_scale
    if spec.psf_kind == "gaussian":
        return gaussian_psf(spec.psf_size, fwhm_px)
    return moffat_psf(spec.psf_size, fwhm_px, spec.moffat_beta)


# ---------------------------------------------------------------- priors
# ------------------------------------------------- multi-component light
# A component list is plain data (type, plane, free scale / index, fixed
# values); each side converts it to its own form.
SLACS_COMPS = [
    dict(type="sersic", plane="lens", index=1.0),
    dict(type="sersic", plane="lens", index=4.0),
    dict(type="sersic", plane="source", index=1.0),
    dict(type="sersic", plane="source", index=4.0),
]
MGE_COMPS = (
    [dict(type="gauss", plane="lens", free_scale=False, scale=float(s))
     for s in np.geomspace(0.05, 1.2, 4)]
    + [dict(type="gauss", plane="source", free_scale=False, scale=float(s))
       for s in np.geomspace(0.02, 0.4, 4)])
MGE32_COMPS = (
    [dict(type="gauss", plane="lens", free_scale=False, scale=float(s))
     for s in np.geomspace(0.03, 2.5, 20)]
    + [dict(type="gauss", plane="source", free_scale=False, scale=float(s))
       for s in np.geomspace(0.01, 0.6, 12)])
MULTI_HEAD = 15


@dataclass
class MultiSpec:
    name: str
    ny: int
    nx: int
    pixel_scale: float
    sub: int
    psf_size: int
    psf_kind: str
    psf_fwhm_arcsec: float
    batch: int
    comps: list
    moffat_beta: float = 3.0
    seed_offset: int = 0
    mass: str = "sie"


MULTI_WORKLOADS = {
    "slacs120": MultiSpec("slacs120", 120, 120, 0.05, 4, 21, "moffat", 0.10, 2048,
                          SLACS_COMPS, seed_offset=7),
    "mge120": MultiSpec("mge120", 120, 120, 0.05, 4, 21, "moffat", 0.10, 2048,
                        MGE_COMPS, seed_offset=8),
    "mge32": MultiSpec("mge32", 100, 100, 0.074, 4, 21, "gaussian", 0.15, 1024,
                       MGE32_COMPS, seed_offset=9),
}


def multi_nparam(comps, mass: str = "sie") -> int:
    n = MULTI_HEAD
    for c in comps:
        n += 1 if c.get("free_scale", True) else 0
        n += 1 if c["type"] == "sersic" and c.get("free_index", False) else 0
    return n + (1 if mass == "epl" else 0)


def draw_prior_multi(rng: np.random.Generator, n: int, comps, mass: str = "sie") -> np.ndarray:
    """n multi-component vectors, float32 [n, multi_nparam]: mass, shear and
    the two planes' ellipticities and centres from the priors of draw_prior
    (lens-light centre = mass centre); each free Sersic r_e ~ U[0.1, 1]",
    free index ~ U[1, 4], free Gaussian sigma ~ U[0.05, 0.5]"; EPL slope
    ~ U[1.6, 2.4] last."""
    p = np.zeros((n, multi_nparam(comps, mass)), dtype=np.float64)
    p[:, 0] = rng.uniform(0.5, 1.5, n)
    p[:, 1], p[:, 2] = _eps(rng, n)
    p[:, 3] = rng.normal(0.0, 0.05, n)
    p[:, 4] = rng.normal(0.0, 0.05, n)
    p[:, 5] = rng.normal(0.0, 0.05, n)
    p[:, 6] = rng.normal(0.0, 0.05, n)
    p[:, 7], p[:, 8] = _eps(rng, n)
    p[:, 9] = p[:, 3]
    p[:, 10] = p[:, 4]
    p[:, 11], p[:, 12] = _eps(rng, n)
    rad = 0.3 * np.sqrt(rng.uniform(0.0, 1.0, n))
    ang = rng.uniform(0.0, 2 * math.pi, n)
    p[:, 13] = rad * np.cos(ang)
    p[:, 14] = rad * np.sin(ang)
    k = MULTI_HEAD
    for c in comps:
        if c.get("free_scale", True):
            p[:, k] = (rng.uniform(0.1, 1.0, n) if c["type"] == "sersic"
                       else rng.uniform(0.05, 0.5, n))
            k += 1
        if c["type"] == "sersic" and c.get("free_index", False):
            p[:, k] = rng.uniform(1.0, 4.0, n)
            k += 1
    if mass == "epl":
        p[:, k] = rng.uniform(1.6, 2.4, n)
    return p.astype(np.float32)


def shrinking_draws_multi(rng, truth: np.ndarray, n: int, comps, lo_frac: float = 0.01):
    """As shrinking_draws for a multi-component truth: head widths as the
    prior's, 0.2 for free scales (clipped to [0.03, 3]), 0.87 for free
    indices (clipped to [0.3, 8])."""
    frac = np.geomspace(1.0, lo_frac, n)
    head = np.array([0.29, 0.10, 0.10, 0.05, 0.05, 0.05, 0.05,
                     0.10, 0.10, 0.05, 0.05, 0.10, 0.10, 0.15, 0.15])
    width, kinds = list(head), []
    for c in comps:
        if c.get("free_scale", True):
            width.append(0.2)
            kinds.append("scale")
        if c["type"] == "sersic" and c.get("free_index", False):
            width.append(0.87)
            kinds.append("index")
    if truth.shape[0] > len(width):
        width.append(0.23)
        kinds.append("slope")
    width = np.array(width)
    p = truth[None, :].astype(np.float64) + rng.normal(size=(n, truth.shape[0])) * (
        frac[:, None] * width[None, :])
    p[:, 0] = np.clip(p[:, 0], 0.05, 3.5)
    for a, b in ((1, 2), (7, 8), (11, 12)):
        e = np.hypot(p[:, a], p[:, b])
        s = np.where(e > 0.6, 0.6 / np.maximum(e, 1e-30), 1.0)
        p[:, a] *= s
        p[:, b] *= s
    p[:, 9] = p[:, 3]
    p[:, 10] = p[:, 4]
    for k, kind in enumerate(kinds):
        j = MULTI_HEAD + k
        if kind == "scale":
            p[:, j] = np.clip(p[:, j], 0.03, 3.0)
        elif kind == "index":
            p[:, j] = np.clip(p[:, j], 0.3, 8.0)
        else:
            p[:, j] = np.clip(p[:, j], 1.2, 2.8)
    return p.astype(np.float32)


def synth_multi_lens(rng, ny, nx, pixel_scale, sub, psf, render, comps, peak_snr=50.0,
                     sky_sigma=1.0, truth=None, mass: str = "sie") -> SynthLens:
    """One multi-component lens: truth from draw_prior_multi, blurred unit
    columns from render(truth) ([nc, ny, nx]); each plane's columns get
    amplitudes with random shares (U[0.2, 1], renormalised) scaled so that
    the plane's brightest blurred pixel is peak_snr * sky_sigma; noise
    sigma^2 = sky^2 + max(model, 0)/g as in synth_lens.  truth carries the
    amplitudes in extra["amps"]."""
    if truth is None:
        truth = draw_prior_multi(rng, 1, comps, mass)[0]
    truth = truth.astype(np.float32).copy()
    cols = np.asarray(render(truth), dtype=np.float64)
    amps = np.zeros(len(comps))
    for plane in ("lens", "source"):
        idx = [k for k, c in enumerate(comps) if c["plane"] == plane]
        if not idx:
            continue
        share = rng.uniform(0.2, 1.0, len(idx))
        img = np.tensordot(share, cols[idx], axes=1)
        amps[idx] = share * peak_snr * sky_sigma / max(img.max(), 1e-30)
    model = np.tensordot(amps, cols, axes=1)
    g = peak_snr * sky_sigma / sky_sigma ** 2
    sigma = np.sqrt(sky_sigma ** 2 + np.maximum(model, 0.0) / g)
    data = model + rng.normal(size=model.shape) * sigma
    return SynthLens(ny, nx, f32(pixel_scale), sub, psf.astype(np.float32),
                     data.astype(np.float32), sigma.astype(np.float32), truth,
                     centred_origin(nx, pixel_scale), centred_origin(ny, pixel_scale),
                     extra={"amps": amps, "comps": comps})


def multi_workload(name: str, render_factory, batch: int | None = None):
    """(lens, params [B, nparam]) of a named multi-component workload;
    render_factory(pixel_scale, sub, psf, ny, nx, comps) -> render."""
    spec = MULTI_WORKLOADS[name]
    rng = np.random.Generator(np.random.PCG64(SEED_BASE + spec.seed_offset))
    fwhm_px = spec.psf_fwhm_arcsec / spec.pixel_scale
    psf = (gaussian_psf(spec.psf_size, fwhm_px) if spec.psf_kind == "gaussian"
           else moffat_psf(spec.psf_size, fwhm_px, spec.moffat_beta))
    render = render_factory(f32(spec.pixel_scale), spec.sub, psf, spec.ny, spec.nx, spec.comps)
    lens = synth_multi_lens(rng, spec.ny, spec.nx, spec.pixel_scale, spec.sub, psf, render,
                            spec.comps, mass=spec.mass)
    B = spec.batch if batch is None else batch
    params = draw_prior_multi(rng, B, spec.comps, spec.mass)
    return lens, params


def _eps(rng, n, qlo=0.5, qhi=1.0):
    """Ellipticity components for q ~ U[qlo, qhi], position angle ~ U[0, pi)
    (change of variables to the paper's ellipticity parametrisation)."""
    q = rng.uniform(qlo, qhi, n)
    pa = rng.uniform(0.0, math.pi, n)
    e = (1.0 - q) / (1.0 + q)
    return e * np.cos(2 * pa), e * np.sin(2 * pa)


def draw_prior(rng: np.random.Generator, n: int, mass: str = "sie") -> np.ndarray:
    """n parameter vectors from the workload priors, float32 [n, 21]:
    theta_E ~ U[0.5,1.5]"; mass q ~ U[0.5,1], PA ~ U[0,pi); centre ~ N(0,0.05");
    gamma_1,2 ~ N(0,0.05); lens and source Sersic n ~ U[1,4], r_e ~ U[0.1,1]",
    q ~ U[0.5,1], PA ~ U[0,pi); lens-light centre = mass centre (Table 1);
    source centre uniform in a disc of radius 0.3"; I_e slots = 1.
    mass "epl": [n, 22] with the mass slope gamma ~ U[1.6, 2.4] last (drawn
    after the other entries, so the first 21 columns are the SIE draws)."""
    p = np.zeros((n, NPARAM), dtype=np.float64)
    p[:, 0] = rng.uniform(0.5, 1.5, n)
    p[:, 1], p[:, 2] = _eps(rng, n)
    p[:, 3] = rng.normal(0.0, 0.05, n)
    p[:, 4] = rng.normal(0.0, 0.05, n)
    p[:, 5] = rng.normal(0.0, 0.05, n)
    p[:, 6] = rng.normal(0.0, 0.05, n)
    p[:, 7] = 1.0
    p[:, 8] = rng.uniform(0.1, 1.0, n)
    p[:, 9] = rng.uniform(1.0, 4.0, n)
    p[:, 10], p[:, 11] = _eps(rng, n)
    p[:, 12] = p[:, 3]
    p[:, 13] = p[:, 4]
    p[:, 14] = 1.0
    p[:, 15] = rng.uniform(0.1, 1.0, n)
    p[:, 16] = rng.uniform(1.0, 4.0, n)
    p[:, 17], p[:, 18] = _eps(rng, n)
    rad = 0.3 * np.sqrt(rng.uniform(0.0, 1.0, n))
    ang = rng.uniform(0.0, 2 * math.pi, n)
    p[:, 19] = rad * np.cos(ang)
    p[:, 20] = rad * np.sin(ang)
    if mass == "epl":
        p = np.concatenate([p, rng.uniform(1.6, 2.4, (n, 1))], axis=1)
    return p.astype(np.float32)


def shrinking_draws(rng, truth: np.ndarray, n: int, lo_frac: float = 0.01):
    """n vectors ~ N(truth, sigma_j), sigma_j shrinking geometrically from the
    prior width to lo_frac of it (a stand-in for a sampler converging);
    entries clipped into the valid region.  float32 [n, 21] (or [n, 22] for
    an EPL truth, gamma clipped to [1.2, 2.8])."""
    frac = np.geomspace(1.0, lo_frac, n)
    npar = truth.shape[0]
    width = PRIOR_WIDTH_EPL if npar == NPARAM_EPL else PRIOR_WIDTH
    p = truth[None, :].astype(np.float64) + rng.normal(size=(n, npar)) * (
        frac[:, None] * width[None, :])
    if npar == NPARAM_EPL:
        p[:, 21] = np.clip(p[:, 21], 1.2, 2.8)
    p[:, 0] = np.clip(p[:, 0], 0.05, 3.5)
    for a, b in ((1, 2), (10, 11), (17, 18)):
        e = np.hypot(p[:, a], p[:, b])
        s = np.where(e > 0.6, 0.6 / np.maximum(e, 1e-30), 1.0)
        p[:, a] *= s
        p[:, b] *= s
    p[:, 8] = np.clip(p[:, 8], 0.05, 4.0)
    p[:, 15] = np.clip(p[:, 15], 0.05, 2.0)
    p[:, 9] = np.clip(p[:, 9], 0.3, 8.0)
    p[:, 16] = np.clip(p[:, 16], 0.3, 8.0)
    p[:, 12] = p[:, 3]
    p[:, 13] = p[:, 4]
    return p.astype(np.float32)


# ----------------------------------------------------------------- lenses
@dataclass
class SynthLens:
    ny: int
    nx: int
    pixel_scale: float
    sub: int
    psf: np.ndarray          # float32 [k, k], unit sum
    data: np.ndarray         # float32 [ny, nx]
    noise: np.ndarray        # float32 [ny, nx], sigma per pixel
    truth: np.ndarray        # float32 [21]; I_e slots = true amplitudes
    x0: float = 0.0
    y0: float = 0.0
    extra: dict = field(default_factory=dict)


def f32(v: float) -> float:
    """The float32 value nearest v, as a Python float (the library's grid
    geometry is float32, so inputs are made exactly representable)."""
    return float(np.float32(v))


def centred_origin(n: int, pixel_scale: float) -> float:
    """Coordinate of pixel 0's centre for an image centred on the origin
    (float32-representable)."""
    return f32(-(n - 1) * f32(pixel_scale) / 2.0)


def synth_lens(rng, ny, nx, pixel_scale, sub, psf, render, noise_kind="sky",
               peak_snr=50.0, sky_sigma=1.0, truth=None, mass: str = "sie") -> SynthLens:
    """One lens: truth from the priors, noiseless image from render(truth)
    (blurred unit-amplitude lens and source columns), amplitudes set so that
    each component's brightest blurred pixel is peak_snr * sky_sigma, then
    Gaussian noise.  noise_kind "sky": sigma = sky_sigma; "sky+poisson":
    sigma^2 = sky^2 + max(model,0)/g with g chosen so the Poisson term equals
    sky^2 at the source peak."""
    if truth is None:
        truth = draw_prior(rng, 1, mass)[0]
    truth = truth.astype(np.float32).copy()
    ml, ms = render(truth)
    ml = np.asarray(ml, dtype=np.float64)
    ms = np.asarray(ms, dtype=np.float64)
    al = peak_snr * sky_sigma / max(ml.max(), 1e-30)
    as_ = peak_snr * sky_sigma / max(ms.max(), 1e-30)
    truth[7] = al
    truth[14] = as_
    model = al * ml + as_ * ms
    if noise_kind == "sky":
        var = np.full_like(model, sky_sigma ** 2)
    else:
        g = peak_snr * sky_sigma / sky_sigma ** 2
        var = sky_sigma ** 2 + np.maximum(model, 0.0) / g
    sigma = np.sqrt(var)
    data = model + rng.normal(size=model.shape) * sigma
    return SynthLens(ny, nx, f32(pixel_scale), sub, psf.astype(np.float32),
                     data.astype(np.float32), sigma.astype(np.float32), truth,
                     centred_origin(nx, pixel_scale),
                     centred_origin(ny, pixel_scale))


def workload(name: str, render_factory, batch: int | None = None):
    """(lens, params[B, 21] or [B, 22] for an EPL workload) for a named
    single-lens workload.  render_factory(pixel_scale, sub, psf, ny, nx
    [, mass=...]) -> render(params)."""
    spec = WORKLOADS[name]
    rng = np.random.Generator(np.random.PCG64(SEED_BASE + spec.seed_offset))
    psf = make_psf(spec)
    kw = {} if spec.mass == "sie" else {"mass": spec.mass}
    render = render_factory(f32(spec.pixel_scale), spec.sub, psf, spec.ny, spec.nx, **kw)
    lens = synth_lens(rng, spec.ny, spec.nx, spec.pixel_scale, spec.sub, psf,
                      render, spec.noise_kind, mass=spec.mass)
    if spec.mask is not None:
        kind, r_in, r_out = spec.mask
        apply_mask(lens, annulus_mask(spec.ny, spec.nx, f32(spec.pixel_scale), r_in, r_out,
                                      lens.x0, lens.y0))
    B = spec.batch if batch is None else batch
    params = draw_prior(rng, B, spec.mass)
    return lens, params


# ----------------------------------------------------------- ragged / stream
RAGGED_SIDES = (64, 100, 128, 160, 200)


def ragged_specs(n_lenses: int, seed_offset: int = 4):
    """Image sides and PSF sizes of a ragged multi-lens batch (no rendering):
    side ~ U{64,100,128,160,200}, PSF size ~ U{11,13,...,31}, Gaussian PSF of
    FWHM = size/7 px, 0.074"/px, 4x4 subpixels."""
    rng = np.random.Generator(np.random.PCG64(SEED_BASE + seed_offset))
    sides = rng.choice(RAGGED_SIDES, size=n_lenses)
    ks = 11 + 2 * rng.integers(0, 11, size=n_lenses)
    return rng, [(int(s), int(k)) for s, k in zip(sides, ks)]


def ragged_workload(n_lenses: int, per_lens: int, render_factory,
                    pixel_scale=0.074, sub=4, seed_offset: int = 4):
    """List of (lens, params[per_lens, 21]) for a ragged batch."""
    rng, specs = ragged_specs(n_lenses, seed_offset)
    out = []
    for side, k in specs:
        psf = gaussian_psf(k, k / 7.0)
        render = render_factory(f32(pixel_scale), sub, psf, side, side)
        lens = synth_lens(rng, side, side, pixel_scale, sub, psf, render,
                          "sky+poisson")
        params = shrinking_draws(rng, lens.truth, per_lens)
        out.append((lens, params))
    return out


def request_stream(n_jobs: int, rate_hz: float = 20.0, iters: int = 300,
                   batch_lo: int = 500, batch_hi: int = 5000,
                   side_lo: int = 64, side_hi: int = 200, seed_offset: int = 5):
    """Job descriptors of a Poisson request stream: arrival time (s), image
    side, PSF size, and the batch size of each of its sampler iterations."""
    rng = np.random.Generator(np.random.PCG64(SEED_BASE + seed_offset))
    t = np.cumsum(rng.exponential(1.0 / rate_hz, n_jobs))
    jobs = []
    for j in range(n_jobs):
        side = int(rng.integers(side_lo, side_hi + 1))
        k = int(11 + 2 * rng.integers(0, 11))
        batches = rng.integers(batch_lo, batch_hi + 1, size=iters)
        jobs.append({"arrival": float(t[j]), "side": side, "psf": k,
                     "batches": [int(b) for b in batches],
                     "seed": int(rng.integers(0, 2 ** 31))})
    return jobs
