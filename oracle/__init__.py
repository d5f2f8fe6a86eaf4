"""FP64 CPU oracle for the batched lens log-likelihood -- TEST INFRASTRUCTURE.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline /
reference leg may import this package.  The product library never loads it,
and it shares no code with the CUDA path.

The arithmetic lives in ``tll_oracle.c`` (plain C, FP64, compiled with gcc
-O2 and OpenMP across parameter vectors only).  This module compiles it on
first use and wraps its functions with ctypes; every function cites the
section / equation of arXiv:2503.08586 it follows in the C source.

Parity status per function: every oracle function is pinned by a
``-m "not gpu"`` test in ``tests/test_oracle_pins.py`` against a closed form,
a library routine, brute force or an independent quadrature.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import sys

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "tll_oracle.c")
_LIB = os.path.join(_HERE, "_liboracle.so")
NPARAM = 21
NPARAM_EPL = 22
MASS = {"sie": 0, "epl": 1}

_lib = None


def build(force: bool = False) -> str:
    """Compile tll_oracle.c into oracle/_liboracle.so (gcc, -O2, OpenMP)."""
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    base = ["gcc", "-std=c11", "-D_GNU_SOURCE", "-O2", "-ffp-contract=off", "-fPIC", "-shared",
            "-o", _LIB + ".tmp", _SRC, "-lm"]
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True,
                       capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True)
    os.replace(_LIB + ".tmp", _LIB)
    return _LIB


class _Lens(ctypes.Structure):
    _fields_ = [("ny", ctypes.c_int), ("nx", ctypes.c_int),
                ("sub", ctypes.c_int), ("k", ctypes.c_int),
                ("dpix", ctypes.c_double), ("x0", ctypes.c_double),
                ("y0", ctypes.c_double),
                ("data", ctypes.POINTER(ctypes.c_double)),
                ("sigma", ctypes.POINTER(ctypes.c_double)),
                ("psf", ctypes.POINTER(ctypes.c_double)),
                ("mass", ctypes.c_int)]


class _Comp(ctypes.Structure):
    _fields_ = [("type", ctypes.c_int), ("plane", ctypes.c_int),
                ("flags", ctypes.c_int), ("scale", ctypes.c_double),
                ("index", ctypes.c_double)]


def _load():
    global _lib
    if _lib is not None:
        return _lib
    lib = ctypes.CDLL(build())
    d, i, pd = ctypes.c_double, ctypes.c_int, ctypes.POINTER(ctypes.c_double)
    pf, pi = ctypes.POINTER(ctypes.c_float), ctypes.POINTER(ctypes.c_int)
    pu32 = ctypes.POINTER(ctypes.c_uint32)
    sig = {
        "ora_ellipse": (i, [d, d, pd, pd]),
        "ora_gammainc_P": (d, [d, d]),
        "ora_sersic_bn": (d, [d]),
        "ora_sersic": (d, [d] * 9),
        "ora_sie_alpha": (None, [d] * 7 + [pd, pd]),
        "ora_epl_alpha": (None, [d] * 8 + [pd, pd]),
        "ora_shear_potential": (d, [d] * 4),
        "ora_shear_alpha": (None, [d] * 4 + [pd, pd]),
        "ora_trace_point": (i, [pd, d, d, pd, pd]),
        "ora_convolve": (None, [pd, i, i, pd, i, pd]),
        "ora_psf_normalise": (i, [pd, i, pd]),
        "ora_nnls2": (None, [pd, pd, pd, pd, i, pd]),
        "ora_chi2": (d, [pd, pd, pd, pd, i, d, d]),
        "ora_loglike_full": (d, [ctypes.POINTER(_Lens), pd, i, pd, pd, pd, pd]),
        "ora_unblurred_columns": (i, [ctypes.POINTER(_Lens), pd, pd, pd]),
        "ora_loglike_batch": (None, [ctypes.POINTER(_Lens), pd, i, i, pd, i]),
        "ora_max_threads": (i, []),
        "ora_gauss": (d, [d] * 7),
        "ora_multi_nparam": (i, [ctypes.POINTER(_Comp), i, i]),
        "ora_chol_solve": (i, [pd, pd, i, pd]),
        "ora_fnnls": (i, [pd, pd, i, pd]),
        "ora_loglike_multi": (d, [ctypes.POINTER(_Lens), ctypes.POINTER(_Comp), i, pd,
                                  pd, pd, pd]),
        "ora_multi_unblurred": (i, [ctypes.POINTER(_Lens), ctypes.POINTER(_Comp), i,
                                    pd, pd]),
        "ora_loglike_multi_batch": (None, [ctypes.POINTER(_Lens), ctypes.POINTER(_Comp),
                                           i, pd, i, pd, i]),
        "ora_philox4x32_10": (None, [pu32, pu32, pu32]),
        "ora_stretch_propose": (None, [pf, i, i, i, ctypes.c_longlong, ctypes.c_uint64, d,
                                       pf, pd, pi]),
        "ora_stretch_accept": (i, [pf, pd, i, i, i, ctypes.c_longlong, ctypes.c_uint64, i,
                                   pf, pd, pd, pf, pf, pi]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


# --------------------------------------------------------------- pieces
def ellipse(e1: float, e2: float):
    """Eq. (11) inverted: (q, phi), or None for |eps| >= 1."""
    q, phi = ctypes.c_double(), ctypes.c_double()
    if _load().ora_ellipse(e1, e2, ctypes.byref(q), ctypes.byref(phi)):
        return None
    return q.value, phi.value


def gammainc_P(a: float, x: float) -> float:
    """Regularised lower incomplete gamma (used by Eq. 9)."""
    return _load().ora_gammainc_P(a, x)


def sersic_bn(n: float) -> float:
    """b_n, the root of Eq. (9)."""
    return _load().ora_sersic_bn(n)


def sersic(x, y, cx, cy, q, phi, re, n, bn) -> float:
    """Unit-amplitude elliptical Sersic, Eqs. (8), (10)."""
    return _load().ora_sersic(x, y, cx, cy, q, phi, re, n, bn)


def sie_alpha(x, y, thE, q, phi, xc=0.0, yc=0.0):
    """SIE deflection (Eq. 12 with gamma = 2, Kormann closed form)."""
    ax, ay = ctypes.c_double(), ctypes.c_double()
    _load().ora_sie_alpha(x, y, thE, q, phi, xc, yc, ctypes.byref(ax),
                          ctypes.byref(ay))
    return ax.value, ay.value


def epl_alpha(x, y, thE, q, phi, gamma, xc=0.0, yc=0.0):
    """EPL deflection (Eq. 12, any slope; Tessore & Metcalf closed form)."""
    ax, ay = ctypes.c_double(), ctypes.c_double()
    _load().ora_epl_alpha(x, y, thE, q, phi, xc, yc, gamma, ctypes.byref(ax),
                          ctypes.byref(ay))
    return ax.value, ay.value


def shear_potential(x, y, g1, g2) -> float:
    return _load().ora_shear_potential(x, y, g1, g2)


def shear_alpha(x, y, g1, g2):
    ax, ay = ctypes.c_double(), ctypes.c_double()
    _load().ora_shear_alpha(x, y, g1, g2, ctypes.byref(ax), ctypes.byref(ay))
    return ax.value, ay.value


def trace_point(params, x, y):
    """Lens equation, Eq. (1), at one image-plane point; None if invalid."""
    p = _f64(params)
    bx, by = ctypes.c_double(), ctypes.c_double()
    if _load().ora_trace_point(_p(p), x, y, ctypes.byref(bx), ctypes.byref(by)):
        return None
    return bx.value, by.value


def convolve(img, psf_normalised) -> np.ndarray:
    """Eq. (3), zero-padded, same size; the PSF must already be unit-sum."""
    img = _f64(img)
    psf = _f64(psf_normalised)
    out = np.zeros_like(img)
    _load().ora_convolve(_p(img), img.shape[0], img.shape[1], _p(psf),
                         psf.shape[0], _p(out))
    return out


def psf_normalise(psf) -> np.ndarray:
    psf = _f64(psf)
    out = np.zeros_like(psf)
    if _load().ora_psf_normalise(_p(psf), psf.shape[0], _p(out)):
        raise ValueError("PSF sum is not > 0")
    return out


def nnls2(ml, ms, d, w):
    ml, ms, d, w = _f64(ml), _f64(ms), _f64(d), _f64(w)
    s = np.zeros(2)
    _load().ora_nnls2(_p(ml), _p(ms), _p(d), _p(w), ml.size, _p(s))
    return s


def chi2(ml, ms, d, w, sl, ss) -> float:
    ml, ms, d, w = _f64(ml), _f64(ms), _f64(d), _f64(w)
    return _load().ora_chi2(_p(ml), _p(ms), _p(d), _p(w), ml.size, sl, ss)


# --------------------------------------------------------------- lenses
class Lens:
    """A lens as the oracle sees it: data, noise map, raw PSF and the grid."""

    def __init__(self, data, noise, psf, pixel_scale, sub, x0=None, y0=None,
                 mass: str = "sie"):
        self.data = _f64(data)
        self.noise = _f64(noise)
        self.psf = _f64(psf)
        self.ny, self.nx = self.data.shape
        self.k = self.psf.shape[0]
        self.dpix = float(pixel_scale)
        self.sub = int(sub)
        self.x0 = -(self.nx - 1) * self.dpix / 2 if x0 is None else float(x0)
        self.y0 = -(self.ny - 1) * self.dpix / 2 if y0 is None else float(y0)
        self.mass = mass
        self.nparam = NPARAM_EPL if mass == "epl" else NPARAM
        self._s = _Lens(self.ny, self.nx, self.sub, self.k, self.dpix, self.x0,
                        self.y0, _p(self.data), _p(self.noise), _p(self.psf),
                        MASS[mass])

    def loglike(self, params, mode: int = 0) -> float:
        p = _f64(params)
        return _load().ora_loglike_full(ctypes.byref(self._s), _p(p), mode,
                                        None, None, None, None)

    def model(self, params, mode: int = 0):
        """(log L, blurred lens column, blurred source column, model, amps)."""
        p = _f64(params)
        n = self.ny * self.nx
        ml, ms, mod, amps = np.zeros(n), np.zeros(n), np.zeros(n), np.zeros(2)
        ll = _load().ora_loglike_full(ctypes.byref(self._s), _p(p), mode,
                                      _p(ml), _p(ms), _p(mod), _p(amps))
        sh = (self.ny, self.nx)
        return ll, ml.reshape(sh), ms.reshape(sh), mod.reshape(sh), amps

    def unblurred(self, params):
        """Binned unit-amplitude (lens, source) columns before the PSF."""
        p = _f64(params)
        n = self.ny * self.nx
        il, is_ = np.zeros(n), np.zeros(n)
        if _load().ora_unblurred_columns(ctypes.byref(self._s), _p(p), _p(il),
                                         _p(is_)):
            return None
        return il.reshape(self.ny, self.nx), is_.reshape(self.ny, self.nx)

    def loglike_batch(self, params, mode: int = 0, nthreads: int = 0):
        p = _f64(params).reshape(-1, self.nparam)
        out = np.zeros(p.shape[0])
        _load().ora_loglike_batch(ctypes.byref(self._s), _p(p), p.shape[0],
                                  mode, _p(out), nthreads)
        return out


# ------------------------------------------------- multi-component light
# Sec. 2.3 (Eq. 7): N_l lens-light and N_s source profiles, one column each.
COMP = {"sersic": 0, "gauss": 1}
PLANE = {"lens": 0, "source": 1}
FREE_SCALE = 1
FREE_INDEX = 2
MULTI_HEAD = 15    # mass (7), lens-light geometry (4), source geometry (4)


def gauss(x, y, cx, cy, q, phi, sigma) -> float:
    """Unit-central-intensity elliptical Gaussian (reading R13)."""
    return _load().ora_gauss(x, y, cx, cy, q, phi, sigma)


def fnnls(A, b):
    """FNNLS (Bro & de Jong 1997) on A = Z^T Z, b = Z^T y: (x, steps)."""
    A = _f64(A)
    b = _f64(b)
    n = b.size
    x = np.zeros(n)
    steps = _load().ora_fnnls(_p(A), _p(b), n, _p(x))
    return x, steps


def chol_solve(G, r):
    G, r = _f64(G), _f64(r)
    z = np.zeros(r.size)
    if _load().ora_chol_solve(_p(G), _p(r), r.size, _p(z)):
        return None
    return z


def comp_array(comps):
    """comps: list of dicts {type, plane, free_scale, free_index, scale, index}
    (names as in COMP / PLANE) -> a ctypes array for the C oracle."""
    arr = (_Comp * len(comps))()
    for k, c in enumerate(comps):
        flags = (FREE_SCALE if c.get("free_scale", True) else 0) | (
            FREE_INDEX if c.get("free_index", False) else 0)
        arr[k] = _Comp(COMP[c["type"]], PLANE[c["plane"]], flags,
                       float(c.get("scale", 1.0)), float(c.get("index", 1.0)))
    return arr


class MultiLens(Lens):
    """A lens with a multi-component light model (readings R13-R15)."""

    def __init__(self, data, noise, psf, pixel_scale, sub, comps, x0=None,
                 y0=None, mass: str = "sie"):
        super().__init__(data, noise, psf, pixel_scale, sub, x0, y0, mass)
        self.comps = list(comps)
        self._c = comp_array(self.comps)
        self.nc = len(self.comps)
        self.nparam = _load().ora_multi_nparam(self._c, self.nc, MASS[mass])
        if self.nparam < 0:
            raise ValueError("bad component list")

    def loglike(self, params, mode: int = 0) -> float:
        p = _f64(params)
        return _load().ora_loglike_multi(ctypes.byref(self._s), self._c, self.nc,
                                         _p(p), None, None, None)

    def model(self, params, mode: int = 0):
        """(log L, blurred columns [nc, ny, nx], model, amplitudes [nc])."""
        p = _f64(params)
        n = self.ny * self.nx
        cols, amps, mod = np.zeros(n * self.nc), np.zeros(self.nc), np.zeros(n)
        ll = _load().ora_loglike_multi(ctypes.byref(self._s), self._c, self.nc,
                                       _p(p), _p(cols), _p(amps), _p(mod))
        return (ll, cols.reshape(self.nc, self.ny, self.nx),
                mod.reshape(self.ny, self.nx), amps)

    def unblurred(self, params):
        p = _f64(params)
        cols = np.zeros(self.nc * self.ny * self.nx)
        if _load().ora_multi_unblurred(ctypes.byref(self._s), self._c, self.nc,
                                       _p(p), _p(cols)):
            return None
        return cols.reshape(self.nc, self.ny, self.nx)

    def loglike_batch(self, params, mode: int = 0, nthreads: int = 0):
        p = _f64(params).reshape(-1, self.nparam)
        out = np.zeros(p.shape[0])
        _load().ora_loglike_multi_batch(ctypes.byref(self._s), self._c, self.nc,
                                        _p(p), p.shape[0], _p(out), nthreads)
        return out


def multi_columns_renderer(pixel_scale, sub, psf, ny, nx, comps, mass: str = "sie"):
    """render(params) -> blurred unit columns [nc, ny, nx] of a
    multi-component model (to synthesise data images in the tests)."""
    dummy = np.zeros((ny, nx))
    lens = MultiLens(dummy, np.ones((ny, nx)), psf, pixel_scale, sub, comps, mass=mass)

    def render(params):
        _, cols, _, _ = lens.model(params)
        return cols

    return render


# ------------------------------------------------------- sampler loop
def philox4x32_10(ctr, key):
    """Philox4x32-10 (Salmon et al. 2011): four uint32 outputs."""
    c = (ctypes.c_uint32 * 4)(*[int(v) & 0xffffffff for v in ctr])
    k = (ctypes.c_uint32 * 2)(*[int(v) & 0xffffffff for v in key])
    o = (ctypes.c_uint32 * 4)()
    _load().ora_philox4x32_10(c, k, o)
    return [int(v) for v in o]


def _fp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_float))


def _ip(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int))


def stretch_propose(x, h, step, seed, a=2.0):
    """Half h's proposals of the stretch move: (Y [W/2, P] float32, z, j)."""
    x = np.ascontiguousarray(x, np.float32)
    W, P = x.shape
    Y = np.zeros((W // 2, P), np.float32)
    z = np.zeros(W // 2)
    j = np.zeros(W // 2, np.int32)
    _load().ora_stretch_propose(_fp(x), W, P, h, step, seed, a, _fp(Y), _p(z), _ip(j))
    return Y, z, j


def stretch_accept(x, lp, h, step, seed, ndim, Y, z, lpY, lo, hi):
    """Accept / reject half h in place (x float32 [W, P], lp float64 [W]);
    returns the accepted flags [W/2]."""
    W, P = x.shape
    assert x.dtype == np.float32 and x.flags.c_contiguous and lp.dtype == np.float64
    Y = np.ascontiguousarray(Y, np.float32)
    z, lpY = _f64(z), _f64(lpY)
    lo = np.ascontiguousarray(lo, np.float32)
    hi = np.ascontiguousarray(hi, np.float32)
    acc = np.zeros(W // 2, np.int32)
    _load().ora_stretch_accept(_fp(x), _p(lp), W, P, h, step, seed, ndim, _fp(Y), _p(z),
                               _p(lpY), _fp(lo), _fp(hi), _ip(acc))
    return acc


def stretch_run(x0, logp, nsteps, seed, lo, hi, ndim=None, a=2.0, step0=0):
    """The stretch-move loop with a Python log-density logp(Y [n, P]) -> [n]:
    returns (chain [nsteps, W, P], lp chain [nsteps, W], acceptance rate)."""
    x = np.ascontiguousarray(x0, np.float32).copy()
    W, P = x.shape
    lo = np.asarray(lo, np.float32)
    hi = np.asarray(hi, np.float32)
    ndim = int(np.sum(lo < hi)) if ndim is None else ndim
    lp = np.asarray(logp(x), np.float64).copy()
    chain = np.zeros((nsteps, W, P), np.float32)
    lpc = np.zeros((nsteps, W))
    nacc = 0
    for s in range(nsteps):
        for h in (0, 1):
            Y, z, _ = stretch_propose(x, h, step0 + s, seed, a)
            nacc += int(stretch_accept(x, lp, h, step0 + s, seed, ndim, Y, z, logp(Y), lo,
                                       hi).sum())
        chain[s] = x
        lpc[s] = lp
    return chain, lpc, nacc / (nsteps * W)


def max_threads() -> int:
    return _load().ora_max_threads()


def columns_renderer(pixel_scale, sub, psf, ny, nx, mass: str = "sie"):
    """A render function for the input generator: blurred unit columns from
    the oracle (used to synthesise data images in the tests)."""
    dummy = np.zeros((ny, nx))
    lens = Lens(dummy, np.ones((ny, nx)), psf, pixel_scale, sub, mass=mass)

    def render(params):
        _, ml, ms, _, _ = lens.model(params, mode=1)
        return ml, ms

    return render


if __name__ == "__main__":  # pragma: no cover
    print(build(force="--force" in sys.argv))
