// tll_device.cuh -- device-side arithmetic of the lens likelihood (sm_103a).
//
// Per-vector prologue (ellipse, b_n, SIE prefactors) and the per-subpixel
// forward model of arXiv:2503.08586: SIE + external shear deflection, the
// lens equation (Sec. 2.1, Eq. 1), and unit-amplitude elliptical Sersic light
// (Sec. 2.4, Eqs. 8-11).  Plus double-float (float pair) helpers used by the
// likelihood reduction.  Written for the GPU path only.
#pragma once

#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

namespace tll {

constexpr int NPAR = 21;

// Per-vector constants written by the prologue, NCONST floats per vector.
// Offsets O* are (grid origin - centre) so that a subpixel's coordinate
// relative to a centre is one add from its grid offset.  *H / *L pairs are
// the high and low float parts of a constant (double-float).
enum : int {
    K_VALID = 0,
    // mass: offsets to the SIE centre, rotation, q, prefactor A/f (hi, lo),
    // f = sqrt(1 - q^2), q = 1 flag, shear
    K_OXM, K_OYM, K_CM, K_SM, K_QM, K_AFH, K_AFL, K_F, K_SIS, K_G1, K_G2,
    // lens light: offsets, rotation, q/r_e^2, 1/(q r_e^2), 1/(2n) (hi, lo),
    // b log2(e) (hi, lo)
    K_OXL, K_OYL, K_CL, K_SL, K_A1L, K_A2L, K_KHL, K_KLL, K_BHL, K_BLL,
    // source, same fields
    K_OXS, K_OYS, K_CS, K_SS, K_A1S, K_A2S, K_KHS, K_KLS, K_BHS, K_BLS,
    // fixed amplitudes
    K_IEL, K_IES,
    NCONST_USED
};
constexpr int NCONST = 40;
static_assert(NCONST_USED <= NCONST, "constant block too small");

// ------------------------------------------------------------------ b_n
// Root of P(2n, b) = 1/2 (Eq. 9: Gamma(2n) = 2 gamma(2n, b_n)) by a
// safeguarded Newton iteration in FP64.  Start: the Ciotti & Bertin (1999)
// expansion for n >= 0.36, the MacArthur, Courteau & Holtzman (2003)
// polynomial below.  P(a, x) from the power series of the lower incomplete
// gamma function; dP/dx = x^{a-1} e^{-x} / Gamma(a).
__device__ inline double sersic_bn_dev(double n)
{
    const double a = 2.0 * n;
    const double lga = lgamma(a);
    double b = (n >= 0.36)
        ? 2.0 * n - 1.0 / 3.0 + 4.0 / (405.0 * n) + 46.0 / (25515.0 * n * n)
        : 0.01945 + n * (-0.8902 + n * (10.95 + n * (-19.67 + n * 13.43)));
    double lo = 0.0, hi = a + 1.0;
    if (!(b > lo && b < hi)) b = 0.5 * (lo + hi);
    for (int it = 0; it < 64; ++it) {
        double term = 1.0 / a, sum = term;
        for (int k = 1; k < 2000; ++k) {
            term *= b / (a + k);
            sum += term;
            if (term < 1e-17 * sum) break;
        }
        const double lb = log(b);
        const double P = exp(a * lb - b - lga) * sum;
        const double g = P - 0.5;
        if (g < 0.0) lo = b; else hi = b;
        const double dP = exp((a - 1.0) * lb - b - lga);
        double nb = b - g / dP;
        if (!(nb > lo && nb < hi)) nb = 0.5 * (lo + hi);
        const bool done = fabs(nb - b) <= 4e-16 * b;
        b = nb;
        if (done || hi - lo <= 4e-16 * hi) break;
    }
    return b;
}

__device__ __forceinline__ void split2(double v, float *o_hi, float *o_lo)
{
    const float h = (float)v;
    *o_hi = h;
    *o_lo = (float)(v - (double)h);
}

// --------------------------------------------------------------- prologue
// Decode one parameter vector into its constant block.  Validity: finite
// entries, theta_E >= 0, |eps| < 1 for the three ellipses, r_e > 0, Sersic
// index in [0.2, 10]; an invalid vector gets K_VALID = 0.  (X0, Y0) is the
// coordinate of the grid centre, the origin of subpixel offsets (FP64).
__device__ inline void decode_vector(const float *__restrict__ p, float *__restrict__ o,
                                     double X0, double Y0)
{
    bool ok = true;
    double v[NPAR];
#pragma unroll
    for (int k = 0; k < NPAR; ++k) {
        v[k] = (double)p[k];
        ok = ok && isfinite(v[k]);
    }
    ok = ok && v[0] >= 0.0;
    ok = ok && v[8] > 0.0 && v[15] > 0.0;
    ok = ok && v[9] >= 0.2 && v[9] <= 10.0 && v[16] >= 0.2 && v[16] <= 10.0;
    const double e_m = sqrt(v[1] * v[1] + v[2] * v[2]);
    const double e_l = sqrt(v[10] * v[10] + v[11] * v[11]);
    const double e_s = sqrt(v[17] * v[17] + v[18] * v[18]);
    ok = ok && e_m < 1.0 && e_l < 1.0 && e_s < 1.0;
#pragma unroll
    for (int k = 0; k < NCONST; ++k) o[k] = 0.0f;
    if (!ok) return;
    o[K_VALID] = 1.0f;
    const double LOG2E = 1.4426950408889634;
    {   // mass: q = (1-e)/(1+e), angle = atan2(e2, e1)/2, f = 2 sqrt(e)/(1+e)
        const double q = (1.0 - e_m) / (1.0 + e_m);
        const double ang = 0.5 * atan2(v[2], v[1]);
        const double f = 2.0 * sqrt(e_m) / (1.0 + e_m);
        const double A = v[0] * sqrt(q);
        o[K_OXM] = (float)(X0 - v[3]);
        o[K_OYM] = (float)(Y0 - v[4]);
        o[K_CM] = (float)cos(ang);
        o[K_SM] = (float)sin(ang);
        o[K_QM] = (float)q;
        o[K_F] = (float)f;
        if (f < 1e-6) { o[K_SIS] = 1.0f; split2(A, &o[K_AFH], &o[K_AFL]); }
        else { o[K_SIS] = 0.0f; split2(A / f, &o[K_AFH], &o[K_AFL]); }
        o[K_G1] = (float)v[5];
        o[K_G2] = (float)v[6];
    }
    // Sersic components: lens light (centre in slots 12, 13) and source
    const int base[2] = {K_OXL, K_OXS};
    const int par[2] = {8, 15};   // r_e, n, eps1, eps2, x, y follow r_e's slot
    const double e_c[2] = {e_l, e_s};
#pragma unroll
    for (int comp = 0; comp < 2; ++comp) {
        const int P0 = par[comp], B0 = base[comp];
        const double re = v[P0], n = v[P0 + 1];
        const double q = (1.0 - e_c[comp]) / (1.0 + e_c[comp]);
        const double ang = 0.5 * atan2(v[P0 + 3], v[P0 + 2]);
        o[B0 + 0] = (float)(X0 - v[P0 + 4]);
        o[B0 + 1] = (float)(Y0 - v[P0 + 5]);
        o[B0 + 2] = (float)cos(ang);
        o[B0 + 3] = (float)sin(ang);
        o[B0 + 4] = (float)(q / (re * re));
        o[B0 + 5] = (float)(1.0 / (q * re * re));
        split2(0.5 / n, &o[B0 + 6], &o[B0 + 7]);
        split2(sersic_bn_dev(n) * LOG2E, &o[B0 + 8], &o[B0 + 9]);
    }
    o[K_IEL] = (float)v[7];
    o[K_IES] = (float)v[14];
}

// ------------------------------------------------------------ subpixel
struct Ellipse {   // one Sersic component in registers
    float ox, oy, c, s, a1, a2, kh, kl, bh, bl;
};
struct Mass {
    float ox, oy, c, s, q, afh, afl, f, g1, g2;
    bool sis;
};

__device__ __forceinline__ Ellipse load_ellipse(const float *kc, int b)
{
    Ellipse e;
    e.ox = kc[b + 0]; e.oy = kc[b + 1]; e.c = kc[b + 2]; e.s = kc[b + 3];
    e.a1 = kc[b + 4]; e.a2 = kc[b + 5]; e.kh = kc[b + 6]; e.kl = kc[b + 7];
    e.bh = kc[b + 8]; e.bl = kc[b + 9];
    return e;
}

__device__ __forceinline__ Mass load_mass(const float *kc)
{
    Mass m;
    m.ox = kc[K_OXM]; m.oy = kc[K_OYM]; m.c = kc[K_CM]; m.s = kc[K_SM];
    m.q = kc[K_QM]; m.afh = kc[K_AFH]; m.afl = kc[K_AFL]; m.f = kc[K_F];
    m.g1 = kc[K_G1]; m.g2 = kc[K_G2];
    m.sis = kc[K_SIS] != 0.0f;
    return m;
}

// Unit-amplitude elliptical Sersic at offset (u, v) from its centre:
// rotate (Eq. 10), (R_p/r_e)^2 = q x1^2/r_e^2 + x2^2/(q r_e^2),
// t = (R_p/r_e)^{1/n} = 2^{log2((R_p/r_e)^2)/(2n)},
// I = exp(-b (t - 1)) = 2^{b log2(e) (1 - t)} (Eq. 8).
__device__ __forceinline__ float sersic_unit(const Ellipse &e, float u, float v)
{
    const float x1 = fmaf(u, e.c, v * e.s);
    const float x2 = fmaf(v, e.c, -u * e.s);
    const float r2 = fmaf(x1 * x1, e.a1, x2 * x2 * e.a2);
    const float L = log2f(r2);
    const float t = exp2f(fmaf(e.kh, L, e.kl * L));
    const float omt = 1.0f - t;
    return exp2f(fmaf(e.bh, omt, e.bl * omt));
}

// 1/sqrt(a) to about 1 ulp: the hardware estimate plus one Newton step.
__device__ __forceinline__ float rsqrt_nr(float a)
{
    const float y = rsqrtf(a);
    const float hy = 0.5f * a * y;
    return fmaf(y, fmaf(-hy, y, 0.5f), y);
}

// Deflection of SIE (Eq. 12 at gamma = 2, elliptical radius of Eq. 10) at
// offset (dx, dy) from the mass centre, plus external shear (Eqs. 13, 14) at
// the absolute position (x, y).  SIE in the frame rotated by the mass angle:
// with psi = sqrt(q^2 x'^2 + y'^2),
//   alpha_x' = A/f atan(f x'/psi),  alpha_y' = A/f atanh(f y'/psi),
// A = theta_E sqrt(q), f = sqrt(1 - q^2); for f -> 0 the q = 1 limit
// alpha' = A (x', y')/psi.  Shear: alpha = (g1 x + g2 y, g2 x - g1 y).
__device__ __forceinline__ void deflection(const Mass &m, float dx, float dy,
                                           float x, float y, float &ax, float &ay)
{
    const float xp = fmaf(dx, m.c, dy * m.s);
    const float yp = fmaf(dy, m.c, -dx * m.s);
    const float qx = m.q * xp;
    const float psi2 = fmaxf(fmaf(qx, qx, yp * yp), 1e-24f);
    const float rpsi = rsqrt_nr(psi2);
    float axp, ayp;
    if (m.sis) {
        const float tx = xp * rpsi, ty = yp * rpsi;
        axp = fmaf(m.afh, tx, m.afl * tx);
        ayp = fmaf(m.afh, ty, m.afl * ty);
    } else {
        const float fr = m.f * rpsi;
        const float zy = fminf(fmaxf(yp * fr, -0.99999994f), 0.99999994f);
        const float at = atanf(xp * fr), ah = atanhf(zy);
        axp = fmaf(m.afh, at, m.afl * at);
        ayp = fmaf(m.afh, ah, m.afl * ah);
    }
    ax = fmaf(axp, m.c, -ayp * m.s) + fmaf(m.g1, x, m.g2 * y);
    ay = fmaf(axp, m.s, ayp * m.c) + fmaf(m.g2, x, -m.g1 * y);
}

// ------------------------------------------------------ double-float
// A value is carried as an unevaluated sum hi + lo of two floats.
// two_prod: a*b = p + e exactly (FMA).  acc: (hi, lo) += (p + e) with the
// rounding error of hi + p recovered by the TwoSum of Knuth / Moller.
__device__ __forceinline__ void df_acc(float &hi, float &lo, float p, float e)
{
    const float s = hi + p;
    const float bp = s - hi;
    const float err = (hi - (s - bp)) + (p - bp);
    hi = s;
    lo += err + e;
}

__device__ __forceinline__ void df_add(float &ahi, float &alo, float bhi, float blo)
{
    const float s = ahi + bhi;
    const float bp = s - ahi;
    const float err = (ahi - (s - bp)) + (bhi - bp);
    const float lo = err + alo + blo;
    const float hi = s + lo;
    alo = lo - (hi - s);
    ahi = hi;
}

}  // namespace tll
