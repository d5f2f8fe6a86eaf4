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
constexpr int NPAR_EPL = 22;     // elliptical power-law mass: slope gamma at [21]
constexpr int kEplMaxN = 63;     // highest power of the EPL deflection series
// The EPL series as a per-vector table over cos(2 vphi) in [-1, 1]:
// kEplTab cubic Hermite intervals of width 2 / kEplTab, one more at each
// end (kEplTab + 2 in all), two float4 per interval; used where the
// series' ratio (1 - q)/(1 + q) is at most kEplTabR (q >= 0.48), where the
// interpolation is below 2e-8 of the sum for slopes 1.2 .. 2.8.
constexpr int kEplTab = 128;
constexpr float kEplTabR = 0.35f;
// shared memory of the EPL staging per vector: the table, or the series'
// coefficients c_0 .. c_63 where the table is not used
constexpr int kEplSmemFloats = 8 * (kEplTab + 2);
static_assert(kEplSmemFloats >= kEplMaxN + 1, "EPL staging");

// Per-vector constants written by the prologue, NCONST floats per vector.
// Every coordinate a subpixel needs is an affine function of its integer
// offsets (fj, fi) from the grid centre: C0 + CJ fj + CI fi.  Constants
// whose rounding to float would move the model coherently are float pairs
// (hi + lo): the hi parts sit in the slots below, every lo part in the
// aligned block at K_LO (layout LO_*), which the trace reads once per
// pixel (load_pixlo) instead of holding it in registers.
enum : int {
    K_VALID = 0,
    // mass frame: x' = PX0 + PXJ fj + PXI fi, y' = PY0 + PYJ fj + PYI fi;
    // q, f = sqrt(1 - q^2); SIE form (1 fast, 2 mid, 0 general)
    K_PX0, K_PXJ, K_PXI, K_PY0, K_PYJ, K_PYI, K_QM, K_F, K_FAST,
    // lens light, scaled frame (x1 sqrt(q)/r_e, x2/(sqrt(q) r_e)):
    // affine coefficients, 1/(2n), b log2(e)
    K_LX0, K_LXJ, K_LXI, K_LY0, K_LYJ, K_LYI, K_KHL, K_BHL,
    // source, scaled frame at theta minus shear (linear part), 1/(2n),
    // b log2(e) ...
    K_SX0, K_SXJ, K_SXI, K_SY0, K_SYJ, K_SYI, K_KHS, K_BHS,
    // ... minus the SIE deflection A (ux, uy) mapped from the mass frame:
    // [Q11 Q12; Q21 Q22]
    K_Q11H, K_Q12H, K_Q21H, K_Q22H,
    // fixed amplitudes
    K_IEL, K_IES,
    // elliptical power law (Eq. 12 at any slope): flag, highest power N of
    // the deflection series, the magnitude's exponent e0 + e1 log2(psi^2)
    // (hi, lo each), and whether the kernels take the series from a table
    K_EPL, K_EN, K_E0H, K_E0L, K_E1H, K_E1L, K_ETAB,
    // the lo parts (float4-aligned), then the EPL series coefficients c_0 .. c_N
    K_LO = (K_E1L + 4) & ~3,
    K_EC0 = K_LO + 28,
    NCONST_USED = K_EC0 + kEplMaxN + 1
};
// Layout of the lo block: the affine maps' (c0, cj, ci) of the mass frame
// (PX, PY), the lens-light frame (LX, LY) and the source frame (SX, SY);
// q and f of the mass; 1/(2n) and b log2(e) of the lens light (KL, BL)
// and of the source (KS, BS); the deflection map Q.
enum : int {
    LO_PX = 0, LO_PY = 3, LO_LX = 6, LO_LY = 9, LO_SX = 12, LO_SY = 15,
    LO_Q = 18, LO_F = 19, LO_KL = 20, LO_BL = 21, LO_KS = 22, LO_BS = 23,
    LO_Q11 = 24, LO_Q12 = 25, LO_Q21 = 26, LO_Q22 = 27, LO_N = 28
};
constexpr int NCONST = 336;
static_assert(NCONST_USED <= NCONST, "constant block too small");
static_assert(K_ETAB < K_LO, "constant slots");
static_assert(K_LO % 4 == 0 && LO_N % 4 == 0 && NCONST % 4 == 0 && K_EC0 == K_LO + LO_N,
              "float4 reads of the lo block");

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

// b_n table: two uniform segments, n in [0.2, 1] and [1, 10], BN_NT nodes
// each plus one guard node below and two above, filled once per device by
// k_bn_table (sersic_bn_dev at each node) and read by cubic Lagrange
// interpolation through the four nearest nodes (relative error < 3e-12).
constexpr int BN_NT = 2048;
constexpr int BN_SEG = BN_NT + 3;
__host__ __device__ __forceinline__ double bn_lo(int seg) { return seg ? 1.0 : 0.2; }
__host__ __device__ __forceinline__ double bn_hi(int seg) { return seg ? 10.0 : 1.0; }

__device__ __forceinline__ double bn_node(int seg, int k)   // k = -1 .. BN_NT + 1
{
    const double h = (bn_hi(seg) - bn_lo(seg)) / (BN_NT - 1);
    return bn_lo(seg) + h * k;
}

__device__ inline double sersic_bn_lookup(const double *__restrict__ tab, double n)
{
    const int seg = n < 1.0 ? 0 : 1;
    const double h = (bn_hi(seg) - bn_lo(seg)) / (BN_NT - 1);
    const double u = (n - bn_lo(seg)) * (1.0 / h);
    int i = (int)floor(u);
    i = max(0, min(i, BN_NT - 2));
    const double t = u - i;
    const double *p = tab + seg * BN_SEG + i;   // nodes i-1 .. i+2
    const double tm1 = t - 1.0, tm2 = t - 2.0, tp1 = t + 1.0;
    return (-t * tm1 * tm2 * (1.0 / 6.0)) * p[0] + (tp1 * tm1 * tm2 * 0.5) * p[1]
           - (tp1 * t * tm2 * 0.5) * p[2] + (tp1 * t * tm1 * (1.0 / 6.0)) * p[3];
}

// (cos phi, sin phi) of phi = atan2(e2, e1)/2 (Eq. 11's position angle) by
// the half-angle formulas, without trigonometric calls.
__device__ __forceinline__ void half_angle(double e1, double e2, double e,
                                           double *c, double *s)
{
    if (!(e > 0.0)) { *c = 1.0; *s = 0.0; return; }
    const double c2 = e1 / e, s2 = e2 / e;
    if (c2 >= 0.0) {
        const double cc = sqrt(0.5 * (1.0 + c2));
        *c = cc;
        *s = s2 / (2.0 * cc);
    } else {
        const double ss = copysign(sqrt(0.5 * (1.0 - c2)), s2);
        *s = ss;
        *c = s2 / (2.0 * ss);
    }
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
// index in [0.2, 10]; an invalid vector gets K_VALID = 0.  (XC, YC) is the
// grid centre and d the subpixel step: subpixel (fj, fi) sits at
// (XC + fj d, YC + fi d).  All arithmetic here is FP64, rounded once.
//
// Derivation of the folded coefficients (R(phi) = rotation by +phi):
//   mass frame        x' = R(-phi_m) (theta - c_m)                  (Eq. 10)
//   SIE deflection    alpha = R(phi_m) A (ux, uy), A = theta_E sqrt(q_m)
//   shear             alpha_sh = G theta, G = [[g1, g2], [g2, -g1]] (Eq. 13/14)
//   source position   beta = theta - alpha - G theta                 (Eq. 1)
//   source frame      (x1, x2) = R(-phi_s) (beta - c_s), scaled by
//                     (sqrt(q_s)/r_e, 1/(sqrt(q_s) r_e)) so (R_p/r_e)^2 =
//                     x1^2 + x2^2                                    (Eq. 10)
// so the scaled source coordinates are an affine map of theta minus
// S R(phi_m - phi_s) A (ux, uy), S = diag of the scales.
//
// part: which slots to write -- all of them (part < 0), or one of four
// disjoint sets, so that four threads (one per warp of a (32, 4) block)
// decode one vector together: 0 validity, mass frame, q, f, SIE form,
// fixed amplitudes; 1 lens light; 2 source frame and Sersic; 3 the
// deflection map Q and the EPL series.  A part recomputes the few shared
// quantities it needs (the mass angle and q for part 3, ...).  Every part
// finds the same validity; an invalid vector's part 0 writes K_VALID = 0
// and nothing else is read.  |eps| < 1 is tested as eps1^2 + eps2^2 < 1,
// the same decision as sqrt(.) < 1 under correctly rounded sqrt.
__device__ __forceinline__ void zero_range(float *o, int a, int b)
{
    for (int k = a; k < b; ++k) o[k] = 0.0f;
}

__device__ inline void decode_vector(const float *__restrict__ p, float *__restrict__ o,
                                     double XC, double YC, double d,
                                     const double *__restrict__ bn_tab, bool epl = false,
                                     int part = -1)
{
    const bool all = part < 0;
    bool ok = true;
    double v[NPAR_EPL];
#pragma unroll
    for (int k = 0; k < NPAR; ++k) {
        v[k] = (double)p[k];
        ok = ok && isfinite(v[k]);
    }
    v[21] = epl ? (double)p[21] : 2.0;
    ok = ok && v[21] > 1.0 && v[21] < 3.0;   // slope (EPL), non-finite fails too
    ok = ok && v[0] >= 0.0;
    ok = ok && v[8] > 0.0 && v[15] > 0.0;
    ok = ok && v[9] >= 0.2 && v[9] <= 10.0 && v[16] >= 0.2 && v[16] <= 10.0;
    const double e2_m = v[1] * v[1] + v[2] * v[2];
    const double e2_l = v[10] * v[10] + v[11] * v[11];
    const double e2_s = v[17] * v[17] + v[18] * v[18];
    ok = ok && e2_m < 1.0 && e2_l < 1.0 && e2_s < 1.0;
    float *lo = o + K_LO;
    if (all) {
        zero_range(o, 0, NCONST_USED);
    } else if (part == 0) {
        zero_range(o, K_VALID, K_FAST + 1);
        zero_range(o, K_IEL, K_IES + 1);
        zero_range(lo, LO_PX, LO_PY + 3);
        zero_range(lo, LO_Q, LO_F + 1);
    } else if (part == 1) {
        zero_range(o, K_LX0, K_BHL + 1);
        zero_range(lo, LO_LX, LO_LY + 3);
        zero_range(lo, LO_KL, LO_BL + 1);
    } else if (part == 2) {
        zero_range(o, K_SX0, K_BHS + 1);
        zero_range(lo, LO_SX, LO_SY + 3);
        zero_range(lo, LO_KS, LO_BS + 1);
    } else {
        zero_range(o, K_Q11H, K_Q22H + 1);
        zero_range(o, K_EPL, K_LO);
        zero_range(lo, LO_Q11, LO_Q22 + 1);
        zero_range(o, K_EC0, NCONST_USED);
    }
    if (!ok) return;
    if (all || part == 0) o[K_VALID] = 1.0f;
    const double LOG2E = 1.4426950408889634;

    // mass: q = (1-e)/(1+e), f = sqrt(1 - q^2) = 2 sqrt(e)/(1+e)
    double qm = 0.0, f = 0.0, A = 0.0, cm = 1.0, sm = 0.0;
    bool fast = false, mid = false;
    if (all || part == 0 || part == 3) {
        const double e_m = sqrt(e2_m);
        qm = (1.0 - e_m) / (1.0 + e_m);
        f = 2.0 * sqrt(e_m) / (1.0 + e_m);
        A = v[0] * sqrt(qm);
        half_angle(v[1], v[2], e_m, &cm, &sm);
        // fast form when |f x'/psi| <= f/q <= 1 and |f y'/psi| <= f <= 1/2
        // for every point: no atan range reduction, no atanh logarithm;
        // mid form when f/q <= 1 but f > 1/2: no atan range reduction, the
        // atanh by logarithms (1/f < 2 keeps them accurate)
        fast = f <= qm && f <= 0.5;
        mid = f <= qm && !fast;
    }
    if (all || part == 0) {
        const double dx = XC - v[3], dy = YC - v[4];
        split2(dx * cm + dy * sm, &o[K_PX0], &lo[LO_PX]);
        split2(d * cm, &o[K_PXJ], &lo[LO_PX + 1]);
        split2(d * sm, &o[K_PXI], &lo[LO_PX + 2]);
        split2(-dx * sm + dy * cm, &o[K_PY0], &lo[LO_PY]);
        split2(-d * sm, &o[K_PYJ], &lo[LO_PY + 1]);
        split2(d * cm, &o[K_PYI], &lo[LO_PY + 2]);
        split2(qm, &o[K_QM], &lo[LO_Q]);
        split2(f, &o[K_F], &lo[LO_F]);
        o[K_FAST] = fast ? 1.0f : mid ? 2.0f : 0.0f;
        o[K_IEL] = (float)v[7];
        o[K_IES] = (float)v[14];
    }
    const double g1 = v[5], g2 = v[6];

    // lens light (centre in slots 12, 13)
    if (all || part == 1) {
        const double re = v[8], n = v[9];
        const double e_l = sqrt(e2_l);
        const double q = (1.0 - e_l) / (1.0 + e_l);
        double c, s;
        half_angle(v[10], v[11], e_l, &c, &s);
        const double s1 = sqrt(q) / re, s2 = 1.0 / (sqrt(q) * re);
        const double dx = XC - v[12], dy = YC - v[13];
        split2(s1 * (dx * c + dy * s), &o[K_LX0], &lo[LO_LX]);
        split2(s1 * d * c, &o[K_LXJ], &lo[LO_LX + 1]);
        split2(s1 * d * s, &o[K_LXI], &lo[LO_LX + 2]);
        split2(s2 * (-dx * s + dy * c), &o[K_LY0], &lo[LO_LY]);
        split2(-s2 * d * s, &o[K_LYJ], &lo[LO_LY + 1]);
        split2(s2 * d * c, &o[K_LYI], &lo[LO_LY + 2]);
        split2(0.5 / n, &o[K_KHL], &lo[LO_KL]);
        split2(sersic_bn_lookup(bn_tab, n) * LOG2E, &o[K_BHL], &lo[LO_BL]);
    }
    // source
    if (all || part == 2 || part == 3) {
        const double re = v[15], n = v[16];
        const double e_s = sqrt(e2_s);
        const double q = (1.0 - e_s) / (1.0 + e_s);
        double c, s;
        half_angle(v[17], v[18], e_s, &c, &s);
        const double s1 = sqrt(q) / re, s2 = 1.0 / (sqrt(q) * re);
        if (all || part == 2) {
            // linear part: beta_lin = (I - G) theta - c_s, theta = (XC + fj d, YC + fi d)
            const double bx0 = (1.0 - g1) * XC - g2 * YC - v[19];
            const double by0 = -g2 * XC + (1.0 + g1) * YC - v[20];
            const double bxj = (1.0 - g1) * d, bxi = -g2 * d;
            const double byj = -g2 * d, byi = (1.0 + g1) * d;
            // double-float: rounding these to float alone would move the whole
            // source plane coherently (a shift and scale near 1e-7), which the
            // likelihood near its optimum resolves
            split2(s1 * (c * bx0 + s * by0), &o[K_SX0], &lo[LO_SX]);
            split2(s1 * (c * bxj + s * byj), &o[K_SXJ], &lo[LO_SX + 1]);
            split2(s1 * (c * bxi + s * byi), &o[K_SXI], &lo[LO_SX + 2]);
            split2(s2 * (-s * bx0 + c * by0), &o[K_SY0], &lo[LO_SY]);
            split2(s2 * (-s * bxj + c * byj), &o[K_SYJ], &lo[LO_SY + 1]);
            split2(s2 * (-s * bxi + c * byi), &o[K_SYI], &lo[LO_SY + 2]);
            split2(0.5 / n, &o[K_KHS], &lo[LO_KS]);
            split2(sersic_bn_lookup(bn_tab, n) * LOG2E, &o[K_BHS], &lo[LO_BS]);
        }
        if (all || part == 3) {
            // deflection term: S R(-phi_s) R(phi_m) A = S R(phi_m - phi_s) A
            const double cd = cm * c + sm * s;    // cos(phi_m - phi_s)
            const double sd = sm * c - cm * s;    // sin(phi_m - phi_s)
            // The fast form's (ux, uy) are atan(zx)/f, atanh(zy)/f; the general
            // form's are atan(zx) and log2((1 + zy)/(1 - zy)) = 2 atanh(zy)/ln 2,
            // so its columns carry 1/f and ln 2/(2f); the mid form has the fast
            // ux and the general uy.
            double c1 = (fast || mid) ? 1.0 : 1.0 / f;
            double c2 = fast ? 1.0 : 0.34657359027997264 / f;
            double Am = A;
            if (epl) {
                // EPL (Tessore & Metcalf 2015 in this normalisation): with
                // t = gamma - 1, b = theta_E sqrt(q), psi^2 = q^2 x'^2 + y'^2 and
                // psi e^{i vphi} = q x' + i y', the deflection in the mass frame
                // is 2b/(1+q) (b/psi)^(t-1) e^{i vphi} sum_n c_n e^{2 i n vphi},
                // c_n = prod_{k<=n} (2k - 2 + t)/(2k + 2 - t) (-(1-q)/(1+q))^n
                // (the series of 2F1(1, t/2; 2 - t/2; .)).  (ux, uy) is that sum
                // times (b/psi)^(t-1) = 2^(e0 + e1 log2 psi^2); Q carries 2b/(1+q).
                const double t = v[21] - 1.0, fr = -(1.0 - qm) / (1.0 + qm);
                o[K_EPL] = 1.0f;
                // e0 bounded to [-60, 60] (and 0 at theta_E = 0, where Q = 0
                // makes the deflection vanish whatever the magnitude), so the
                // kernel's exp2 argument e0 + e1 log2 psi^2 (|e1| < 1/2,
                // log2 psi^2 in [-80, 50]) stays within its unclamped range;
                // the bound only acts for theta_E outside [1e-18, 1e18]
                const double e0 = A > 0.0 ? fmin(fmax((t - 1.0) * log2(A), -60.0), 60.0) : 0.0;
                split2(e0, &o[K_E0H], &o[K_E0L]);
                split2(0.5 * (1.0 - t), &o[K_E1H], &o[K_E1L]);
                double cn = 1.0;
                int N = 0;
                o[K_EC0] = 1.0f;
                for (int nn = 1; nn <= kEplMaxN; ++nn) {
                    cn *= fr * (2.0 * nn - 2.0 + t) / (2.0 * nn + 2.0 - t);
                    o[K_EC0 + nn] = (float)cn;
                    N = nn;
                    if (fabs(cn) < 1e-9) break;   // the rest of the series is below float rounding
                }
                o[K_EN] = (float)N;
                o[K_ETAB] = -fr <= (double)kEplTabR ? 1.0f : 0.0f;
                c1 = c2 = 1.0;
                Am = 2.0 * A / (1.0 + qm);
            }
            split2(s1 * Am * cd * c1, &o[K_Q11H], &lo[LO_Q11]);
            split2(-s1 * Am * sd * c2, &o[K_Q12H], &lo[LO_Q12]);
            split2(s2 * Am * sd * c1, &o[K_Q21H], &lo[LO_Q21]);
            split2(s2 * Am * cd * c2, &o[K_Q22H], &lo[LO_Q22]);
        }
    }
}

// ------------------------------------------------------------ subpixel
// Per-vector constants in registers.
struct Affine {    // v = c0 + cj fj + ci fi
    float c0, cj, ci;
};
struct VecConst {
    Affine px, py, lx, ly, sx, sy;
    float q, f;           // q, f of the mass (hi parts)
    bool fast, mid;       // SIE form (general when neither)
    float khl, bhl, khs, bhs;
    float q11h, q12h, q21h, q22h;
    bool epl;                       // elliptical power-law mass
    bool etab;                      // its series from the table
    int en;                         // highest power of its series
    float e0h, e0l, e1h, e1l;       // its magnitude's exponent
};

__device__ __forceinline__ Affine load_affine(const float *kc, int b)
{
    return Affine{kc[b], kc[b + 1], kc[b + 2]};
}

__device__ __forceinline__ VecConst load_consts(const float *kc)
{
    VecConst v;
    v.px = load_affine(kc, K_PX0); v.py = load_affine(kc, K_PY0);
    v.lx = load_affine(kc, K_LX0); v.ly = load_affine(kc, K_LY0);
    v.sx = load_affine(kc, K_SX0); v.sy = load_affine(kc, K_SY0);
    v.q = kc[K_QM]; v.f = kc[K_F];
    v.fast = kc[K_FAST] == 1.0f;
    v.mid = kc[K_FAST] == 2.0f;
    v.khl = kc[K_KHL]; v.bhl = kc[K_BHL]; v.khs = kc[K_KHS]; v.bhs = kc[K_BHS];
    v.q11h = kc[K_Q11H]; v.q12h = kc[K_Q12H]; v.q21h = kc[K_Q21H]; v.q22h = kc[K_Q22H];
    v.epl = kc[K_EPL] != 0.0f;
    v.etab = kc[K_ETAB] != 0.0f;
    v.en = (int)kc[K_EN];
    v.e0h = kc[K_E0H]; v.e0l = kc[K_E0L]; v.e1h = kc[K_E1H]; v.e1l = kc[K_E1L];
    return v;
}

// The lo block of a vector's constants (LO_* layout), read at a pixel's
// first subpixel: seven float4 loads (L1-resident: every thread of the CTA
// reads the same block), live only until the pixel's lo terms are formed.
// The loads are volatile so that the compiler keeps them in the pixel loop
// rather than hoisting them out of it and holding 28 registers throughout;
// plain (coherent) global loads, since a kernel may have written the block
// itself before a barrier (the fused prologue of small batches).
struct PixLo {
    float w[LO_N];
};

__device__ __forceinline__ PixLo load_pixlo(const float *__restrict__ kc)
{
    PixLo p;
    const float *s = kc + K_LO;
#pragma unroll
    for (int k = 0; k < LO_N / 4; ++k)
        asm volatile("ld.global.v4.f32 {%0, %1, %2, %3}, [%4];"
                     : "=f"(p.w[4 * k]), "=f"(p.w[4 * k + 1]), "=f"(p.w[4 * k + 2]),
                       "=f"(p.w[4 * k + 3])
                     : "l"(s + 4 * k));
    return p;
}

// SFU instructions (PTX ISA: ex2.approx, lg2.approx, rcp.approx).
__device__ __forceinline__ float sfu_ex2(float x)
{
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float sfu_lg2(float x)
{
    float y;
    asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float sfu_rcp(float x)
{
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// 2^x for x <= 30 by range reduction x = k + f, k = rint(x), |f| <= 1/2:
// ex2.approx on f (unbiased on that interval, unlike on wide arguments),
// times 2^k added into the exponent field.  rint: adding 1.5 * 2^23 leaves
// k in the low mantissa bits of kf, and kf's bits << 23 are k << 23.
// CLAMP: x is first clamped below at -125 so the result stays a normal
// float (smaller values only enter pixel sums far below the model's
// rounding); a NaN x (only from 0 * inf at r = 0, where 2^x -> 0 is wanted)
// also becomes -125.  Without CLAMP the caller guarantees x >= -125.
template <bool CLAMP = true>
__device__ __forceinline__ float exp2_rr(float x)
{
    if (CLAMP) x = fmaxf(x, -125.0f);
    const float kf = x + 12582912.0f;
    const float f = x - (kf - 12582912.0f);
    const float y = sfu_ex2(f);
    return __int_as_float(__float_as_int(y) + (__float_as_int(kf) << 23));
}

// Horner in s for the Q(s) polynomials of tll_poly.cuh.
__device__ __forceinline__ float poly_atan_q(float s)
{
    float q = -1.753930119e-03f;
    q = fmaf(q, s, 1.072694361e-02f);
    q = fmaf(q, s, -3.080459684e-02f);
    q = fmaf(q, s, 5.755210295e-02f);
    q = fmaf(q, s, -8.377315104e-02f);
    q = fmaf(q, s, 1.094203070e-01f);
    q = fmaf(q, s, -1.426193267e-01f);
    q = fmaf(q, s, 1.999826580e-01f);
    return fmaf(q, s, -3.333328366e-01f);
}
__device__ __forceinline__ float poly_atanh_q(float s)
{
    float q = 1.785548776e-01f;
    q = fmaf(q, s, 4.985036701e-02f);
    q = fmaf(q, s, 1.187057048e-01f);
    q = fmaf(q, s, 1.421579868e-01f);
    q = fmaf(q, s, 2.000301927e-01f);
    return fmaf(q, s, 3.333328366e-01f);
}

// Unit-amplitude Sersic (Eq. 8) from L = log2((R_p/r_e)^2) (Eq. 10 folded
// into the scaled-frame coordinates x1, x2 with (R_p/r_e)^2 = x1^2 + x2^2):
// t = (R_p/r_e)^{1/n} = 2^{L/(2n)}, I = exp(-b (t - 1)) = 2^{b log2(e) (1 - t)}.
// 1/(2n) = kh + kl and b log2(e) = bh + bl are float pairs; the lo parts
// of the two exponents, kl L and bl (1 - t), come in as c and d (the pixel
// loop passes those of the pixel's first subpixel).  The pow's exponential
// is range-reduced (its bias would scale with b t); the outer one is not (a
// bias there is a near-uniform relative scale).
__device__ __forceinline__ float sersic_omt(float L, float kh, float c)
{
    return 1.0f - exp2_rr<false>(fmaf(kh, L, c));
}

// (R_p/r_e)^2 = x1^2 + x2^2 with a floor of 2^-50 added inside the FMA:
// log2 of it is >= -50, so kh L >= -125 for every valid index (n >= 0.2,
// kh = 1/(2n) <= 2.5) and the pow's exp2 needs no clamp.  The floor changes
// (R_p/r_e)^2 by less than an ulp wherever R_p/r_e > 3e-4.
constexpr float kR2Floor = 8.8817842e-16f;   // 2^-50
__device__ __forceinline__ float radius2(float x1, float x2)
{
    return fmaf(x1, x1, fmaf(x2, x2, kR2Floor));
}
__device__ __forceinline__ float sersic_outer(float omt, float bh, float d)
{
    return sfu_ex2(fmaf(bh, omt, d));
}

// 1/sqrt(a) to about 1 ulp for normal a: the hardware estimate
// (rsqrt.approx) plus one Newton step.
__device__ __forceinline__ float rsqrt_nr(float a)
{
    float y;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(a));
    const float hy = 0.5f * a * y;
    return fmaf(y, fmaf(-hy, y, 0.5f), y);
}

// Per-pixel parts of the float-pair constants, taken at the pixel's first
// subpixel and reused by the others.  nlx, nly: minus the source position's
// lo terms -- the source-plane affine map's lo constants, and the lo parts
// of the deflection map Q times the deflection; cl, cs: the lo parts of
// 1/(2n) of the lens and source Sersics times the log-radii, dl, ds: the
// lo parts of b log2(e) times 1 - t; dq, dfx, dfy:
// the lo parts of q and f times the mass-frame x' and the SIE's x'/psi,
// y'/psi (EPL: de, the magnitude exponent's lo part e1l log2 psi^2 + e0l).
// Across a pixel these terms change by at most an ulp of what they enter
// near the lens and light centres, where the deflection turns and t moves
// fastest, and by far less elsewhere.
struct PixelLo {
    float nlx, nly, cl, cs, dl, ds, dq, dfx, dfy;
};

// SIE deflection (Eq. 12 at gamma = 2, elliptical radius of Eq. 10) in the
// mass frame at (xp, yp), as alpha' = A (ux, uy) up to the column scales the
// prologue folds into Q: with psi = sqrt(q^2 xp^2 + yp^2), zx = f xp/psi,
// zy = f yp/psi (f = sqrt(1 - q^2), A = theta_E sqrt(q)):
//  FAST (vectors with f/q <= 1 and f <= 1/2, so |zx| <= 1, |zy| <= 1/2):
//   ux = atan(zx)/f = (xp/psi) P_atan(zx^2), uy = atanh(zy)/f = (yp/psi)
//   P_atanh(zy^2), with atan(w) = w P_atan(w^2), atanh(w) = w P_atanh(w^2)
//   (tll_poly.cuh); relative accuracy, and the q = 1 limit needs no special
//   case.
//  general (f > 1/2 here, so 1/f is bounded): ux = atan(zx), reduced to
//   sign(z) pi/2 - atan(1/z) where |z| > 1; uy = log2(1 + zy) - log2(1 - zy)
//   = 2 atanh(zy)/ln 2 (|zy| <= f < 1), accurate in absolute terms.
//  mid (f/q <= 1 but f > 1/2): the fast ux (|zx| <= 1, no reduction) and
//   the general uy.
// FORM: 0 fast, 1 general, 2 mid (decided once per vector by the prologue).
// ql, fl: the lo parts of q and f (read when FIRST).
template <int FORM, bool FIRST>
__device__ __forceinline__ void sie_unit(const VecConst &v, float ql, float fl, float xp,
                                         float yp, PixelLo &P, float &ux, float &uy)
{
    // q and f enter as double-float constants (their rounding would change
    // the profile coherently); the products are rounded once, their lo
    // parts taken at the pixel's first subpixel
    if (FIRST) P.dq = ql * xp;
    const float qx = fmaf(v.q, xp, P.dq);
    // psi^2 >= 1e-24 (the singular centre, reading R4), added inside the FMA
    const float rpsi = rsqrt_nr(fmaf(qx, qx, fmaf(yp, yp, 1e-24f)));
    const float xr = xp * rpsi, yr = yp * rpsi;
    if (FIRST) {
        P.dfx = fl * xr;
        P.dfy = fl * yr;
    }
    const float zx = fmaf(v.f, xr, P.dfx), zy = fmaf(v.f, yr, P.dfy);
    if (FORM == 0) {
        const float sx = zx * zx, sy = zy * zy;
        ux = fmaf(xr * sx, poly_atan_q(sx), xr);
        uy = fmaf(yr * sy, poly_atanh_q(sy), yr);
    } else if (FORM == 2) {
        const float sx = zx * zx;
        ux = fmaf(xr * sx, poly_atan_q(sx), xr);
        uy = sfu_lg2(1.0f + zy) - sfu_lg2(1.0f - zy);
    } else {
        const float ax = fabsf(zx);
        const bool big = ax > 1.0f;
        const float w = big ? sfu_rcp(ax) : ax;
        const float sw = w * w;
        const float pw = fmaf(w * sw, poly_atan_q(sw), w);
        const float at = big ? (1.57079637f - pw) - 4.37113883e-08f : pw;
        ux = copysignf(at, zx);
        uy = sfu_lg2(1.0f + zy) - sfu_lg2(1.0f - zy);
    }
}

// EPL deflection (Eq. 12 at slope gamma) in the mass frame at (xp, yp), as
// alpha' = (2b/(1+q)) (ux, uy) with Q carrying 2b/(1+q):
//   (ux + i uy) = (b/psi)^(t-1) e^{i vphi} sum_{n<=N} c_n w^n,
//   psi e^{i vphi} = q xp + i yp, w = e^{2 i vphi},
// the magnitude as 2^(e0 + e1 log2 psi^2) with a range-reduced exp2 (the
// prologue bounds e0, so no clamp).  The sum's real and imaginary parts,
// C = sum c_n cos(n th) and S = sum c_n sin(n th) with th = 2 vphi, come
// from one Clenshaw recurrence,
//   b_k = c_k + 2 cos(th) b_{k+1} - b_{k+2},  C = b_0 - b_1 cos(th),
//   S = b_1 sin(th),
// two operations per term where complex Horner takes four; as accurate in
// FP32 (both about 5e-8 rms of the sum over q >= 0.5, slopes 1.6-2.4, in a
// float32 emulation).  With c = cos vphi, s = sin vphi, cos th = c^2 - s^2
// and sin th = 2 c s, the rotation by e^{i vphi} collapses:
//   Re = c C - s S = c (b_0 - b_1),  Im = s C + c S = s (b_0 + b_1).
// ec: the coefficients c_0 .. c_63 staged in shared memory per vector,
// 16-byte aligned and zero beyond N, read four at a time.  ql: the lo part
// of q (read when FIRST).
// TAB: the two sums F1 = b_0 - b_1 and F2 = b_0 + b_1, functions of
// x = cos th alone, from the vector's table at ec (epl_table): interval k
// covers x in [-1 + (k - 1) h, -1 + k h], h = 2 / kEplTab; its position
// U = (x + 1)/h + 1 is split as k = floor(U) by rounding U - 1/2 against
// 1.5 * 2^23 (the integer in the sum's low mantissa bits) and t = U - k,
// then one cubic per sum, ((a3 t + a2) t + a1) t + a0.
template <bool FIRST, bool TAB = false>
__device__ __forceinline__ void epl_unit(const VecConst &v, float ql, float xp, float yp,
                                         const float *ec, PixelLo &P, float &ux, float &uy)
{
    if (FIRST) P.dq = ql * xp;
    const float qx = fmaf(v.q, xp, P.dq);
    const float a = fmaf(qx, qx, fmaf(yp, yp, 1e-24f));
    const float rpsi = rsqrt_nr(a);
    const float c = qx * rpsi, s = yp * rpsi;            // e^{i vphi}
    const float al = 2.0f * fmaf(c, c, -s * s);          // 2 cos th
    const float4 *ec4 = reinterpret_cast<const float4 *>(ec);
    float F1, F2;
    if constexpr (TAB) {
        constexpr float kMagic = 12582912.0f;            // 1.5 * 2^23
        const float um = fmaf(al, 0.25f * kEplTab, 0.5f * kEplTab + 0.5f);   // U - 1/2
        const float sm = __fadd_rn(um, kMagic);
        const float fk = __fsub_rn(sm, kMagic);
        const float t = __fadd_rn(__fsub_rn(um, fk), 0.5f);
        const int k = min(max(__float_as_int(sm) - 0x4B400000, 0), kEplTab + 1);
        const float4 A = ec4[2 * k], B = ec4[2 * k + 1];
        F1 = fmaf(fmaf(fmaf(A.w, t, A.z), t, A.y), t, A.x);
        F2 = fmaf(fmaf(fmaf(B.w, t, B.z), t, B.y), t, B.x);
    } else {
        float b1 = 0.0f, b2 = 0.0f;
#pragma unroll 1
        for (int g = v.en >> 2; g >= 0; --g) {
            const float4 cc = ec4[g];
            float b0;
            b0 = fmaf(al, b1, cc.w - b2); b2 = b1; b1 = b0;
            b0 = fmaf(al, b1, cc.z - b2); b2 = b1; b1 = b0;
            b0 = fmaf(al, b1, cc.y - b2); b2 = b1; b1 = b0;
            b0 = fmaf(al, b1, cc.x - b2); b2 = b1; b1 = b0;
        }
        F1 = b1 - b2;
        F2 = b1 + b2;
    }
    const float L = sfu_lg2(a);
    if (FIRST) P.dfx = fmaf(v.e1l, L, v.e0l);   // de
    const float m = exp2_rr<false>(fmaf(v.e1h, L, P.dfx) + v.e0h);
    ux = (m * c) * F1;
    uy = (m * s) * F2;
}

// One vector's EPL staging in shared memory (buf, kEplSmemFloats floats,
// 16-byte aligned), before its trace: the table when v.etab, else the
// series' coefficients.  Table interval k (threads take one each): the
// sums F1, F2 and their x-derivatives at both ends by the Clenshaw
// recurrence in alpha = 2x with its derivative
//   b_k' = b_{k+1} + alpha b_{k+1}' - b_{k+2}',
// then the cubic Hermite coefficients on t in [0, 1]:
//   a0 = F(x0), a1 = h F'(x0), a2 = 3 (F(x1) - F(x0)) - h (2 F'(x0) + F'(x1)),
//   a3 = 2 (F(x0) - F(x1)) + h (F'(x0) + F'(x1)).
// No barrier.
__device__ __forceinline__ void epl_sums_d(const float *c, int en, float x, float &F1, float &F2,
                                           float &D1, float &D2)
{
    const float al = 2.0f * x;
    float b1 = 0.0f, b2 = 0.0f, d1 = 0.0f, d2 = 0.0f;
    for (int n = en; n >= 0; --n) {
        const float b0 = fmaf(al, b1, c[n] - b2);
        const float d0 = fmaf(al, d1, b1 - d2);
        b2 = b1; b1 = b0;
        d2 = d1; d1 = d0;
    }
    F1 = b1 - b2;
    F2 = b1 + b2;
    D1 = 2.0f * (d1 - d2);       // d/dx = 2 d/dalpha
    D2 = 2.0f * (d1 + d2);
}

__device__ __forceinline__ void epl_stage(const float *kc, const VecConst &v, float *buf, int tid,
                                          int nthr)
{
    if (!v.etab) {
        for (int t = tid; t <= kEplMaxN; t += nthr) buf[t] = kc[K_EC0 + t];
        return;
    }
    const float *c = kc + K_EC0;
    const float h = 2.0f / kEplTab;
    float4 *tab = reinterpret_cast<float4 *>(buf);
    for (int k = tid; k < kEplTab + 2; k += nthr) {
        const float x0 = fmaf((float)(k - 1), h, -1.0f), x1 = x0 + h;
        float F1a, F2a, D1a, D2a, F1b, F2b, D1b, D2b;
        epl_sums_d(c, v.en, x0, F1a, F2a, D1a, D2a);
        epl_sums_d(c, v.en, x1, F1b, F2b, D1b, D2b);
        tab[2 * k] = make_float4(F1a, h * D1a, 3.0f * (F1b - F1a) - h * (2.0f * D1a + D1b),
                                 2.0f * (F1a - F1b) + h * (D1a + D1b));
        tab[2 * k + 1] = make_float4(F2a, h * D2a, 3.0f * (F2b - F2a) - h * (2.0f * D2a + D2b),
                                     2.0f * (F2a - F2b) + h * (D2a + D2b));
    }
}

// The two unit columns at one subpixel (fj, fi), given the row terms
// r* = c0 + ci fi of the six affine coordinates.
struct RowTerms {
    float px, py, lx, ly, sx, sy;
};

// A pixel's constant terms of the four image-plane coordinates (mass frame
// x', y'; lens-light frame x1, x2): c0 plus the lo parts of the whole map
// at the pixel's first subpixel (fj0, fi0), c0_lo + cj_lo fj0 + ci_lo fi0.
// Rounded to float, the steps cj, ci alone would stretch these frames
// coherently over the field -- by up to half an ulp of the step per
// subpixel of offset, about a third of an ulp of the coordinate at the edge
// of an 11 arcsec field -- a shift and scale of the whole model that the
// likelihood near its optimum resolves.  Across a pixel the lo sum changes
// by (s - 1) ulps of the step's lo part, far below a coordinate's rounding,
// so it is formed once per pixel and enters every subpixel through the row
// terms.
struct PixOrigin {
    float px, py, lx, ly;
};

__device__ __forceinline__ PixOrigin pixel_origin(const VecConst &v, const PixLo &lc, float fj0,
                                                  float fi0)
{
    const float *w = lc.w;
    return PixOrigin{v.px.c0 + fmaf(w[LO_PX + 1], fj0, fmaf(w[LO_PX + 2], fi0, w[LO_PX])),
                     v.py.c0 + fmaf(w[LO_PY + 1], fj0, fmaf(w[LO_PY + 2], fi0, w[LO_PY])),
                     v.lx.c0 + fmaf(w[LO_LX + 1], fj0, fmaf(w[LO_LX + 2], fi0, w[LO_LX])),
                     v.ly.c0 + fmaf(w[LO_LY + 1], fj0, fmaf(w[LO_LY + 2], fi0, w[LO_LY]))};
}

// Minus the source-plane affine map's lo part at the pixel's first subpixel
// (the source position's lo terms start from it; P.nlx, P.nly).
__device__ __forceinline__ void source_lo(const PixLo &lc, float fj0, float fi0, float &nlx,
                                          float &nly)
{
    const float *w = lc.w;
    nlx = -fmaf(w[LO_SX + 1], fj0, fmaf(w[LO_SX + 2], fi0, w[LO_SX]));
    nly = -fmaf(w[LO_SY + 1], fj0, fmaf(w[LO_SY + 2], fi0, w[LO_SY]));
}

__device__ __forceinline__ RowTerms row_terms(const VecConst &v, const PixOrigin &o, float fi)
{
    return RowTerms{fmaf(v.px.ci, fi, o.px), fmaf(v.py.ci, fi, o.py),
                    fmaf(v.lx.ci, fi, o.lx), fmaf(v.ly.ci, fi, o.ly),
                    fmaf(v.sx.ci, fi, v.sx.c0), fmaf(v.sy.ci, fi, v.sy.c0)};
}

// The mass deflection (the lens equation's alpha, Eq. 1) in its frame at
// subpixel column fj of row r.  MODE: 0 SIE fast form, 1 SIE general form,
// 2 EPL (series ec), 4 SIE mid form, 5 EPL from the table at ec.  ql, fl:
// lo parts of q and f (FIRST).
template <int MODE, bool FIRST>
__device__ __forceinline__ void deflect(const VecConst &v, float ql, float fl, const RowTerms &r,
                                        float fj, const float *ec, PixelLo &P, float &ux,
                                        float &uy)
{
    if constexpr (MODE == 2 || MODE == 5)
        epl_unit<FIRST, MODE == 5>(v, ql, fmaf(v.px.cj, fj, r.px), fmaf(v.py.cj, fj, r.py), ec,
                                   P, ux, uy);
    else
        sie_unit<MODE == 0 ? 0 : MODE == 4 ? 2 : 1, FIRST>(
            v, ql, fl, fmaf(v.px.cj, fj, r.px), fmaf(v.py.cj, fj, r.py), P, ux, uy);
}

// The two unit columns at the pixel's first subpixel (fj, row r), in full;
// fixes the pixel's lo terms from the lo block lc (P.nlx, P.nly come in
// with the affine map's part and leave with Q's added).
template <int MODE>
__device__ __forceinline__ void subpixel_first(const VecConst &v, const PixLo &lc,
                                               const RowTerms &r, float fj, const float *ec,
                                               PixelLo &P, float &il, float &is)
{
    const float *w = lc.w;
    float ux, uy;
    deflect<MODE, true>(v, w[LO_Q], w[LO_F], r, fj, ec, P, ux, uy);
    P.nlx = fmaf(w[LO_Q11], ux, fmaf(w[LO_Q12], uy, P.nlx));
    P.nly = fmaf(w[LO_Q21], ux, fmaf(w[LO_Q22], uy, P.nly));
    // lens light at theta (Eq. 2, first term)
    const float x1 = fmaf(v.lx.cj, fj, r.lx), x2 = fmaf(v.ly.cj, fj, r.ly);
    const float Ll = sfu_lg2(radius2(x1, x2));
    P.cl = w[LO_KL] * Ll;
    const float ol = sersic_omt(Ll, v.khl, P.cl);
    P.dl = w[LO_BL] * ol;
    il = sersic_outer(ol, v.bhl, P.dl);
    // source at beta = theta - alpha_SIE - alpha_shear (Eq. 2, second term)
    const float y1 = fmaf(v.sx.cj, fj, r.sx) - fmaf(v.q11h, ux, fmaf(v.q12h, uy, P.nlx));
    const float y2 = fmaf(v.sy.cj, fj, r.sy) - fmaf(v.q21h, ux, fmaf(v.q22h, uy, P.nly));
    const float Ls = sfu_lg2(radius2(y1, y2));
    P.cs = w[LO_KS] * Ls;
    const float os = sersic_omt(Ls, v.khs, P.cs);
    P.ds = w[LO_BS] * os;
    is = sersic_outer(os, v.bhs, P.ds);
}

// The two unit columns at any other subpixel of the pixel.
template <int MODE>
__device__ __forceinline__ void subpixel(const VecConst &v, const RowTerms &r, float fj,
                                         const float *ec, PixelLo &P, float &il, float &is)
{
    float ux, uy;
    deflect<MODE, false>(v, 0.0f, 0.0f, r, fj, ec, P, ux, uy);
    const float x1 = fmaf(v.lx.cj, fj, r.lx), x2 = fmaf(v.ly.cj, fj, r.ly);
    il = sersic_outer(sersic_omt(sfu_lg2(radius2(x1, x2)), v.khl, P.cl), v.bhl, P.dl);
    const float y1 = fmaf(v.sx.cj, fj, r.sx) - fmaf(v.q11h, ux, fmaf(v.q12h, uy, P.nlx));
    const float y2 = fmaf(v.sy.cj, fj, r.sy) - fmaf(v.q21h, ux, fmaf(v.q22h, uy, P.nly));
    is = sersic_outer(sersic_omt(sfu_lg2(radius2(y1, y2)), v.khs, P.cs), v.bhs, P.ds);
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

// a += b in double-float with the result symmetric in a and b bit for bit
// (TwoSum's error term is exact either way and the lo parts are added first),
// so both lanes of a butterfly step end with the same pair.
__device__ __forceinline__ void df_add_sym(float &ahi, float &alo, float bhi, float blo)
{
    const float s = ahi + bhi;
    const float bp = s - ahi;
    const float err = (ahi - (s - bp)) + (bhi - bp);
    const float lo = err + (alo + blo);
    const float hi = s + lo;
    alo = lo - (hi - s);
    ahi = hi;
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
