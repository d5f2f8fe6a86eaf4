// tll_multi.cuh -- the multi-column likelihood kernel (templates).
//
// Sec. 2.3, Eq. 7: the lens light and the source light are sums of N_l and
// N_s unit-amplitude profiles, one column of L = [L_l | L_s] each; the
// amplitudes s >= 0 minimise ||(B L s - d)/n|| (the penalty after Eq. 7),
// solved by FNNLS (Bro & de Jong 1997) on the normal equations.  Sec. 3.2's
// SLACS model is two Sersics per galaxy (indices fixed at 1 and 4, one centre
// and one ellipticity per galaxy); Sec. 4.3 names the Gaussian expansion.
// Here a lens carries a list of up to kMaxComps components, each a Sersic
// (Eq. 8) or a unit-central-intensity Gaussian exp(-R_p^2 / 2 sigma^2), in
// the lens plane (at theta) or the source plane (at beta of Eq. 1); all
// components of a plane share that plane's centre and ellipticity (Eqs. 10,
// 11).
//
// Per parameter vector (one persistent CTA at a time):
//   1. trace passes: each pass evaluates up to kPassMax components of one
//      plane on every subpixel (the deflection once per subpixel for a
//      source pass), bins them, and writes the binned columns U[c] to the
//      CTA's global slot (L2-resident);
//   2. PSF: the columns two at a time through the compiled band convolution
//      (or the generic one), blurred columns M[c] written to the slot;
//   3. normal equations A = M^T W M, b = M^T W d: work items (row a, pixel
//      chunk) over the warps, products exact as float pairs, double-float
//      sums per lane, FP64 per item, FP64 over chunks;
//   4. one thread: FNNLS on (A, b) in FP64, chi^2 = dWd - 2 s^T b + s^T A s,
//      log L (Eq. 5).
#pragma once

#include "tll_kernels.cuh"

namespace tll {

constexpr int kMaxComps = 8;        // components (columns) per lens
constexpr int kPassMax = 4;         // components traced per pass
constexpr int kNcChunks = 8;        // pixel chunks per row of the normal equations
constexpr int K_C0 = NCONST_USED;   // per-component constants, 6 floats each
static_assert(K_C0 + 6 * kMaxComps <= NCONST, "constant block too small");

enum : int { COMP_SERSIC = 0, COMP_GAUSS = 1 };
enum : int { PLANE_LENS = 0, PLANE_SOURCE = 1 };
enum : int { FREE_SCALE = 1, FREE_INDEX = 2 };
constexpr int kMultiHead = 15;      // mass (7), lens geometry (4), source geometry (4)

// A lens's component list and its trace schedule (kernel parameter).
struct MultiDev {
    int nc, npar, npass;
    int type[kMaxComps], plane[kMaxComps], flags[kMaxComps];
    float scale[kMaxComps], index[kMaxComps];
    int pass_plane[kMaxComps], pass_n[kMaxComps];
    int pass_comp[kMaxComps][kPassMax];
};

// Arguments of one multi-column launch.
struct NcArgs {
    const float *kc;      // [B][NCONST]
    int B;
    double *out;          // [B]
    float *gscr;          // per-CTA slots of gslot floats: U [nc][npix],
    long long gslot;      // M [nc + 1][npix], H [2][npix] (generic separable)
    double *wr_res;       // WRITE: [nc amplitudes, log L] of vector 0, or null
};

// ------------------------------------------------------------- prologue
// One multi-component vector (layout: [0..6] mass and shear, [7..10] lens
// light eps1, eps2, x, y, [11..14] the same for the source, then each
// component's free scale and free Sersic index in component order, the EPL
// slope last) into its constant block.  The mass, shear and the two planes'
// frames come from decode_vector given unit r_e (so the planes' coordinates
// are R_p itself); per component c, at K_C0 + 6c:
//   Sersic:   1/r_e^2, 1/(2n), b_n log2(e)   (hi, lo each)
//   Gaussian: -log2(e) / (2 sigma^2)          (hi, lo)
__device__ inline void decode_multi(const float *__restrict__ p, float *__restrict__ o,
                                    const LensDev &L, const MultiDev &M,
                                    const double *__restrict__ bn_tab)
{
    float v[NPAR_EPL];
#pragma unroll
    for (int k = 0; k < 7; ++k) v[k] = p[k];
    v[7] = 1.0f; v[8] = 1.0f; v[9] = 1.0f;
    v[10] = p[7]; v[11] = p[8]; v[12] = p[9]; v[13] = p[10];
    v[14] = 1.0f; v[15] = 1.0f; v[16] = 1.0f;
    v[17] = p[11]; v[18] = p[12]; v[19] = p[13]; v[20] = p[14];
    v[21] = L.epl ? p[M.npar - 1] : 2.0f;
    decode_vector(v, o, L.XC, L.YC, L.d, bn_tab, L.epl != 0);
    if (o[K_VALID] == 0.0f) return;
    const double LOG2E = 1.4426950408889634;
    int slot = kMultiHead;
    bool ok = true;
    for (int c = 0; c < M.nc; ++c) {
        const double sc = (M.flags[c] & FREE_SCALE) ? (double)p[slot++] : (double)M.scale[c];
        ok = ok && isfinite(sc) && sc > 0.0;
        float *q = o + K_C0 + 6 * c;
#pragma unroll
        for (int e = 0; e < 6; ++e) q[e] = 0.0f;
        if (M.type[c] == COMP_SERSIC) {
            const double n = (M.flags[c] & FREE_INDEX) ? (double)p[slot++] : (double)M.index[c];
            ok = ok && n >= 0.2 && n <= 10.0;
            if (ok) {
                split2(1.0 / (sc * sc), &q[0], &q[1]);
                split2(0.5 / n, &q[2], &q[3]);
                split2(sersic_bn_lookup(bn_tab, n) * LOG2E, &q[4], &q[5]);
            }
        } else if (ok) {
            split2(-LOG2E / (2.0 * sc * sc), &q[0], &q[1]);
        }
    }
    if (!ok) o[K_VALID] = 0.0f;
}

// ---------------------------------------------------------------- trace
// One component at R2 = R_p^2 (its plane's shared frame), constants q[0..5].
// Sersic (Eq. 8): (R_p/r_e)^2 = R2 / r_e^2, then the same steps as
// sersic_scaled.  Gaussian: 2^(-log2(e) R2 / (2 sigma^2)).
__device__ __forceinline__ float comp_value(bool gauss, float R2, float q0, float q1, float q2,
                                            float q3, float q4, float q5)
{
    if (gauss) return sfu_ex2(fmaf(q0, R2, q1 * R2));
    const float r2 = fmaf(q1, R2, q0 * R2);
    const float Lg = sfu_lg2(r2);
    const float t = exp2_rr(fmaf(q2, Lg, q3 * Lg));
    const float omt = 1.0f - t;
    return sfu_ex2(fmaf(q4, omt, q5 * omt));
}

// One trace pass: the ncp (<= kPassMax) components listed in pc (their
// constants cq[6 * k], Gaussian flags in gmask) of one plane on every
// subpixel, binned by the mean, written to U + chan[k] * npix.
// MODE: 0 / 1 / 2 source plane with the SIE fast / general form or the EPL
// series (ec); 3 lens plane (no deflection).
// skip: trace only the lens's listed pixels (as trace_image).
template <int SUB, int MODE>
__device__ __forceinline__ void trace_pass(const LensDev &L, const VecConst &v,
                                           const float *cq, int gmask, int ncp,
                                           const int *chan, float *U, int tid, int nthr,
                                           const float *ec, bool skip)
{
    const int sub = SUB > 0 ? SUB : L.sub;
    const int nx = L.nx, npix = L.npix;
    const int *list = skip ? L.tlist : nullptr;
    const int n = list ? L.ntrace : npix;
    float q[kPassMax][6];
#pragma unroll
    for (int k = 0; k < kPassMax; ++k)
#pragma unroll
        for (int e = 0; e < 6; ++e) q[k][e] = k < ncp ? cq[6 * k + e] : 0.0f;
    for (int t = tid; t < n; t += nthr) {
        const int pix = list ? list[t] : t;
        const int i = pix / nx, j = pix - i * nx;
        const float fj0 = (float)(j * sub) - L.JCX;
        const float fi0 = (float)(i * sub) - L.JCY;
        float nlx = 0.0f, nly = 0.0f;
        if (MODE != 3) {
            nlx = -fmaf(v.sxl.cj, fj0, fmaf(v.sxl.ci, fi0, v.sxl.c0));
            nly = -fmaf(v.syl.cj, fj0, fmaf(v.syl.ci, fi0, v.syl.c0));
        }
        float acc[kPassMax];
#pragma unroll
        for (int k = 0; k < kPassMax; ++k) acc[k] = 0.0f;
#pragma unroll 1
        for (int a = 0; a < sub; ++a) {
            const RowTerms r = row_terms(v, fi0 + (float)a);
#pragma unroll
            for (int c = 0; c < (SUB > 0 ? SUB : 1); ++c) {
                for (int cr = 0; cr < (SUB > 0 ? 1 : sub); ++cr) {
                    const float fj = fj0 + (float)(SUB > 0 ? c : cr);
                    float X, Y;
                    if constexpr (MODE == 3) {
                        X = fmaf(v.lx.cj, fj, r.lx);
                        Y = fmaf(v.ly.cj, fj, r.ly);
                    } else {
                        float ux, uy;
                        if constexpr (MODE == 2)
                            epl_unit(v, fmaf(v.px.cj, fj, r.px), fmaf(v.py.cj, fj, r.py), ec,
                                     ux, uy);
                        else
                            sie_unit<MODE == 0>(v, fmaf(v.px.cj, fj, r.px),
                                                fmaf(v.py.cj, fj, r.py), ux, uy);
                        const float t1 = fmaf(v.q11h, ux, fmaf(v.q11l, ux,
                                         fmaf(v.q12h, uy, fmaf(v.q12l, uy, nlx))));
                        const float t2 = fmaf(v.q21h, ux, fmaf(v.q21l, ux,
                                         fmaf(v.q22h, uy, fmaf(v.q22l, uy, nly))));
                        X = fmaf(v.sx.cj, fj, r.sx) - t1;
                        Y = fmaf(v.sy.cj, fj, r.sy) - t2;
                    }
                    const float R2 = fmaf(X, X, Y * Y);
#pragma unroll
                    for (int k = 0; k < kPassMax; ++k)
                        if (k < ncp)
                            acc[k] += comp_value((gmask >> k) & 1, R2, q[k][0], q[k][1],
                                                 q[k][2], q[k][3], q[k][4], q[k][5]);
                }
            }
        }
#pragma unroll
        for (int k = 0; k < kPassMax; ++k)
            if (k < ncp) U[(size_t)chan[k] * npix + pix] = acc[k] * L.inv_s2;
    }
}

// ----------------------------------------------------- normal equations
// Row a of the normal equations over pixels [p0, p1): lane-strided, each
// lane holds double-float sums of w m_a m_e (e = a .. nc-1) and w d m_a
// (products exact as float pairs, as accum_pixel), reduced over the warp;
// lane 0 returns them in FP64 to out[0 .. nc - a] (the last is b_a).
__device__ __forceinline__ void nc_row_sums(const LensDev &L, const float *M, int nc, int a,
                                            int p0, int p1, int lane, double *out)
{
    const int npix = L.npix;
    float acc[2 * (kMaxComps + 1)];
#pragma unroll
    for (int k = 0; k < 2 * (kMaxComps + 1); ++k) acc[k] = 0.0f;
    const float *Ma = M + (size_t)a * npix;
    for (int pix = p0 + lane; pix < p1; pix += 32) {
        const float4 wp = L.wpack[pix];
        const float ma = Ma[pix];
        const float p1v = wp.x * ma;
        float e1 = fmaf(wp.x, ma, -p1v);
        e1 = fmaf(wp.y, ma, e1);
#pragma unroll
        for (int k = 0; k < kMaxComps; ++k) {
            if (a + k < nc) {
                const float me = M[(size_t)(a + k) * npix + pix];
                const float p = p1v * me;
                float e = fmaf(p1v, me, -p);
                e = fmaf(e1, me, e);
                df_acc(acc[2 * k], acc[2 * k + 1], p, e);
            }
        }
        const float p = wp.z * ma;
        float e = fmaf(wp.z, ma, -p);
        e = fmaf(wp.w, ma, e);
        df_acc(acc[2 * kMaxComps], acc[2 * kMaxComps + 1], p, e);
    }
#pragma unroll
    for (int k = 0; k <= kMaxComps; ++k) {
        if (k == kMaxComps || a + k < nc) {
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                const float oh = __shfl_xor_sync(0xffffffffu, acc[2 * k], o);
                const float ol = __shfl_xor_sync(0xffffffffu, acc[2 * k + 1], o);
                df_add(acc[2 * k], acc[2 * k + 1], oh, ol);
            }
        }
    }
    if (lane == 0) {
#pragma unroll
        for (int k = 0; k < kMaxComps; ++k)
            if (a + k < nc) out[k] = (double)acc[2 * k] + (double)acc[2 * k + 1];
        out[nc - a] = (double)acc[2 * kMaxComps] + (double)acc[2 * kMaxComps + 1];
    }
}

// -------------------------------------------------------------- FNNLS
// Solve G z = r for the passive columns listed in idx[0..k) of the n x n
// matrix A (row-major): Cholesky G = R^T R, R upper triangular, stored
// in place in F.  Returns false if a pivot is not positive.
__device__ inline bool nc_passive_solve(const double *A, const double *b, int n,
                                        const int *idx, int k, double *F, double *z)
{
    for (int i = 0; i < k; ++i) {
        for (int j = i; j < k; ++j) {
            double v = A[idx[i] * n + idx[j]];
            for (int t = 0; t < i; ++t) v = fma(-F[t * kMaxComps + i], F[t * kMaxComps + j], v);
            if (j == i) {
                if (!(v > 0.0)) return false;
                F[i * kMaxComps + i] = sqrt(v);
            } else {
                F[i * kMaxComps + j] = v / F[i * kMaxComps + i];
            }
        }
    }
    for (int i = 0; i < k; ++i) {
        double v = b[idx[i]];
        for (int t = 0; t < i; ++t) v = fma(-F[t * kMaxComps + i], z[t], v);
        z[i] = v / F[i * kMaxComps + i];
    }
    for (int i = k - 1; i >= 0; --i) {
        double v = z[i];
        for (int t = i + 1; t < k; ++t) v = fma(-F[i * kMaxComps + t], z[t], v);
        z[i] = v / F[i * kMaxComps + i];
    }
    return true;
}

// Least squares on the passive set (mask bit i set: column i free):
// s = A_PP^{-1} b_P there, 0 elsewhere.
__device__ inline bool nc_solve_set(const double *A, const double *b, int n, unsigned mask,
                                    double *s, double *F)
{
    int idx[kMaxComps];
    double z[kMaxComps];
    int k = 0;
    for (int i = 0; i < n; ++i) {
        s[i] = 0.0;
        if (mask >> i & 1u) idx[k++] = i;
    }
    if (k == 0) return true;
    if (!nc_passive_solve(A, b, n, idx, k, F, z)) return false;
    for (int t = 0; t < k; ++t) s[idx[t]] = z[t];
    return true;
}

// FNNLS (Bro & de Jong 1997): the Lawson-Hanson active-set method on the
// normal equations A x = b, x >= 0 (one thread, FP64, n <= kMaxComps).
// All columns start at zero; while a zero column has gradient
// g = b - A x above tol = 10 eps ||A||_1 n, the largest one is freed and
// the free set's least-squares solution s is taken, stepping back to the
// feasible boundary (freed columns that reach zero return to the zero set)
// while some free s_i <= 0.  A column whose own least-squares value comes
// out non-positive on entry is passed over until x next changes.  At most
// 30 n steps.
__device__ inline void nc_fnnls(const double *A, const double *b, int n, double *x)
{
    double F[kMaxComps * kMaxComps], s[kMaxComps], g[kMaxComps];
    double norm1 = 0.0;
    for (int j = 0; j < n; ++j) {
        double cs = 0.0;
        for (int i = 0; i < n; ++i) cs += fabs(A[i * n + j]);
        norm1 = fmax(norm1, cs);
    }
    const double tol = 10.0 * 2.220446049250313e-16 * norm1 * n;
    unsigned P = 0u, skip = 0u;
    for (int i = 0; i < n; ++i) {
        x[i] = 0.0;
        g[i] = b[i];
    }
    for (int step = 0; step < 30 * n; ++step) {
        int j = -1;
        double gmax = tol;
        for (int i = 0; i < n; ++i)
            if (!((P | skip) >> i & 1u) && g[i] > gmax) {
                gmax = g[i];
                j = i;
            }
        if (j < 0) return;
        P |= 1u << j;
        if (!nc_solve_set(A, b, n, P, s, F) || !(s[j] > 0.0)) {
            P &= ~(1u << j);
            skip |= 1u << j;
            continue;
        }
        for (int inner = 0; inner <= n; ++inner) {
            double alpha = 2.0;
            int kmin = -1;
            for (int i = 0; i < n; ++i)
                if ((P >> i & 1u) && s[i] <= 0.0) {
                    const double t = x[i] / (x[i] - s[i]);
                    if (t < alpha) {
                        alpha = t;
                        kmin = i;
                    }
                }
            if (kmin < 0) break;
            for (int i = 0; i < n; ++i) x[i] = fma(alpha, s[i] - x[i], x[i]);
            x[kmin] = 0.0;
            for (int i = 0; i < n; ++i)
                if ((P >> i & 1u) && x[i] <= 0.0) {
                    P &= ~(1u << i);
                    x[i] = 0.0;
                }
            if (!nc_solve_set(A, b, n, P, s, F)) return;
        }
        skip = 0u;
        for (int i = 0; i < n; ++i) x[i] = s[i];
        for (int i = 0; i < n; ++i) {
            double v = b[i];
            for (int k = 0; k < n; ++k) v = fma(-A[i * n + k], x[k], v);
            g[i] = v;
        }
    }
}

// --------------------------------------------------------------- kernel
// Shared memory: static -- partial sums, the normal equations, the
// components' constants, the EPL series; dynamic -- K > 0: the padded band
// buffer of the compiled convolution (2 channels x (band_rows + 2h + kCR)
// rows x W); K == 0: the PSF taps of the generic convolution.
template <int SUB, int K>
__global__ void __launch_bounds__(kThreads)
k_loglike_nc(const __grid_constant__ LensDev L, const __grid_constant__ MultiDev M,
             const __grid_constant__ NcArgs R)
{
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ double sPart[kMaxComps * kNcChunks * (kMaxComps + 1)];
    __shared__ double sA[kMaxComps * kMaxComps], sb[kMaxComps];
    __shared__ float sq[kMaxComps * 6];
    __shared__ float sepl[kEplMaxN + 1];
    const int tid = threadIdx.x, nthr = blockDim.x;
    const int lane = tid & 31, warp = tid >> 5, nwarp = nthr >> 5;
    const int nc = M.nc, npix = L.npix;
    float *spsf = reinterpret_cast<float *>(smem);
    float *U = R.gscr + (size_t)blockIdx.x * R.gslot;
    float *Mb = U + (size_t)nc * npix;
    float *H = Mb + (size_t)(nc + 1) * npix;
    setup_lens(L, spsf, tid, nthr);
    // pixels never traced (masked lenses) must start finite
    if (L.tlist)
        for (int t = tid; t < nc * npix; t += nthr) U[t] = 0.0f;
    __syncthreads();
    const bool skip = R.wr_res == nullptr;   // model columns: every pixel
    const int nch = max(1, min(kNcChunks, (2 * nwarp + nc - 1) / nc));
    for (int b = blockIdx.x; b < R.B; b += gridDim.x) {
        const float *kc = R.kc + (size_t)b * NCONST;
        if (kc[K_VALID] == 0.0f) {
            if (tid == 0) {
                R.out[b] = -INFINITY;
                if (R.wr_res) R.wr_res[nc] = -INFINITY;
            }
            continue;
        }
        const VecConst v = load_consts(kc);
        for (int t = tid; t < 6 * nc; t += nthr) sq[t] = kc[K_C0 + t];
        if (v.epl)
            for (int t = tid; t <= v.en; t += nthr) sepl[t] = kc[K_EC0 + t];
        __syncthreads();
        // 1. trace passes
        for (int ps = 0; ps < M.npass; ++ps) {
            const int ncp = M.pass_n[ps];
            float cq[6 * kPassMax];
            int gmask = 0;
#pragma unroll
            for (int k = 0; k < kPassMax; ++k) {
                const int c = k < ncp ? M.pass_comp[ps][k] : 0;
#pragma unroll
                for (int e = 0; e < 6; ++e) cq[6 * k + e] = sq[6 * c + e];
                if (k < ncp && M.type[c] == COMP_GAUSS) gmask |= 1 << k;
            }
            const int *chan = M.pass_comp[ps];
            if (M.pass_plane[ps] == PLANE_LENS)
                trace_pass<SUB, 3>(L, v, cq, gmask, ncp, chan, U, tid, nthr, sepl, skip);
            else if (v.epl)
                trace_pass<SUB, 2>(L, v, cq, gmask, ncp, chan, U, tid, nthr, sepl, skip);
            else if (v.fast)
                trace_pass<SUB, 0>(L, v, cq, gmask, ncp, chan, U, tid, nthr, sepl, skip);
            else
                trace_pass<SUB, 1>(L, v, cq, gmask, ncp, chan, U, tid, nthr, sepl, skip);
        }
        __syncthreads();
        // 2. PSF, two columns at a time (an odd last column pairs with itself)
        for (int c = 0; c < nc; c += 2) {
            const int c2 = min(c + 1, nc - 1);
            const float *Il = U + (size_t)c * npix, *Is = U + (size_t)c2 * npix;
            if constexpr (K > 0) {
                const int h = L.h, W = L.W, HL = L.HL, ny = L.ny, nx = L.nx;
                const int step = L.band_rows;
                float *Pl = spsf, *Ps = spsf + (step + 2 * h + kCR) * W;
                PairStore st{Mb + (size_t)c * npix, Mb + (size_t)c2 * npix};
                for (int b0 = 0; b0 < ny; b0 += step) {
                    const int nrows = min(step, ny - b0);
                    const int nbr = nrows + 2 * h;
                    for (int t = tid; t < 2 * nbr * nx; t += nthr) {
                        const int ch = t / (nbr * nx), rem = t - ch * nbr * nx;
                        const int br = rem / nx, j = rem - br * nx;
                        const int ir = b0 - h + br;
                        const float val = (ir >= 0 && ir < ny) ? (ch ? Is : Il)[ir * nx + j] : 0.0f;
                        (ch ? Ps : Pl)[br * W + HL + j] = val;
                    }
                    __syncthreads();
                    if (L.sep)
                        conv_sep_band<K>(L, Pl, Ps, b0, nrows, max(0, h - b0),
                                         min(nbr, ny - b0 + h), tid, nthr, st);
                    else
                        conv_direct_band<K>(L, Pl, Ps, b0, nrows, tid, nthr, st);
                    __syncthreads();
                }
            } else {
                RunArgs ra = {};
                ra.wr_blurred = Mb + (size_t)c * npix;
                float dummy[10];
                // writes M[c] and M[c + 1] (the spare column M[nc] for an odd
                // last column); its five sums go unused
                conv_generic<true>(L, ra, spsf, const_cast<float *>(Il), const_cast<float *>(Is),
                                   H, H + npix, dummy, tid, nthr, false);
                __syncthreads();
            }
        }
        __syncthreads();
        // 3. normal equations: items (row a, chunk) over the warps
        const int per = (npix + nch - 1) / nch;
        for (int item = warp; item < nc * nch; item += nwarp) {
            const int a = item / nch, ch = item - a * nch;
            const int p0 = ch * per, p1 = min(npix, p0 + per);
            nc_row_sums(L, Mb, nc, a, p0, p1, lane,
                        sPart + (size_t)(a * kNcChunks + ch) * (kMaxComps + 1));
        }
        __syncthreads();
        if (tid < nc * (nc + 1)) {   // sum over chunks; A symmetric
            const int a = tid / (nc + 1), k = tid - a * (nc + 1);
            if (k >= a || k == nc) {
                const int kk = k == nc ? nc - a : k - a;
                double s = 0.0;
                for (int ch = 0; ch < nch; ++ch)
                    s += sPart[(size_t)(a * kNcChunks + ch) * (kMaxComps + 1) + kk];
                if (k == nc) sb[a] = s;
                else { sA[a * nc + k] = s; sA[k * nc + a] = s; }
            }
        }
        __syncthreads();
        // 4. amplitudes and log L
        if (tid == 0) {
            double x[kMaxComps];
            nc_fnnls(sA, sb, nc, x);
            double chi2 = L.dWd;
            for (int i = 0; i < nc; ++i) {
                double Ax = 0.0;
                for (int k = 0; k < nc; ++k) Ax = fma(sA[i * nc + k], x[k], Ax);
                chi2 += x[i] * (Ax - 2.0 * sb[i]);
            }
            const double ll = -0.5 * chi2 + L.lognorm;
            R.out[b] = ll;
            if (R.wr_res) {
                for (int i = 0; i < nc; ++i) R.wr_res[i] = x[i];
                R.wr_res[nc] = ll;
            }
        }
        __syncthreads();
    }
}

using NcKernel = void (*)(const LensDev, const MultiDev, const NcArgs);

// Kernels of one translation unit; nullptr when (sub, K) is not in it.
struct KernelSet {
    SingleKernel (*single)(int sub, int K, bool write);
    MultiKernel (*multi)(int sub, int K);
    NcKernel (*nc)(int sub, int K);
};

template <int K>
inline NcKernel nc_for(int sub)
{
    switch (sub_class(sub)) {
        case 4: return k_loglike_nc<4, K>;
        case 5: return k_loglike_nc<5, K>;
        default: return k_loglike_nc<0, K>;
    }
}

}  // namespace tll
