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
//   1. trace passes: each pass evaluates the components it lists (up to 4
//      of any kind, or up to 8 Gaussians) of one plane on every subpixel (the
//      deflection once per subpixel for a source pass), bins them, and
//      writes the binned columns U[c] to the CTA's global slot (L2-resident);
//   2. PSF: the columns two at a time through the compiled band convolution
//      (or the generic one), blurred columns M[c] written to the slot;
//   3. normal equations A = M^T W M, b = M^T W d: the blurred columns and
//      the weights staged in shared memory a pixel tile at a time; thread
//      (sum s, phase r) accumulates sum s over every R-th pixel of each tile
//      in double-float (products exact as float pairs), then the R partials
//      of each sum are added in FP64 in a fixed order;
//   4. warp 0: FNNLS on (A, b) in FP64 with the passive-set Cholesky solves
//      spread over the lanes, chi^2 = dWd - 2 s^T b + s^T A s, log L (Eq. 5).
#pragma once

#include "tll_kernels.cuh"

namespace tll {

constexpr int kPassSrcG = 6;        // ... source-plane Gaussians (the deflection's registers)
constexpr int kPassMix = 4;         // ... a pass with Sersic components
constexpr int K_C0 = NCONST_USED;   // per-component constants, 6 floats each
static_assert(K_C0 + 6 * kMaxComps <= NCONST, "constant block too small");

enum : int { COMP_SERSIC = 0, COMP_GAUSS = 1 };
enum : int { PLANE_LENS = 0, PLANE_SOURCE = 1 };
enum : int { FREE_SCALE = 1, FREE_INDEX = 2 };
constexpr int kMultiHead = 15;      // mass (7), lens geometry (4), source geometry (4)

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
// sersic_omt and sersic_outer.  Gaussian: 2^(-log2(e) R2 / (2 sigma^2)).
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

// One trace pass: ncp (<= NP) components (their constants cq[6 * k],
// Gaussian flags in gmask) of one plane on every subpixel, binned by the
// mean, component k written to U + k * npix, or to U + chan[k] * npix when
// full.  GAUSS: every component is a Gaussian (only its first two constants
// are kept).
// MODE: 0 / 1 / 4 / 2 source plane with the SIE fast / general / mid form or
// the EPL series (ec); 3 lens plane (no deflection).
// skip: trace only the lens's listed pixels (as trace_image).
template <int SUB, int MODE, int NP, bool GAUSS>
__device__ __forceinline__ void trace_pass(const LensDev &L, const VecConst &v,
                                           const float *kc, const float *cq, int gmask, int ncp,
                                           const int *chan, bool full, float *U, int tid,
                                           int nthr,
                                           const float *ec, bool skip)
{
    constexpr int NQ = GAUSS ? 2 : 6;
    const int sub = SUB > 0 ? SUB : L.sub;
    const int nx = L.nx, npix = L.npix;
    const int *list = skip ? L.tlist : nullptr;
    const int n = list ? L.ntrace : npix;
    float q[NP][NQ];
#pragma unroll
    for (int k = 0; k < NP; ++k)
#pragma unroll
        for (int e = 0; e < NQ; ++e) q[k][e] = k < ncp ? cq[6 * k + e] : 0.0f;
    for (int t = tid; t < n; t += nthr) {
        const int pix = list ? list[t] : t;
        const int i = div_nx(L, pix), j = pix - i * nx;
        const float fj0 = (float)(j * sub) - L.JCX;
        const float fi0 = (float)(i * sub) - L.JCY;
        const PixLo lc = load_pixlo(kc);
        float nlx = 0.0f, nly = 0.0f;
        if (MODE != 3) source_lo(lc, fj0, fi0, nlx, nly);
        const PixOrigin po = pixel_origin(v, lc, fj0, fi0);
        float acc[NP];
#pragma unroll
        for (int k = 0; k < NP; ++k) acc[k] = 0.0f;
#pragma unroll 1
        for (int a = 0; a < sub; ++a) {
            const RowTerms r = row_terms(v, po, fi0 + (float)a);
#pragma unroll
            for (int c = 0; c < (SUB > 0 ? SUB : 1); ++c) {
                for (int cr = 0; cr < (SUB > 0 ? 1 : sub); ++cr) {
                    const float fj = fj0 + (float)(SUB > 0 ? c : cr);
                    float X, Y;
                    if constexpr (MODE == 3) {
                        X = fmaf(v.lx.cj, fj, r.lx);
                        Y = fmaf(v.ly.cj, fj, r.ly);
                    } else {
                        // the lo parts of q and f taken at every subpixel here
                        float ux, uy;
                        PixelLo pl;
                        const float *w = lc.w;
                        if constexpr (MODE == 2)
                            epl_unit<true>(v, w[LO_Q], fmaf(v.px.cj, fj, r.px),
                                           fmaf(v.py.cj, fj, r.py), ec, pl, ux, uy);
                        else
                            sie_unit<MODE == 0 ? 0 : MODE == 4 ? 2 : 1, true>(
                                v, w[LO_Q], w[LO_F], fmaf(v.px.cj, fj, r.px),
                                fmaf(v.py.cj, fj, r.py), pl, ux, uy);
                        const float t1 = fmaf(v.q11h, ux, fmaf(w[LO_Q11], ux,
                                         fmaf(v.q12h, uy, fmaf(w[LO_Q12], uy, nlx))));
                        const float t2 = fmaf(v.q21h, ux, fmaf(w[LO_Q21], ux,
                                         fmaf(v.q22h, uy, fmaf(w[LO_Q22], uy, nly))));
                        X = fmaf(v.sx.cj, fj, r.sx) - t1;
                        Y = fmaf(v.sy.cj, fj, r.sy) - t2;
                    }
                    const float R2 = fmaf(X, X, Y * Y);
#pragma unroll
                    for (int k = 0; k < NP; ++k) {
                        if (k < ncp) {
                            if constexpr (GAUSS)
                                acc[k] += sfu_ex2(fmaf(q[k][0], R2, q[k][1] * R2));
                            else
                                acc[k] += comp_value((gmask >> k) & 1, R2, q[k][0], q[k][1],
                                                     q[k][2], q[k][3], q[k][4], q[k][5]);
                        }
                    }
                }
            }
        }
#pragma unroll
        for (int k = 0; k < NP; ++k)
            if (k < ncp) U[(size_t)(full ? chan[k] : k) * npix + pix] = acc[k] * L.inv_s2;
    }
}

// ----------------------------------------------------- normal equations
// Shared-memory tiles of the sums, T pixels each, in float offsets from the
// base: two buffers of the blurred columns M_c (R0 at 0, R1 at nc TS; row
// stride TS = T + 1, odd, so the lanes of a warp -- different columns at
// one pixel -- hit distinct banks), the pair operands at WM (every weighted
// column w M_c as an exact float pair, then the pixels' w d pairs as row nc;
// same stride) and two buffers of the pixels' weight records at WW (float4,
// 16-byte aligned).  The next tile's columns and records are copied
// asynchronously into the other buffers while the current tile is summed.
struct NcTileLayout {
    int TS;
    long long r1, wm, ww, floats;
    __host__ __device__ NcTileLayout(int nc, int T)
    {
        TS = T + 1;
        r1 = (long long)nc * TS;
        wm = (2 * r1 + 3) & ~3LL;
        ww = (wm + 2LL * (nc + 1) * TS + 3) & ~3LL;
        floats = ww + 8LL * T;
    }
};

__host__ __device__ inline long long nc_tile_bytes(int nc, int T)
{
    return 4 * NcTileLayout(nc, T).floats;
}

// The largest tile (pixels, a multiple of 32 in [32, 4096]) that fits.
__host__ __device__ inline int nc_tile_pixels(int nc, long long smem_bytes)
{
    long long t = smem_bytes / (16LL * nc + 40);
    t = t < 32 ? 32 : (t & ~31LL) > 4096 ? 4096 : (t & ~31LL);
    while (t > 32 && nc_tile_bytes(nc, (int)t) > smem_bytes) t -= 32;
    return (int)t;
}

// Sum s of the normal equations: s < nc(nc+1)/2 is A[a][e] (e >= a, row by
// row), then b_a for a = s - nc(nc+1)/2.
__device__ __forceinline__ void nc_sum_index(int nc, int s, int &a, int &e, bool &bsum)
{
    const int nA = nc * (nc + 1) / 2;
    bsum = s >= nA;
    if (bsum) {
        a = s - nA;
        e = a;
        return;
    }
    int rem = s;
    a = 0;
    while (rem >= nc - a) {
        rem -= nc - a;
        ++a;
    }
    e = a + rem;
}

// The normal equations as 2 x 2 blocks of an extended matrix: rows are the
// pair operands w M_0 .. w M_{nc-1} and w d (row nc), columns the blurred
// columns M_0 .. M_{nc-1}; A[a][e] (a <= e) is (row a, column e) and b_e is
// (row nc, column e).  Unit u is row block i (rows 2i, 2i + 1) by column
// block j (columns 2j, 2j + 1), for j >= i up to the row block holding row
// nc (i = nc/2), which takes every j.  Rows past nc and columns past nc - 1
// (odd counts) are read as the last valid one and their sums dropped, as is
// the block-diagonal entry below the diagonal.
__device__ __forceinline__ int nc_units(int nc)
{
    const int rb = nc >> 1, cb = (nc + 1) >> 1;
    return rb * cb - rb * (rb - 1) / 2 + cb;
}

// Unit u's rows r[0..1], columns c[0..1] (clamped to valid operands) and the
// sum index of each of its four entries (row k, column l) at s[2k + l], or
// -1 when dropped: A[a][e] is sum a nc - a (a - 1)/2 + e - a, b_e is sum
// nc (nc + 1)/2 + e.
__device__ __forceinline__ void nc_unit(int nc, int u, int *r, int *c, int *sx)
{
    const int rb = nc >> 1, cb = (nc + 1) >> 1;
    int i = 0, j = 0;
    for (i = 0; i < rb; ++i) {
        if (u < cb - i) { j = i + u; break; }
        u -= cb - i;
    }
    if (i == rb) j = u;
    const int nA = nc * (nc + 1) / 2;
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        r[k] = min(2 * i + k, nc);
        c[k] = min(2 * j + k, nc - 1);
    }
#pragma unroll
    for (int k = 0; k < 2; ++k)
#pragma unroll
        for (int l = 0; l < 2; ++l) {
            const int rk = 2 * i + k, cl = 2 * j + l;
            int idx = -1;
            if (rk <= nc && cl < nc) {
                if (rk == nc) idx = nA + cl;
                else if (rk <= cl) idx = rk * nc - rk * (rk - 1) / 2 + cl - rk;
            }
            sx[2 * k + l] = idx;
        }
}

// Unit unit's four sums (those with sx >= 0) accumulated over the pixels
// r, r + R, ... of every tile in double-float; FP64 partials to part[0..3].
// Every term is a float pair times a float, the product kept exact as a
// pair: A[a][e] takes (w M_a) M_e, b_e takes (w d) M_e, where the pairs
// w M_a are formed once per tile pixel from the staged columns.  Each pixel
// reads two pairs and two floats for four terms through running pointers.
// Every thread of the CTA takes part in the copies (unit < 0: no sums).
// Per tile: wait for its copies, barrier, start the next tile's copies, form
// the pairs, barrier, sum; a final barrier frees the shared memory.
__device__ __forceinline__ void nc_tile_sums22(const LensDev &L, const float *M, int nc, int unit,
                                               int r, int R, float *tile, int T, int tid,
                                               int nthr, double *part)
{
    const int npix = L.npix;
    const NcTileLayout lay(nc, T);
    const int TS = lay.TS;
    float2 *wm = reinterpret_cast<float2 *>(tile + lay.wm);
    float4 *ww = reinterpret_cast<float4 *>(tile + lay.ww);
    int rr[2], cc[2], sx[4];
    nc_unit(nc, max(unit, 0), rr, cc, sx);
    float hi[4], lo[4];
#pragma unroll
    for (int g = 0; g < 4; ++g) hi[g] = lo[g] = 0.0f;
    // copies of tile [p0, p0 + n) into buffer b: entry k = c n + i of the
    // columns, c = k / n by a multiply-high (exact as k n < 2^32: nc <= 32
    // columns of n <= 4096 pixels; nmul = ceil(2^32 / n) for n > 1, and
    // n = 1 takes c = k), then the n weight records
    auto issue = [&](int p0, int b) {
        const int n = min(T, npix - p0);
        const unsigned nmul = 0xffffffffu / (unsigned)n + 1u;
        float *Rb = tile + b * lay.r1;
        for (int k = tid; k < nc * n; k += nthr) {
            const int c = n > 1 ? (int)__umulhi((unsigned)k, nmul) : k, i = k - c * n;
            cp_async4(Rb + c * TS + i, M + (size_t)c * npix + p0 + i);
        }
        for (int i = tid; i < n; i += nthr) cp_async16(ww + b * T + i, L.wpack + p0 + i);
        cp_async_commit();
    };
    if (npix > 0) issue(0, 0);
    int b = 0;
    for (int p0 = 0; p0 < npix; p0 += T, b ^= 1) {
        const int n = min(T, npix - p0);
        cp_async_wait_all();
        __syncthreads();
        if (p0 + T < npix) issue(p0 + T, b ^ 1);
        const float *Rc = tile + b * lay.r1;
        const float4 *wc = ww + b * T;
        const unsigned nmul = 0xffffffffu / (unsigned)n + 1u;
        for (int k = tid; k < nc * n; k += nthr) {
            const int c = n > 1 ? (int)__umulhi((unsigned)k, nmul) : k, i = k - c * n;
            const float m = Rc[c * TS + i];
            const float4 w = wc[i];
            const float p1 = w.x * m;
            float e1 = fmaf(w.x, m, -p1);
            e1 = fmaf(w.y, m, e1);
            wm[c * TS + i] = make_float2(p1, e1);
        }
        for (int i = tid; i < n; i += nthr) {
            const float4 w = wc[i];
            wm[nc * TS + i] = make_float2(w.z, w.w);
        }
        __syncthreads();
        if (unit >= 0) {
            const float2 *q0 = wm + rr[0] * TS + r, *q1 = wm + rr[1] * TS + r;
            const float *f0 = Rc + cc[0] * TS + r, *f1 = Rc + cc[1] * TS + r;
#pragma unroll 2
            for (int i = r; i < n; i += R, q0 += R, q1 += R, f0 += R, f1 += R) {
                const float2 a = *q0, bq = *q1;
                const float x = *f0, y = *f1;
                float p, er;
                p = a.x * x; er = fmaf(a.x, x, -p); er = fmaf(a.y, x, er); df_acc(hi[0], lo[0], p, er);
                p = a.x * y; er = fmaf(a.x, y, -p); er = fmaf(a.y, y, er); df_acc(hi[1], lo[1], p, er);
                p = bq.x * x; er = fmaf(bq.x, x, -p); er = fmaf(bq.y, x, er); df_acc(hi[2], lo[2], p, er);
                p = bq.x * y; er = fmaf(bq.x, y, -p); er = fmaf(bq.y, y, er); df_acc(hi[3], lo[3], p, er);
            }
        }
    }
    __syncthreads();
#pragma unroll
    for (int g = 0; g < 4; ++g) part[g] = (double)hi[g] + (double)lo[g];
}

// -------------------------------------------------------------- FNNLS
// Warp-cooperative least squares on the passive set (mask bit i set:
// column i free) of the n x n system A x = b (row-major in shared memory,
// n <= 32): lane p owns row p of the compacted k x k matrix G in F (stride
// kMaxComps + 1); Cholesky G = L L^T column by column (the pivot lane takes
// the square root, every lane below it its own entry), then the two
// triangular solves with the solved entry broadcast by shuffle.  s (all
// lanes, registers: lane i holds s_i) gets the solution on the passive
// set and 0 elsewhere.  Returns false (all lanes) if a pivot is not
// positive.
__device__ inline bool nc_warp_solve(const double *A, const double *b, int n, unsigned P,
                                     double *F, int lane, double &s)
{
    const bool mine = lane < n && (P >> lane & 1u);
    const int k = __popc(P);
    const int p = __popc(P & ((1u << lane) - 1u));   // my compacted position
    // compacted rows: G[p][q] = A[lane][col of q]
    if (mine) {
        int q = 0;
        for (int c = 0; c < n; ++c)
            if (P >> c & 1u) F[p * (kMaxComps + 1) + q++] = A[lane * n + c];
    }
    __syncwarp();
    const double bp = mine ? b[lane] : 0.0;
    // Cholesky (lower): row p of L overwrites row p of G
    bool ok = true;
    for (int j = 0; j < k; ++j) {
        double v = 0.0;
        if (mine && p >= j) {
            v = F[p * (kMaxComps + 1) + j];
            for (int t = 0; t < j; ++t)
                v = fma(-F[p * (kMaxComps + 1) + t], F[j * (kMaxComps + 1) + t], v);
        }
        // the pivot first: from the lane holding compacted row j
        const int src = __ffs(__ballot_sync(0xffffffffu, mine && p == j)) - 1;
        const double piv2 = __shfl_sync(0xffffffffu, v, src);
        if (!(piv2 > 0.0)) { ok = false; break; }
        const double piv = sqrt(piv2);
        if (mine && p > j) F[p * (kMaxComps + 1) + j] = v / piv;
        if (mine && p == j) F[p * (kMaxComps + 1) + j] = piv;
        __syncwarp();
    }
    if (!ok) return false;
    // L y = b_P (forward), then L^T z = y (backward)
    double y = bp;
    for (int j = 0; j < k; ++j) {
        const int src = __ffs(__ballot_sync(0xffffffffu, mine && p == j)) - 1;
        double yj = 0.0;
        if (mine && p == j) yj = y / F[p * (kMaxComps + 1) + p];
        yj = __shfl_sync(0xffffffffu, yj, src);
        if (mine && p == j) y = yj;
        if (mine && p > j) y = fma(-F[p * (kMaxComps + 1) + j], yj, y);
    }
    double z = y;
    for (int j = k - 1; j >= 0; --j) {
        const int src = __ffs(__ballot_sync(0xffffffffu, mine && p == j)) - 1;
        double zj = 0.0;
        if (mine && p == j) zj = z / F[p * (kMaxComps + 1) + p];
        zj = __shfl_sync(0xffffffffu, zj, src);
        if (mine && p == j) z = zj;
        // row j of L^T is column j of L: L[q][j] for q > j sits in row q
        const double lij = (mine && p < j) ? F[j * (kMaxComps + 1) + p] : 0.0;
        if (mine && p < j) z = fma(-lij, zj, z);
    }
    s = mine ? z : 0.0;
    __syncwarp();
    return true;
}

// FNNLS (Bro & de Jong 1997): the Lawson-Hanson active-set method on the
// normal equations A x = b, x >= 0, run by one warp (lane i holds x_i, the
// gradient g_i and the solution s_i; n <= 32).  All columns start at zero;
// while a zero column has gradient g = b - A x above tol = 10 eps ||A||_1 n,
// the largest one is freed and the free set's least-squares solution s is
// taken, stepping back to the feasible boundary (freed columns that reach
// zero return to the zero set) while some free s_i <= 0.  A column whose own
// least-squares value comes out non-positive on entry is passed over until x
// next changes.  At most 30 n steps.  Lane i returns x_i.
__device__ inline double nc_fnnls_warp(const double *A, const double *b, int n, double *F,
                                       int lane)
{
    const bool in = lane < n;
    double cs = 0.0;
    if (in)
        for (int i = 0; i < n; ++i) cs += fabs(A[i * n + lane]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) cs = fmax(cs, __shfl_xor_sync(0xffffffffu, cs, o));
    const double tol = 10.0 * 2.220446049250313e-16 * cs * n;
    unsigned P = 0u, skip = 0u;
    double x = 0.0, g = in ? b[lane] : 0.0, s = 0.0;
    for (int step = 0; step < 30 * n; ++step) {
        // the largest gradient among zero, not-skipped columns (ties: lowest index)
        double gv = (in && !((P | skip) >> lane & 1u) && g > tol) ? g : -1.0;
        int gi = gv > 0.0 ? lane : 64;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const double ov = __shfl_xor_sync(0xffffffffu, gv, o);
            const int oi = __shfl_xor_sync(0xffffffffu, gi, o);
            if (ov > gv || (ov == gv && oi < gi)) { gv = ov; gi = oi; }
        }
        if (gi >= 64) break;
        P |= 1u << gi;
        bool ok = nc_warp_solve(A, b, n, P, F, lane, s);
        const double sj = __shfl_sync(0xffffffffu, s, gi);
        if (!ok || !(sj > 0.0)) {
            P &= ~(1u << gi);
            skip |= 1u << gi;
            continue;
        }
        for (int inner = 0; inner <= n; ++inner) {
            const bool neg = in && (P >> lane & 1u) && s <= 0.0;
            double al = neg ? x / (x - s) : 2.0;
            int ai = neg ? lane : 64;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                const double ov = __shfl_xor_sync(0xffffffffu, al, o);
                const int oi = __shfl_xor_sync(0xffffffffu, ai, o);
                if (ov < al || (ov == al && oi < ai)) { al = ov; ai = oi; }
            }
            if (ai >= 64) break;
            if (in) x = fma(al, s - x, x);
            if (lane == ai) x = 0.0;
            const unsigned drop = __ballot_sync(0xffffffffu, in && (P >> lane & 1u) && x <= 0.0);
            P &= ~drop;
            if (drop >> lane & 1u) x = 0.0;
            if (!nc_warp_solve(A, b, n, P, F, lane, s)) return x;
        }
        skip = 0u;
        x = s;
        // g = b - A x: lane i needs row i of A and every x_k
        double v = in ? b[lane] : 0.0;
        for (int c = 0; c < n; ++c) {
            const double xc = __shfl_sync(0xffffffffu, x, c);
            if (in) v = fma(-A[lane * n + c], xc, v);
        }
        g = v;
    }
    return x;
}

// --------------------------------------------------------------- kernels
// Static shared memory of the multi-column kernels: the normal equations,
// the Cholesky work space, the components' constants, the EPL series.
struct NcShared {
    double A[kMaxComps * kMaxComps], b[kMaxComps];
    double F[kMaxComps * (kMaxComps + 1)];
    float q[kMaxComps * 6];
    alignas(16) float epl[kEplMaxN + 1];
};

// FNNLS on the normal equations in sh (nc columns), chi^2 = dWd - 2 x^T b
// + x^T A x and log L (Eq. 5) to *outp; the amplitudes and log L also to
// wres when given.  One warp (all 32 lanes).
__device__ inline void nc_solve(NcShared &sh, int nc, double dWd, double lognorm, double *outp,
                                double *wres, int lane)
{
    const double x = nc_fnnls_warp(sh.A, sh.b, nc, sh.F, lane);
    double Ax = 0.0;
    for (int k = 0; k < nc; ++k) {
        const double xk = __shfl_sync(0xffffffffu, x, k);
        if (lane < nc) Ax = fma(sh.A[lane * nc + k], xk, Ax);
    }
    double term = lane < nc ? x * (Ax - 2.0 * sh.b[lane]) : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) term += __shfl_xor_sync(0xffffffffu, term, o);
    const double ll = -0.5 * (dWd + term) + lognorm;
    if (lane == 0) *outp = ll;
    if (wres) {
        if (lane < nc) wres[lane] = x;
        if (lane == 0) wres[nc] = ll;
    }
    __syncwarp();
}

// A vector whose normal equations wait in sh.A, sh.b for their solve: the
// CTA's last warp (the solver) takes it while the other warps trace and
// convolve the next vector (sh.A, sh.b are rewritten only by that vector's
// sums, after a full barrier), or after the CTA's last vector.  Written and
// read by the solver warp only.
constexpr int kDeferCols = 8;
struct NcPending {
    double dWd, lognorm;
    double *outp;
    int nc, valid;
};

__device__ __forceinline__ void nc_solve_pending(NcShared &sh, NcPending &pf, int lane)
{
    if (!pf.valid) return;
    nc_solve(sh, pf.nc, pf.dWd, pf.lognorm, pf.outp, nullptr, lane);
    if (lane == 0) pf.valid = 0;
    __syncwarp();
}

// One valid parameter vector of a multi-column lens (constant block kc):
// trace passes each followed by the PSF of its columns, normal equations,
// FNNLS; log L to *outp (and, when wres is given, the amplitudes and log L
// to wres).  U: the CTA's global slot (U [nc] binned columns, of which a
// pass uses the first ncp; M [nc + 1] blurred columns; H [2] images); spsf:
// the dynamic shared memory (band buffer or PSF taps, reused for the sums'
// tiles of T pixels).  Warps 0 .. nwarp-2 (the workers, named barrier 1)
// trace and convolve; meanwhile the last warp (the solver) runs the
// previous vector's FNNLS (pf); all warps form the sums.  With wres the
// solve is this vector's own, at the end.  Starts and ends with all threads
// in step.
template <int SUB, int K, int ROWS>
__device__ __forceinline__ void nc_vector(const LensDev &L, const MultiDev &M, const float *kc,
                                          double *outp, double *wres, float *U, float *spsf,
                                          NcShared &sh, NcPending &pf, bool skip, int T, int tid,
                                          int nthr)
{
    const int lane = tid & 31;
    const int nc = M.nc, npix = L.npix;
    // the solve is deferred to the solver warp from kDeferCols columns on
    // (below, FNNLS is cheap next to the warp's share of the trace)
    const bool defer = wres == nullptr && nc >= kDeferCols;
    const int nwk = defer ? nthr - 32 : nthr;   // worker threads
    float *Mb = U + (size_t)nc * npix;
    float *H = Mb + (size_t)(nc + 1) * npix;
    for (int t = tid; t < 6 * nc; t += nthr) sh.q[t] = kc[K_C0 + t];
    if (kc[K_EPL] != 0.0f)
        for (int t = tid; t <= kEplMaxN; t += nthr) sh.epl[t] = kc[K_EC0 + t];
    __syncthreads();
    // the previous vector's amplitudes and log L, when deferred (the last
    // warp; it then joins the workers unless this vector defers too)
    if (tid >= nthr - 32) nc_solve_pending(sh, pf, lane);
    if (tid < nwk) {
        // the workers: the sums of the previous vector used the dynamic
        // shared memory, so its zero halos (or the PSF taps) are set first
        setup_lens(L, spsf, tid, nwk);
        phase_sync<1>(nwk);
        // stage 2 ps: trace pass ps; stage 2 ps + 1: its convolutions (the
        // vector's constants live within a trace stage only, not through
        // the convolutions)
#pragma unroll 1
        for (int stage = 0; stage < 2 * M.npass; ++stage) {
          const int ps = stage >> 1;
          const int ncp = M.pass_n[ps];
          const int *chan = M.pass_comp[ps];
          const bool full = wres != nullptr;
          if (!(stage & 1)) {
            // 1. one trace pass: its ncp columns to U[0 .. ncp)
            const VecConst v = load_consts(kc);
            float cq[6 * kPassMax];
            int gmask = 0;
#pragma unroll
            for (int k = 0; k < kPassMax; ++k) {
                const int c = k < ncp ? M.pass_comp[ps][k] : 0;
#pragma unroll
                for (int e = 0; e < 6; ++e) cq[6 * k + e] = sh.q[6 * c + e];
                if (k < ncp && M.type[c] == COMP_GAUSS) gmask |= 1 << k;
            }
            // binned columns: the pass's own slots 0 .. ncp-1, or each
            // component's slot when the binned columns are written out
            if (M.pass_gauss[ps]) {
                if (M.pass_plane[ps] == PLANE_LENS)
                    trace_pass<SUB, 3, kPassMax, true>(L, v, kc, cq, gmask, ncp, chan, full, U, tid, nwk, sh.epl, skip);
                else if (v.epl)
                    trace_pass<SUB, 2, kPassSrcG, true>(L, v, kc, cq, gmask, ncp, chan, full, U, tid, nwk, sh.epl, skip);
                else if (v.fast)
                    trace_pass<SUB, 0, kPassSrcG, true>(L, v, kc, cq, gmask, ncp, chan, full, U, tid, nwk, sh.epl, skip);
                else if (v.mid)
                    trace_pass<SUB, 4, kPassSrcG, true>(L, v, kc, cq, gmask, ncp, chan, full, U, tid, nwk, sh.epl, skip);
                else
                    trace_pass<SUB, 1, kPassSrcG, true>(L, v, kc, cq, gmask, ncp, chan, full, U, tid, nwk, sh.epl, skip);
            } else {
                if (M.pass_plane[ps] == PLANE_LENS)
                    trace_pass<SUB, 3, kPassMix, false>(L, v, kc, cq, gmask, ncp, chan, full, U, tid, nwk, sh.epl, skip);
                else if (v.epl)
                    trace_pass<SUB, 2, kPassMix, false>(L, v, kc, cq, gmask, ncp, chan, full, U, tid, nwk, sh.epl, skip);
                else if (v.fast)
                    trace_pass<SUB, 0, kPassMix, false>(L, v, kc, cq, gmask, ncp, chan, full, U, tid, nwk, sh.epl, skip);
                else if (v.mid)
                    trace_pass<SUB, 4, kPassMix, false>(L, v, kc, cq, gmask, ncp, chan, full, U, tid, nwk, sh.epl, skip);
                else
                    trace_pass<SUB, 1, kPassMix, false>(L, v, kc, cq, gmask, ncp, chan, full, U, tid, nwk, sh.epl, skip);
            }
            phase_sync<1>(nwk);
            continue;
          }
            // 2. the pass's columns through the PSF two at a time (an odd
            //    last one pairs with itself), blurred to M[chan[k]]: the
            //    binned columns are read back while they are still in L2
            for (int k = 0; k < ncp; k += 2) {
                const int k2 = min(k + 1, ncp - 1);
                const float *Il = U + (size_t)(full ? chan[k] : k) * npix;
                const float *Is = U + (size_t)(full ? chan[k2] : k2) * npix;
                float *Ml = Mb + (size_t)chan[k] * npix, *Ms = Mb + (size_t)chan[k2] * npix;
                if constexpr (K > 0) {
                    const int h = L.h, W = L.W, HL = L.HL, ny = L.ny, nx = L.nx;
                    const int step = L.band_rows;
                    float *Pl = spsf, *Ps = spsf + (step + 2 * h + kCR) * W;
                    PairStore<ROWS> st{Ml, Ms};
                    for (int b0 = 0; b0 < ny; b0 += step) {
                        const int nrows = min(step, ny - b0);
                        const int nbr = nrows + 2 * h;
                        stage_band(L, Il, Is, Pl, (int)(Ps - Pl), b0, nbr, tid, nwk);
                        phase_sync<1>(nwk);
                        if (L.sep)
                            conv_sep_band<K, PairStore<ROWS>, 1>(L, Pl, Ps, b0, nrows,
                                                                max(0, h - b0),
                                                                min(nbr, ny - b0 + h), tid, nwk,
                                                                st);
                        else
                            conv_direct_band<K>(L, Pl, Ps, b0, nrows, tid, nwk, st);
                        phase_sync<1>(nwk);
                    }
                } else {
                    RunArgs ra = {};
                    ra.wr_blurred = Ml;
                    ra.wr_blurred_s = Ms;
                    float dummy[10];
                    // (its five sums go unused)
                    conv_generic<true, 1>(L, ra, spsf, const_cast<float *>(Il),
                                          const_cast<float *>(Is), H, H + npix, dummy, tid, nwk,
                                          false);
                    phase_sync<1>(nwk);
                }
            }
        }
    }
    __syncthreads();
    // 3. normal equations through shared-memory tiles (the dynamic shared
    //    memory is free again once the convolution is done): thread
    //    (unit, r) takes a 2 x 2 block of sums (nc_unit) over pixel phase r
    //    of RP; the FP64 partials go to the same space after the last tile
    //    ([RP][S]), then are added in a fixed order
    {
        const int S = nc * (nc + 1) / 2 + nc;
        const long long cap = (long long)L.nc_smem / (long long)sizeof(double);
        const int NU = nc_units(nc);
        int RP = max(1, nthr / NU);
        while (RP > 1 && (long long)RP * S > cap) --RP;
        const int r = tid / NU;
        const int unit = r < RP ? tid - r * NU : -1;
        double part[4];
        nc_tile_sums22(L, Mb, nc, unit, r, RP, spsf, T, tid, nthr, part);
        double *parts = reinterpret_cast<double *>(spsf);
        if (unit >= 0) {
            int rr[2], cc[2], sx[4];
            nc_unit(nc, unit, rr, cc, sx);
#pragma unroll
            for (int g = 0; g < 4; ++g)
                if (sx[g] >= 0) parts[(size_t)r * S + sx[g]] = part[g];
        }
        __syncthreads();
        for (int t = tid; t < S; t += nthr) {
            double sum = 0.0;
            for (int q = 0; q < RP; ++q) sum += parts[(size_t)q * S + t];
            int a, e;
            bool bsum;
            nc_sum_index(nc, t, a, e, bsum);
            if (bsum) {
                sh.b[a] = sum;
            } else {
                sh.A[a * nc + e] = sum;
                sh.A[e * nc + a] = sum;
            }
        }
    }
    __syncthreads();
    // 4. amplitudes and log L: deferred to the solver during the next
    //    vector, or now (the last warp)
    if (tid >= nthr - 32) {
        if (defer) {
            if (lane == 0) pf = NcPending{L.dWd, L.lognorm, outp, nc, 1};
            __syncwarp();
        } else {
            nc_solve(sh, nc, L.dWd, L.lognorm, outp, wres, lane);
        }
    }
    __syncthreads();
}

// One lens: persistent CTAs over the batch.  Dynamic shared memory: K > 0,
// the padded band buffer of the compiled convolution (2 channels x
// (band_rows + 2h + kCR) rows x W); K == 0, the PSF taps of the generic
// convolution; at least the sums' smallest tile either way.
template <int SUB, int K>
__global__ void __launch_bounds__(kThreads)
k_loglike_nc(const __grid_constant__ LensDev L, const __grid_constant__ MultiDev M,
             const __grid_constant__ NcArgs R)
{
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ NcShared sh;
    __shared__ NcPending spf;
    const int tid = threadIdx.x, nthr = blockDim.x;
    const int nc = M.nc, npix = L.npix;
    float *spsf = reinterpret_cast<float *>(smem);
    float *U = R.gscr + (size_t)blockIdx.x * R.gslot;
    if (tid == 0) spf.valid = 0;
    setup_lens(L, spsf, tid, nthr);
    // pixels never traced (masked lenses) must start finite
    if (L.tlist)
        for (int t = tid; t < nc * npix; t += nthr) U[t] = 0.0f;
    __syncthreads();
    const bool skip = R.wr_res == nullptr;   // model columns: every pixel
    const int T = nc_tile_pixels(nc, (long long)L.nc_smem);
    for (int b = blockIdx.x; b < R.B; b += gridDim.x) {
        const float *kc = R.kc + (size_t)b * NCONST;
        if (kc[K_VALID] == 0.0f) {
            if (tid == 0) {
                R.out[b] = -INFINITY;
                if (R.wr_res) R.wr_res[nc] = -INFINITY;
            }
            continue;
        }
        // two output rows per direct-convolution item up to K = 21 (above,
        // the longer windows would spill); one in the multi-lens kernel
        nc_vector<SUB, K, (K <= 21 ? 2 : 1)>(L, M, kc, R.out + b, R.wr_res, U, spsf, sh, spf,
                                             skip, T, tid, nthr);
    }
    if (tid >= nthr - 32) nc_solve_pending(sh, spf, tid & 31);
}

// Many lenses (the batcher's multi-column groups): at most kMultiSlots
// lenses per launch, their descriptors and component lists in the launch's
// parameters (LensSlots) read through the slot index where they are used;
// each CTA starts on its home slot and then takes the following ones in
// turn, every slot's vectors handed out by its counter (as
// k_loglike_multi).
template <int SUB, int K>
__global__ void __launch_bounds__(kThreads) k_loglike_nc_multi(const __grid_constant__ MultiArgs A,
                                                               int group,
                                                               const __grid_constant__ LensSlots S)
{
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ NcShared sh;
    __shared__ NcPending spf;
    // the vector in hand and its output, in shared memory (tid 0 writes
    // them between barriers) so that they take no registers across a vector
    __shared__ int s_t;
    __shared__ double *s_out;
    const int tid = threadIdx.x, nthr = blockDim.x;
    if (tid == 0) spf.valid = 0;
    float *spsf = reinterpret_cast<float *>(smem);
    int home = 0;
    while (home < S.n - 1 && (int)blockIdx.x >= S.cta_end[home]) ++home;
    for (int k = 0; k < S.n; ++k) {
        int s0 = home + k;
        if (s0 >= S.n) s0 -= S.n;
        for (bool ready = false;; ready = true) {
            // the slot index made opaque for each vector: with it fixed for
            // the whole slot the compiler keeps lens fields in registers
            // across nc_vector and spills (736 B of spill stores, 1344 B of
            // loads per thread, against 60 and 100 this way)
            int s = s0;
            asm volatile("" : "+r"(s));
            const LensDev &L = S.lens[s];
            const MultiDev &M = S.md[s];
            if (tid == 0) {
                const int i = atomicAdd(A.counter + kMultiCounters + group * kMultiSlots + s, 1);
                const int t = i < S.count[s] ? S.first[s] + i : -1;
                s_t = t;
                if (t >= 0) {
                    const MultiHdr hd = A.groups[group];
                    const Segment &sg = A.segs[find_segment(A.segs, hd.seg0, hd.nseg, t)];
                    s_out = sg.out + (t - sg.first);
                }
            }
            __syncthreads();
            const int t = s_t;
            if (t < 0) break;
            float *U = A.gscr + (size_t)blockIdx.x * A.gslot_floats;
            if (!ready) {
                // the slot's lens in the CTA's shared memory; pixels never
                // traced (masked lenses) start finite
                setup_lens(L, spsf, tid, nthr);
                if (L.tlist)
                    for (int q = tid; q < M.nc * L.npix; q += nthr) U[q] = 0.0f;
                __syncthreads();
            }
            const float *kc = A.kc + (size_t)t * NCONST;
            if (kc[K_VALID] == 0.0f) {
                if (tid == 0) *s_out = -INFINITY;
            } else {
                nc_vector<SUB, K, 1>(L, M, kc, s_out, nullptr, U, spsf, sh, spf, true,
                                     nc_tile_pixels(M.nc, (long long)L.nc_smem), tid, nthr);
            }
            // every thread has read s_t and s_out before tid 0 rewrites them
            __syncthreads();
        }
    }
    if (tid >= nthr - 32) nc_solve_pending(sh, spf, tid & 31);
}

using NcKernel = void (*)(const LensDev, const MultiDev, const NcArgs);

// Kernels of one translation unit; nullptr when (sub, K) is not in it.
struct KernelSet {
    SingleKernel (*single)(int sub, int K, bool write);
    MultiKernel (*multi)(int sub, int K);
    NcKernel (*nc)(int sub, int K);
    MultiKernel (*nc_multi)(int sub, int K);
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

template <int K>
inline MultiKernel nc_multi_for(int sub)
{
    switch (sub_class(sub)) {
        case 4: return k_loglike_nc_multi<4, K>;
        case 5: return k_loglike_nc_multi<5, K>;
        default: return k_loglike_nc_multi<0, K>;
    }
}

}  // namespace tll
