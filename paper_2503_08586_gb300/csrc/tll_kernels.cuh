// tll_kernels.cuh -- the likelihood kernels (templates).  Included by the
// tll_kern_*.cu translation units, each of which instantiates the kernels
// for a few PSF sides K (the compiled convolutions are specialised per K),
// so the kernels compile in parallel; the host finds them through the
// registry at the end of this file.
#pragma once

#include <math.h>

#include "tll_core.cuh"

namespace tll {

// Amplitudes and log L from the five sums (thread-local, FP64).
// NNLS over two columns: the optimum is the unconstrained minimiser of one
// face {none, lens only, source only, both} that is feasible; chi^2 of a
// face's minimiser s is dWd - s^T b.  Fixed mode: s = (I_e^L, I_e^S) and
// chi^2 = dWd - 2 s^T b + s^T A s.
__device__ __forceinline__ void finish_core(int mode, double dWd, double lognorm,
                                            const double *S, float IeL, float IeS,
                                            double *sl_o, double *ss_o, double *ll_o)
{
    const double All = S[0], Als = S[1], Ass = S[2], bl = S[3], bs = S[4];
    double sl, ss, chi2;
    if (mode == TLL_AMP_FIXED) {
        sl = IeL;
        ss = IeS;
        chi2 = dWd - 2.0 * (sl * bl + ss * bs) + sl * sl * All +
               2.0 * sl * ss * Als + ss * ss * Ass;
    } else {
        sl = 0.0; ss = 0.0; chi2 = dWd;
        if (All > 0.0 && bl > 0.0) {
            const double c = dWd - bl * (bl / All);
            if (c < chi2) { chi2 = c; sl = bl / All; ss = 0.0; }
        }
        if (Ass > 0.0 && bs > 0.0) {
            const double c = dWd - bs * (bs / Ass);
            if (c < chi2) { chi2 = c; sl = 0.0; ss = bs / Ass; }
        }
        // Both columns free only when they are not collinear to rounding:
        // det / (A_ll A_ss) = 1 - rho^2 must exceed the sums' rounding
        // (~1e-14) by a wide margin; collinear columns reach their optimum
        // on a single-column face.  The candidate's chi^2 is the full
        // quadratic form, exact for any s given A and b.
        const double det = All * Ass - Als * Als;
        if (det > 1e-9 * All * Ass) {
            const double tl = (Ass * bl - Als * bs) / det;
            const double ts = (All * bs - Als * bl) / det;
            if (tl > 0.0 && ts > 0.0) {
                const double c = dWd - 2.0 * (tl * bl + ts * bs) + tl * tl * All +
                                 2.0 * tl * ts * Als + ts * ts * Ass;
                if (c < chi2) { chi2 = c; sl = tl; ss = ts; }
            }
        }
    }
    *sl_o = sl;
    *ss_o = ss;
    *ll_o = -0.5 * chi2 + lognorm;
}

__device__ __forceinline__ void finish_vector(const LensDev &L, const double *S,
                                              float IeL, float IeS, double *sl_o,
                                              double *ss_o, double *ll_o)
{
    finish_core(L.mode, L.dWd, L.lognorm, S, IeL, IeS, sl_o, ss_o, ll_o);
}

// The five sums of a vector from the warps' double-float partials
// sred[w*5 + k] (w < nwarp): one warp adds them as a double-float butterfly
// over its lanes (every lane ends with the same bits) and converts each sum
// to FP64 once; called by all 32 lanes of that warp.  (FP64 runs at a small
// fraction of the FP32 rate here, so the partials stay float pairs until
// the end.)
__device__ __forceinline__ void block_sums(const float2 *sred, int nwarp, int lane, double *S)
{
    float a[10];
#pragma unroll
    for (int k = 0; k < 5; ++k) {
        const float2 v = lane < nwarp ? sred[lane * 5 + k] : make_float2(0.0f, 0.0f);
        a[2 * k] = v.x;
        a[2 * k + 1] = v.y;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
        for (int k = 0; k < 5; ++k) {
            const float oh = __shfl_xor_sync(0xffffffffu, a[2 * k], o);
            const float ol = __shfl_xor_sync(0xffffffffu, a[2 * k + 1], o);
            df_add_sym(a[2 * k], a[2 * k + 1], oh, ol);
        }
    }
#pragma unroll
    for (int k = 0; k < 5; ++k) S[k] = (double)a[2 * k] + (double)a[2 * k + 1];
}

// The amplitude solve and log L of a vector whose five sums wait in sred
// (the warps' partials of the last convolution): deferred to the CTA's last
// warp, which takes it at the start of the next vector's trace (its sums
// stay in sred until that vector's convolution, after the trace barrier) or
// after the CTA's last vector.  The last warp traces the fewest pixels when
// the threads do not divide them evenly, so the other warps never wait for
// the FP64 solve.  Record written and read by that warp only.
struct PendingFinish {
    double dWd, lognorm;
    double *outp;
    float IeL, IeS;
    int mode, valid;
};

__device__ __forceinline__ void finish_pending(PendingFinish &pf, const float2 *sred,
                                               int lane, int nwarp)
{
    if (!pf.valid) return;
    double S[5];
    block_sums(sred, nwarp, lane, S);
    if (lane == 0) {
        double sl, ss, ll;
        finish_core(pf.mode, pf.dWd, pf.lognorm, S, pf.IeL, pf.IeS, &sl, &ss, &ll);
        *pf.outp = ll;
        pf.valid = 0;
    }
    __syncwarp();
}

// --------------------------------------------------------- trace phase
// Ray-trace + light on the s x s subpixels of every pixel, mean-binned:
// pixel (i, j) of the lens / source image goes to Il / Is [i*stride + off + j].
// Subpixel (J, I) of the supersampled grid has exact integer-or-half
// offsets (fj, fi) = (J - JCX, I - JCY) from the grid centre; every
// coordinate is an affine function of them (see decode_vector).
// MODE: 0 SIE fast form, 1 SIE general form, 2 EPL (series coefficients ec),
// 4 SIE mid form, 5 EPL (the series' table at ec).
// skip: trace only the lens's listed pixels (L.tlist), those within the PSF's
// reach of an unmasked pixel; the others keep whatever finite value they
// hold, which only ever meets a zero weight.
template <int SUB, int MODE>
__device__ __forceinline__ void trace_image(const LensDev &L, const VecConst &v, const float *kc,
                                            float *Il, float *Is, int stride, int off,
                                            int tid, int nthr, const float *ec, bool skip)
{
    const int sub = SUB > 0 ? SUB : L.sub;
    const int nx = L.nx;
    const int *list = skip ? L.tlist : nullptr;
    const int n = list ? L.ntrace : L.npix;
    for (int t = tid; t < n; t += nthr) {
        const int pix = list ? list[t] : t;
        const int i = div_nx(L, pix), j = pix - i * nx;
        const float fj0 = (float)(j * sub) - L.JCX;
        const float fi0 = (float)(i * sub) - L.JCY;
        const PixLo lc = load_pixlo(kc);
        PixelLo lo;
        source_lo(lc, fj0, fi0, lo.nlx, lo.nly);
        const PixOrigin po = pixel_origin(v, lc, fj0, fi0);
        float accl, accs;
        subpixel_first<MODE>(v, lc, row_terms(v, po, fi0), fj0, ec, lo, accl, accs);
        float fi = fi0;
#pragma unroll
        for (int a = 0; a < (SUB > 0 ? SUB : sub); ++a, fi += 1.0f) {
            const RowTerms r = row_terms(v, po, fi);
#pragma unroll
            for (int c = 0; c < (SUB > 0 ? SUB : 1); ++c) {
                for (int cr = 0; cr < (SUB > 0 ? 1 : sub); ++cr) {
                    if (a == 0 && c == 0 && cr == 0) continue;   // the first, done above
                    float il, is;
                    subpixel<MODE>(v, r, fj0 + (float)(SUB > 0 ? c : cr), ec, lo, il, is);
                    accl += il;
                    accs += is;
                }
            }
        }
        Il[i * stride + off + j] = accl * L.inv_s2;
        Is[i * stride + off + j] = accs * L.inv_s2;
    }
}

// ------------------------------------------------ generic convolution
// Any PSF side, images unpadded with row stride nx (in shared memory, with
// the row pass in place, or in a global scratch slot with separate H
// buffers).  Separable: H(i,j) = sum_c v[c] I(i, j+h-c), then
// m(i,j) = sum_r u[r] H(i+h-r, j); direct: m = sum_{r,c} K[r][c] I(i+h-r, j+h-c);
// zero outside the image (Eq. 3).  Each output pixel's (m_l, m_s) goes to
// accum_pixel.
template <bool WRITE, int BAR = 0>
__device__ __forceinline__ void conv_generic(const LensDev &L, const RunArgs &R,
                                             const float *spsf, float *Il, float *Is,
                                             float *Hl, float *Hs, float *acc, int tid,
                                             int nthr, bool INPLACE)
{
    const int K = L.K, h = L.h, nx = L.nx, ny = L.ny, npix = L.npix;
    const int lane = tid & 31, warp = tid >> 5, nwarp = nthr >> 5;
    if (L.sep) {
        const float *su = spsf, *sv = spsf + K;
        for (int row = warp; row < 2 * ny; row += nwarp) {
            const float *src = row < ny ? Il + row * nx : Is + (row - ny) * nx;
            float *dst = row < ny ? Hl + row * nx : Hs + (row - ny) * nx;
            if (INPLACE) {
                float o[kHMax];
#pragma unroll
                for (int q = 0; q < kHMax; ++q) {
                    const int j = lane + 32 * q;
                    float sacc = 0.0f;
                    if (j < nx) {
                        const int c0 = max(0, j + h - nx + 1), c1 = min(K - 1, j + h);
                        for (int c = c0; c <= c1; ++c) sacc = fmaf(sv[c], src[j + h - c], sacc);
                    }
                    o[q] = sacc;
                }
                __syncwarp();
#pragma unroll
                for (int q = 0; q < kHMax; ++q) {
                    const int j = lane + 32 * q;
                    if (j < nx) dst[j] = o[q];
                }
                __syncwarp();
            } else {
                for (int j = lane; j < nx; j += 32) {
                    const int c0 = max(0, j + h - nx + 1), c1 = min(K - 1, j + h);
                    float sacc = 0.0f;
                    for (int c = c0; c <= c1; ++c) sacc = fmaf(sv[c], src[j + h - c], sacc);
                    dst[j] = sacc;
                }
            }
        }
        phase_sync<BAR>(nthr);
        const int nb = max(1, nthr / nx);
        const int rb = (ny + nb - 1) / nb;
        for (int it = tid; it < nx * nb; it += nthr) {
            const int j = it % nx, band = it / nx;
            const int r0 = band * rb, r1 = min(ny, r0 + rb);
            for (int i = r0; i < r1; ++i) {
                const int q0 = max(0, i + h - ny + 1), q1 = min(K - 1, i + h);
                float ml = 0.0f, ms = 0.0f;
                for (int r = q0; r <= q1; ++r) {
                    const int o = (i + h - r) * nx + j;
                    ml = fmaf(su[r], Hl[o], ml);
                    ms = fmaf(su[r], Hs[o], ms);
                }
                const int pix = i * nx + j;
                if (WRITE) {
                    R.wr_blurred[pix] = ml;
                    (R.wr_blurred_s ? R.wr_blurred_s : R.wr_blurred + npix)[pix] = ms;
                }
                accum_pixel(ml, ms, L.wpack[pix], acc);
            }
        }
    } else {
        for (int pix = tid; pix < npix; pix += nthr) {
            const int i = pix / nx, j = pix - i * nx;
            const int r0 = max(0, i + h - ny + 1), r1 = min(K - 1, i + h);
            const int c0 = max(0, j + h - nx + 1), c1 = min(K - 1, j + h);
            float ml = 0.0f, ms = 0.0f;
            for (int r = r0; r <= r1; ++r) {
                const float *kr = spsf + r * K;
                const int base = (i + h - r) * nx + j + h;
                float rl = 0.0f, rs = 0.0f;
                for (int c = c0; c <= c1; ++c) {
                    rl = fmaf(kr[c], Il[base - c], rl);
                    rs = fmaf(kr[c], Is[base - c], rs);
                }
                ml += rl;
                ms += rs;
            }
            if (WRITE) {
                R.wr_blurred[pix] = ml;
                (R.wr_blurred_s ? R.wr_blurred_s : R.wr_blurred + npix)[pix] = ms;
            }
            accum_pixel(ml, ms, L.wpack[pix], acc);
        }
    }
}

// Both compiled convolutions work on a zero-padded band buffer: per
// channel, buffer row br holds image row b0 - h + br (zeros outside the
// image), interior column j at buffer column HL + j, zeros elsewhere; the
// s channel follows the l channel at Ps.  Outputs are image rows
// [b0, b0 + nrows); each output pixel's (m_l, m_s) goes to accum_pixel.

// Separable: row pass in place over buffer rows [rlo, rhi) (a lane makes
// 4 adjacent outputs from one float4 window), then the column pass (a lane
// makes kCR rows of its column from one window) fused with the sums.
// Output sinks of the compiled convolutions: SumsSink adds each output
// pixel's pair to the five weighted sums (the fused reduction); PairStore
// writes the pair to two images (the multi-column path).  kRows: output
// rows per item of the direct convolution -- two (each window read feeds
// twice the outputs) where the registers allow it, one where the sink's
// accumulators or the kernel's other live state would spill.
struct SumsSink {
    static constexpr int kRows = 1;
    const LensDev &L;
    float a[10];
    __device__ __forceinline__ void operator()(int pix, float ml, float ms)
    {
        accum_pixel(ml, ms, L.wpack[pix], a);
    }
};
template <int ROWS>
struct PairStore {
    static constexpr int kRows = ROWS;
    float *ol, *os;
    __device__ __forceinline__ void operator()(int pix, float ml, float ms)
    {
        ol[pix] = ml;
        os[pix] = ms;
    }
};

// Column pass of the separable convolution: thread unit u = (column j,
// row block rb) makes output rows [CR rb, CR rb + CR) of column j in both
// channels from one window of CR + K - 1 buffer rows (lanes of a warp hold
// consecutive columns: conflict-free shared-memory reads).
template <int K, int CR, class Sink>
__device__ __forceinline__ void conv_sep_cols(const LensDev &L, const float *Pl,
                                              const float *Ps, int b0, int nrows, int tid,
                                              int nthr, Sink &sink)
{
    using G = PadGeom<K>;
    static_assert(CR <= kCR, "the padded layout keeps kCR rows below the image");
    const int nx = L.nx, W = L.W;
    const int nrb = (nrows + CR - 1) / CR;
    for (int u = tid; u < nx * nrb; u += nthr) {
        const int rb = div_nx(L, u), j = u - rb * nx, r0 = rb * CR;
        float ml[CR], ms[CR];
#pragma unroll
        for (int ch = 0; ch < 2; ++ch) {
            const float *col = (ch == 0 ? Pl : Ps) + r0 * W + G::HL + j;
            float win[CR + K - 1];
#pragma unroll
            for (int t = 0; t < CR + K - 1; ++t) win[t] = col[t * W];
#pragma unroll
            for (int r = 0; r < CR; ++r) {
                float a = 0.0f;
#pragma unroll
                for (int c = 0; c < K; ++c) a = fmaf(L.tu[c], win[r + K - 1 - c], a);
                if (ch == 0) ml[r] = a; else ms[r] = a;
            }
        }
#pragma unroll
        for (int r = 0; r < CR; ++r)
            if (r0 + r < nrows) sink((b0 + r0 + r) * nx + j, ml[r], ms[r]);
    }
}

// Band staging: buffer rows [0, nbr) of both channels (Ps = Pl + off_s)
// <- image rows [b0 - h, b0 - h + nbr) of Il / Is, rows outside the image
// as zero.  The images sit in global memory (L2, or DRAM once evicted):
// every element is an asynchronous copy, so a band costs about one memory
// round trip.  Entry t = (channel, buffer row, column) flattened; its row is
// t / nx by a multiply-high where nx > 1 and t nx < 2^32 (exact there:
// nx_mul = ceil(2^32 / nx)), else by a division.  Ends with the thread's own
// copies complete; no barrier.
__device__ __forceinline__ void stage_band(const LensDev &L, const float *Il, const float *Is,
                                           float *Pl, int off_s, int b0, int nbr, int tid,
                                           int nthr)
{
    const int nx = L.nx, ny = L.ny, W = L.W, HL = L.HL, r0 = b0 - L.h;
    const int tot = 2 * nbr * nx;
    const bool fast = nx > 1 && (unsigned long long)tot * (unsigned)nx < (1ULL << 32);
    for (int t = tid; t < tot; t += nthr) {
        const int row = fast ? (int)__umulhi((unsigned)t, L.nx_mul) : t / nx;
        const int j = t - row * nx;
        const int ch = row >= nbr ? 1 : 0;
        const int br = row - ch * nbr, ir = r0 + br;
        const bool in = ir >= 0 && ir < ny;
        cp_async4_zfill(Pl + ch * off_s + br * W + HL + j, (ch ? Is : Il) + (in ? ir * nx + j : 0),
                        in);
    }
    cp_async_wait_all();
}

template <int K, class Sink, int BAR = 0>
__device__ __forceinline__ void conv_sep_band(const LensDev &L, float *Pl, float *Ps,
                                              int b0, int nrows, int rlo, int rhi, int tid,
                                              int nthr, Sink &sink)
{
    using G = PadGeom<K>;
    const int nx = L.nx, W = L.W;
    const int lane = tid & 31, warp = tid >> 5, nwarp = nthr >> 5;
    const int ngroups = (nx + 3) >> 2;
    const int nr = rhi - rlo;
    // row pass, in place; each lane holds at most 2 groups (nx <= 256)
    for (int row = warp; row < 2 * nr; row += nwarp) {
        float *P = (row < nr ? Pl + (rlo + row) * W : Ps + (rlo + row - nr) * W);
        float o[2][4];
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            const int g = lane + 32 * q;
            if (g < ngroups) {
                float win[4 * G::NW];
                const float4 *src = reinterpret_cast<const float4 *>(P + 4 * g);
#pragma unroll
                for (int k = 0; k < G::NW; ++k) {
                    const float4 v4 = src[k];
                    win[4 * k] = v4.x; win[4 * k + 1] = v4.y;
                    win[4 * k + 2] = v4.z; win[4 * k + 3] = v4.w;
                }
#pragma unroll
                for (int r = 0; r < 4; ++r) {
                    float a = 0.0f;
#pragma unroll
                    for (int c = 0; c < K; ++c) a = fmaf(L.tv[c], win[G::D + K - 1 + r - c], a);
                    o[q][r] = a;
                }
            }
        }
        __syncwarp();
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            const int g = lane + 32 * q;
            if (g < ngroups) {
                float *dst = P + G::HL + 4 * g;
                if (4 * g + 3 < nx) {
                    *reinterpret_cast<float4 *>(dst) = make_float4(o[q][0], o[q][1], o[q][2], o[q][3]);
                } else {
#pragma unroll
                    for (int r = 0; r < 4; ++r)
                        if (4 * g + r < nx) dst[r] = o[q][r];
                }
            }
        }
        __syncwarp();
    }
    phase_sync<BAR>(nthr);
    // column pass with the fused weighted sums: output row ro (image row
    // b0 + ro) reads buffer rows ro .. ro + K - 1; (column, row block)
    // units spread over every thread of the CTA, CR rows per unit
    const int nu4 = nx * ((nrows + 3) / 4), nu5 = nx * ((nrows + 4) / 5);
    if (((nu5 + nthr - 1) / nthr) * 5 < ((nu4 + nthr - 1) / nthr) * 4)
        conv_sep_cols<K, 5>(L, Pl, Ps, b0, nrows, tid, nthr, sink);
    else
        conv_sep_cols<K, 4>(L, Pl, Ps, b0, nrows, tid, nthr, sink);
}

// Direct K x K convolution (any PSF), m(i,j) = sum_{r,c} K[r][c]
// I(i+h-r, j+h-c), summed per PSF row.  A thread makes 4 adjacent outputs
// of two adjacent rows: each buffer row's float4 window is read once and
// meets PSF row r for the upper output row and row r + 1 for the lower one,
// so a window feeds 8 outputs (half the shared-memory reads of one row at a
// time); taps come from the parameter block in pairs.
//
// direct_window: one window (buffer row `row`, columns from 4g) applied
// with the K taps of PSF row t0 to the upper outputs (R0) and of row t1 to
// the lower ones (R1), each as a partial sum added to o0 / o1.
template <int K, bool R0, bool R1>
__device__ __forceinline__ void direct_window(const float *row, const float *t0,
                                              const float *t1, float (&o0)[4], float (&o1)[4])
{
    using G = PadGeom<K>;
    float win[4 * G::NW];
    const float4 *src = reinterpret_cast<const float4 *>(row);
#pragma unroll
    for (int k = 0; k < G::NW; ++k) {
        const float4 v4 = src[k];
        win[4 * k] = v4.x; win[4 * k + 1] = v4.y;
        win[4 * k + 2] = v4.z; win[4 * k + 3] = v4.w;
    }
    const float2 *p0 = reinterpret_cast<const float2 *>(t0);
    const float2 *p1 = reinterpret_cast<const float2 *>(t1);
    float a[4] = {0.0f, 0.0f, 0.0f, 0.0f}, b[4] = {0.0f, 0.0f, 0.0f, 0.0f};
#pragma unroll
    for (int c2 = 0; c2 < (K + 1) / 2; ++c2) {
        const float2 u = R0 ? p0[c2] : make_float2(0.0f, 0.0f);
        const float2 w = R1 ? p1[c2] : make_float2(0.0f, 0.0f);
#pragma unroll
        for (int e = 0; e < 2; ++e) {
            const int c = 2 * c2 + e;
            if (c < K) {
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const float x = win[G::D + K - 1 + q - c];
                    if (R0) a[q] = fmaf(e ? u.y : u.x, x, a[q]);
                    if (R1) b[q] = fmaf(e ? w.y : w.x, x, b[q]);
                }
            }
        }
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        if (R0) o0[q] += a[q];
        if (R1) o1[q] += b[q];
    }
}

template <int K, class Sink>
__device__ __forceinline__ void conv_direct_band(const LensDev &L, const float *Pl,
                                                 const float *Ps, int b0, int nrows, int tid,
                                                 int nthr, Sink &sink)
{
    constexpr int TS = tap_stride(K), ROWS = Sink::kRows;
    const int nx = L.nx, W = L.W;
    const int ngroups = (nx + 3) >> 2, nitems = (nrows + ROWS - 1) / ROWS;
    for (int item = tid; item < nitems * ngroups; item += nthr) {
        const int rb = item / ngroups, g = item - rb * ngroups, ro = ROWS * rb;
        float m[2][ROWS][4];   // [channel][row][column]
#pragma unroll
        for (int ch = 0; ch < 2; ++ch) {
            // output row ro + k (image row b0 + ro + k) meets buffer row
            // ro + t through PSF row K - 1 + k - t; the lower row of an odd
            // last pair reads the buffer's spare rows and is not stored
            const float *base = (ch == 0 ? Pl : Ps) + ro * W + 4 * g;
            float o0[4] = {0.0f, 0.0f, 0.0f, 0.0f}, o1[4] = {0.0f, 0.0f, 0.0f, 0.0f};
            // (both forms add the PSF rows' partials in the same order, last
            // row first, so that one-lens and multi-lens kernels agree bit
            // for bit)
            if constexpr (ROWS == 1) {
#pragma unroll 1
                for (int t = 0; t < K; ++t)
                    direct_window<K, true, false>(base + t * W, L.tk + (K - 1 - t) * TS,
                                                  nullptr, o0, o1);
            } else {
                direct_window<K, true, false>(base, L.tk + (K - 1) * TS, nullptr, o0, o1);
#pragma unroll 1
                for (int t = 1; t < K; ++t)
                    direct_window<K, true, true>(base + t * W, L.tk + (K - 1 - t) * TS,
                                                 L.tk + (K - t) * TS, o0, o1);
                direct_window<K, false, true>(base + K * W, nullptr, L.tk, o0, o1);
            }
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                m[ch][0][q] = o0[q];
                if constexpr (ROWS == 2) m[ch][ROWS - 1][q] = o1[q];
            }
        }
#pragma unroll
        for (int k = 0; k < ROWS; ++k) {
            if (ro + k < nrows) {
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const int j = 4 * g + q;
                    if (j < nx) sink((b0 + ro + k) * nx + j, m[0][k][q], m[1][k][q]);
                }
            }
        }
    }
}

// ------------------------------------------------------ per-vector body
// Where the two images of lens L live in a CTA: lens / source images Il, Is
// with pixel (i, j) at [i*stride + off + j], row-pass outputs Hl, Hs.
struct ImgPtrs {
    float *Il, *Is, *Hl, *Hs;
    int stride, off;
};

__device__ __forceinline__ int psf_smem_floats(const LensDev &L, int img)
{
    return (img == IMG_PADDED || img == IMG_BANDED) ? 0 : (L.sep ? 2 * L.K : L.K * L.K);
}

__device__ __forceinline__ ImgPtrs img_ptrs(const LensDev &L, float *spsf, float *gslot)
{
    const int IMG = L.img;
    ImgPtrs P;
    if (IMG == IMG_BANDED) {
        // images in the global slot (unpadded); the band buffer is spsf
        P.Il = gslot;
        P.Is = P.Il + L.npix;
        P.Hl = spsf;
        P.Hs = spsf + (L.band_rows + 2 * L.h + kCR) * L.W;
        P.stride = L.nx; P.off = 0;
    } else if (IMG == IMG_PADDED) {
        const int rows = L.ny + 2 * L.h + kCR;   // zero rows above, below, last row block
        P.Il = spsf;
        P.Is = P.Il + rows * L.W;
        P.Hl = P.Il; P.Hs = P.Is;
        P.stride = L.W;
        P.off = L.h * L.W + L.HL;
    } else if (IMG == IMG_SMEM) {
        P.Il = spsf + ((psf_smem_floats(L, IMG) + 3) & ~3);
        P.Is = P.Il + L.npix;
        P.Hl = P.Il;   // the row pass runs in place
        P.Hs = P.Is;
        P.stride = L.nx; P.off = 0;
    } else {
        P.Il = gslot;
        P.Is = P.Il + L.npix;
        P.Hl = P.Is + L.npix;
        P.Hs = P.Hl + L.npix;
        P.stride = L.nx; P.off = 0;
    }
    return P;
}

// Prepare a CTA's memory for lens L: zero the padded layout's halos (they
// stay zero: only interior pixels are ever written) or stage the PSF.
__device__ __forceinline__ void setup_lens(const LensDev &L, float *spsf, int tid, int nthr)
{
    const int IMG = L.img;
    if (IMG == IMG_PADDED || IMG == IMG_BANDED) {
        const int rows = (IMG == IMG_PADDED ? L.ny : L.band_rows) + 2 * L.h + kCR;
        const int n = 2 * rows * L.W;
        for (int t = tid; t < n; t += nthr) spsf[t] = 0.0f;
    } else {
        const int K = L.K, nf = psf_smem_floats(L, IMG);
        for (int t = tid; t < nf; t += nthr)
            spsf[t] = L.sep ? (t < K ? L.pu[t] : L.pv[t - K]) : L.psf[t];
    }
}

// Warp reduction of a thread's five double-float sums; lane 0 stores the
// warp's sums as float pairs to sred[warp*5 + k] (add: adds to what is
// there, in double-float).
__device__ __forceinline__ void warp_sums(float *acc, float2 *sred, int lane, int warp, bool add)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
        for (int k = 0; k < 5; ++k) {
            const float oh = __shfl_xor_sync(0xffffffffu, acc[2 * k], o);
            const float ol = __shfl_xor_sync(0xffffffffu, acc[2 * k + 1], o);
            df_add(acc[2 * k], acc[2 * k + 1], oh, ol);
        }
    }
    if (lane == 0) {
#pragma unroll
        for (int k = 0; k < 5; ++k) {
            float h = acc[2 * k], l = acc[2 * k + 1];
            if (add) {
                const float2 o = sred[warp * 5 + k];
                df_add(h, l, o.x, o.y);
            }
            sred[warp * 5 + k] = make_float2(h, l);
        }
    }
}

// Convolve the two images with the fused sums; each warp's sums end in
// sred[warp*5 + k] (float pairs).  K > 0: the compiled convolution of side K on
// zero-padded bands (IMG_PADDED: the whole image is one band already in
// place; IMG_BANDED: bands filled from the global slot), each band's sums
// reduced over the warp as it ends, so that no accumulator stays live
// across bands; K == 0: the generic convolution (IMG_SMEM, IMG_GLOBAL).
template <int K, bool WRITE>
__device__ __forceinline__ void convolve(const LensDev &L, const RunArgs &R, const ImgPtrs &P,
                                         float *spsf, float2 *sred, int tid, int nthr)
{
    const int lane = tid & 31, warp = tid >> 5;
    if constexpr (K > 0) {
        static_assert(!WRITE, "write-out runs on the generic placements");
        const int h = L.h, W = L.W, HL = L.HL, ny = L.ny, nx = L.nx;
        const bool banded = L.img == IMG_BANDED;
        const int step = banded ? L.band_rows : ny;
        // Both placements convolve in the padded shared buffer at spsf (the
        // same pointers img_ptrs gives), written here from spsf so that the
        // compiler sees shared-memory addresses (32-bit, LDS/STS).
        float *Pl = spsf, *Ps = spsf + (step + 2 * h + kCR) * W;
        for (int b0 = 0; b0 < ny; b0 += step) {
            const int nrows = min(step, ny - b0);
            int rlo = h, rhi = h + ny;   // padded: image rows in place, halos zero
            if (banded) {
                // buffer rows [0, nrows + 2h) <- image rows [b0 - h, b0 + nrows + h)
                const int nbr = nrows + 2 * h;
                stage_band(L, P.Il, P.Is, Pl, (int)(Ps - Pl), b0, nbr, tid, nthr);
                __syncthreads();
                rlo = max(0, h - b0);
                rhi = min(nbr, ny - b0 + h);
            }
            SumsSink sk{L};
#pragma unroll
            for (int k = 0; k < 10; ++k) sk.a[k] = 0.0f;
            if (L.sep) conv_sep_band<K>(L, Pl, Ps, b0, nrows, rlo, rhi, tid, nthr, sk);
            else conv_direct_band<K>(L, Pl, Ps, b0, nrows, tid, nthr, sk);
            warp_sums(sk.a, sred, lane, warp, b0 > 0);
            if (banded) __syncthreads();
        }
    } else {
        float acc[10];
#pragma unroll
        for (int k = 0; k < 10; ++k) acc[k] = 0.0f;
        conv_generic<WRITE>(L, R, spsf, P.Il, P.Is, P.Hl, P.Hs, acc, tid, nthr,
                            L.img == IMG_SMEM);
        warp_sums(acc, sred, lane, warp, false);
    }
}

// One parameter vector (its constant block kc is valid): trace, convolve
// with the fused sums, reduce, finish; log L goes to *outp.  Ends with a
// block barrier.
// Trace one vector with the deflection form it needs (the branch is uniform
// over the CTA); an EPL vector's series table (or its coefficients) is
// first staged in sepl (kEplSmemFloats floats of shared memory,
// epl_stage).  Ends with a block barrier.
template <int SUB>
__device__ __forceinline__ void trace_vector(const LensDev &L, const float *kc, float *Il,
                                             float *Is, int stride, int off, float *sepl,
                                             int tid, int nthr, bool skip,
                                             PendingFinish *pf = nullptr,
                                             const float2 *sred = nullptr)
{
    const VecConst v = load_consts(kc);
    if (v.epl) {
        epl_stage(kc, v, sepl, tid, nthr);
        __syncthreads();
        if (v.etab)
            trace_image<SUB, 5>(L, v, kc, Il, Is, stride, off, tid, nthr, sepl, skip);
        else
            trace_image<SUB, 2>(L, v, kc, Il, Is, stride, off, tid, nthr, sepl, skip);
    } else if (v.fast) {
        trace_image<SUB, 0>(L, v, kc, Il, Is, stride, off, tid, nthr, sepl, skip);
    } else if (v.mid) {
        trace_image<SUB, 4>(L, v, kc, Il, Is, stride, off, tid, nthr, sepl, skip);
    } else {
        trace_image<SUB, 1>(L, v, kc, Il, Is, stride, off, tid, nthr, sepl, skip);
    }
    // the previous vector's solve, by the last warp once its pixels are done
    if (pf && (tid >> 5) == (nthr >> 5) - 1) finish_pending(*pf, sred, tid & 31, nthr >> 5);
    __syncthreads();
}

// Zero the two images of a lens whose traced pixels are listed (placements
// that do not zero them in setup_lens): pixels never traced must start
// finite.
__device__ __forceinline__ void zero_untraced(const LensDev &L, const ImgPtrs &P, int tid,
                                              int nthr)
{
    if (!L.tlist || L.img == IMG_PADDED) return;
    for (int t = tid; t < L.npix; t += nthr) {
        const int i = t / L.nx, j = t - i * L.nx;
        P.Il[i * P.stride + P.off + j] = 0.0f;
        P.Is[i * P.stride + P.off + j] = 0.0f;
    }
}

template <int SUB, int K, bool WRITE>
__device__ __forceinline__ void vector_body(const LensDev &L, const RunArgs &R,
                                            const float *kc, double *outp, const ImgPtrs &P,
                                            float *spsf, float2 *sred, float *sepl,
                                            PendingFinish &pf, int tid, int nthr)
{
    const int lane = tid & 31, warp = tid >> 5, nwarp = nthr >> 5;
    const int nx = L.nx, npix = L.npix;
    trace_vector<SUB>(L, kc, P.Il, P.Is, P.stride, P.off, sepl, tid, nthr, !WRITE,
                      WRITE ? nullptr : &pf, sred);
    if (WRITE) {
        for (int t = tid; t < npix; t += nthr) {
            const int i = t / nx, j = t - i * nx;
            R.wr_unblurred[t] = P.Il[i * P.stride + P.off + j];
            R.wr_unblurred[npix + t] = P.Is[i * P.stride + P.off + j];
        }
        __syncthreads();
    }
    // warp sums in double-float, then per warp in FP64, block sum in FP64
    convolve<K, WRITE>(L, R, P, spsf, sred, tid, nthr);
    __syncthreads();
    if (WRITE) {
        if (warp == 0) {
            double S[5];
            block_sums(sred, nwarp, lane, S);
            if (lane == 0) {
                double sl, ss, ll;
                finish_vector(L, S, kc[K_IEL], kc[K_IES], &sl, &ss, &ll);
                *outp = ll;
                for (int k = 0; k < 5; ++k) R.wr_res[k] = S[k];
                R.wr_res[5] = sl;
                R.wr_res[6] = ss;
                R.wr_res[7] = ll;
            }
        }
        __syncthreads();
    } else if (warp == nwarp - 1) {
        if (lane == 0)
            pf = PendingFinish{L.dWd, L.lognorm, outp, kc[K_IEL], kc[K_IES], L.mode, 1};
        __syncwarp();
    }
    __syncthreads();
}

// One part of a vector's decode (decode_vector), kept out of line so that
// its FP64 working set does not weigh on the likelihood kernel's registers.
static __device__ __noinline__ void decode_part(const float *p, float *o, double XC, double YC,
                                         double d, const double *bn_tab, bool epl, int part)
{
    decode_vector(p, o, XC, YC, d, bn_tab, epl, part);
}

// ------------------------------------------------------- one-lens kernel
// K > 0: compiled convolution of side K (placements IMG_PADDED, IMG_BANDED);
// K == 0: generic convolution (IMG_SMEM, IMG_GLOBAL).
template <int SUB, int K, bool WRITE>
__global__ void __launch_bounds__(kThreads)
k_loglike(const __grid_constant__ LensDev L, const __grid_constant__ RunArgs R)
{
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ __align__(16) float sepl[kEplSmemFloats];
    __shared__ PendingFinish spf;
    const int tid = threadIdx.x, nthr = blockDim.x;
    float2 *sred = reinterpret_cast<float2 *>(smem);
    float *spsf = reinterpret_cast<float *>(smem + kRedBytes);
    if (tid == 0) spf.valid = 0;
    const bool gslot = L.img == IMG_GLOBAL || L.img == IMG_BANDED;
    const ImgPtrs P =
        img_ptrs(L, spsf, gslot ? R.gscr + (size_t)blockIdx.x * R.gslot : nullptr);
    setup_lens(L, spsf, tid, nthr);
    if (!WRITE) zero_untraced(L, P, tid, nthr);
    __syncthreads();
    for (int b = blockIdx.x; b < R.B; b += gridDim.x) {
        const float *kc = R.kc + (size_t)b * NCONST;
        if (!WRITE && R.fused) {
            if (R.smp_on) {
                // the walker's proposal into the vector's parameter row (warp
                // 0, entries over the lanes), visible to the decode after
                // the barrier
                if (tid < 32)
                    stretch_propose_entries(R.smp, b, tid, 32,
                                            const_cast<float *>(R.params) + (size_t)b * R.np,
                                            nullptr);
                __syncthreads();
            }
            // the vector's four decode parts on lane 0 of warps 0-3 (four
            // sub-partitions), visible to the CTA after the barrier
            if ((tid & 31) == 0 && tid < 128)
                decode_part(R.params + (size_t)b * R.np, const_cast<float *>(kc), R.XC, R.YC,
                            R.d, R.bn_tab, R.epl != 0, tid >> 5);
            __syncthreads();
        }
        if (kc[K_VALID] == 0.0f) {
            if (tid == 0) {
                R.out[b] = -INFINITY;
                if (WRITE) R.wr_res[7] = -INFINITY;
            }
            continue;
        }
        vector_body<SUB, K, WRITE>(L, R, kc, R.out + b, P, spsf, sred, sepl, spf, tid, nthr);
    }
    if (!WRITE && (tid >> 5) == (nthr >> 5) - 1) finish_pending(spf, sred, tid & 31, nthr >> 5);
    if (!WRITE && R.smp_on) {
        // the accept / reject of the vector's walker once its log L is in
        // out (written by the last warp, or by thread 0 for an invalid one)
        __syncthreads();
        if (tid == 0)
            for (int b = blockIdx.x; b < R.B; b += gridDim.x)
                stretch_accept_one(R.smp, b, R.params + (size_t)b * R.np, R.out[b]);
    }
}

// ----------------------------------------------------- multi-lens kernel
// One launch over the vectors of one group of segments: at most kMultiSlots
// two-column lenses sharing the supersampling class SUB and the convolution
// class K, their items contiguous per lens (LensSlots).  Each CTA starts on
// its home slot and then takes the following ones in turn, every slot's
// vectors handed out by its counter; the lens descriptor is read from the
// kernel's parameters through the slot index, which depends on blockIdx
// and the loop count only (block-uniform), so its constants stay operands
// of the arithmetic (a copy in shared memory made every tap a load: 10 %
// slower).
template <int SUB, int K>
__global__ void __launch_bounds__(kThreads) k_loglike_multi(const __grid_constant__ MultiArgs A,
                                                            int group,
                                                            const __grid_constant__ LensSlots S)
{
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int s_t, s_seg;
    __shared__ __align__(16) float sepl[kEplSmemFloats];
    __shared__ PendingFinish spf;
    const int tid = threadIdx.x, nthr = blockDim.x;
    if (tid == 0) spf.valid = 0;
    float2 *sred = reinterpret_cast<float2 *>(smem);
    float *spsf = reinterpret_cast<float *>(smem + kRedBytes);
    float *gslot = A.gscr ? A.gscr + (size_t)blockIdx.x * A.gslot_floats : nullptr;
    const MultiHdr hd = A.groups[group];
    int home = 0;
    while (home < S.n - 1 && (int)blockIdx.x >= S.cta_end[home]) ++home;
    for (int k = 0; k < S.n; ++k) {
        int s = home + k;
        if (s >= S.n) s -= S.n;
        const LensDev &L = S.lens[s];
        int *ctr = A.counter + kMultiCounters + group * kMultiSlots + s;
        bool ready = false;
        for (;;) {
            if (tid == 0) {
                const int i = atomicAdd(ctr, 1);
                const int t = i < S.count[s] ? S.first[s] + i : -1;
                s_t = t;
                s_seg = t >= 0 ? find_segment(A.segs, hd.seg0, hd.nseg, t) : 0;
            }
            __syncthreads();
            const int t = s_t;
            if (t < 0) break;
            if (!ready) {
                // the slot's lens in the CTA's shared memory (halos, taps)
                setup_lens(L, spsf, tid, nthr);
                zero_untraced(L, img_ptrs(L, spsf, gslot), tid, nthr);
                __syncthreads();
                ready = true;
            }
            const Segment sg = A.segs[s_seg];
            const float *kc = A.kc + (size_t)t * NCONST;
            double *outp = sg.out + (t - sg.first);
            if (kc[K_VALID] == 0.0f) {
                if (tid == 0) *outp = -INFINITY;
                __syncthreads();
                continue;
            }
            RunArgs R = {};
            const ImgPtrs P = img_ptrs(L, spsf, gslot);
            vector_body<SUB, K, false>(L, R, kc, outp, P, spsf, sred, sepl, spf, tid, nthr);
        }
        __syncthreads();
    }
    if ((tid >> 5) == (nthr >> 5) - 1) finish_pending(spf, sred, tid & 31, nthr >> 5);
}

// --------------------------------------------------------------- registry
using SingleKernel = void (*)(const LensDev, const RunArgs);
using MultiKernel = void (*)(const MultiArgs, int, const LensSlots);

// Supersampling classes with an unrolled subpixel loop.
__host__ __device__ inline int sub_class(int sub) { return (sub == 4 || sub == 5) ? sub : 0; }



template <int K>
inline SingleKernel single_for(int sub)
{
    switch (sub_class(sub)) {
        case 4: return k_loglike<4, K, false>;
        case 5: return k_loglike<5, K, false>;
        default: return k_loglike<0, K, false>;
    }
}

template <int K>
inline MultiKernel multi_for(int sub)
{
    switch (sub_class(sub)) {
        case 4: return k_loglike_multi<4, K>;
        case 5: return k_loglike_multi<5, K>;
        default: return k_loglike_multi<0, K>;
    }
}

}  // namespace tll
