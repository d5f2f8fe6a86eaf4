// tll.cu -- kernels and C ABI of libtll.so (GB300, sm_103a).
//
// Hot path per batch (one stream, two launches):
//   k_prologue  one thread per parameter vector: ellipse, b_n (FP64),
//               SIE prefactors -> a 32-float constant block per vector.
//   k_loglike   persistent CTAs, one parameter vector at a time per CTA:
//               (1) ray-trace + Sersic light on the s x s subpixels of every
//                   pixel, binned to two float images (lens, source) held in
//                   shared memory (or, for images too large for it, in a
//                   per-CTA global scratch slot that stays in L2);
//               (2) PSF convolution of both images -- separable (row pass in
//                   place, then column pass) when the PSF is an outer
//                   product to rounding, direct 2-D otherwise;
//               (3) fused into the convolution's output loop, the five
//                   weighted sums A_ll, A_ls, A_ss, b_l, b_s in double-float
//                   (exact FMA products, compensated sums), promoted to FP64
//                   for the warp / block reduction;
//               (4) one thread: 2-column NNLS or fixed amplitudes, chi^2,
//                   log L in FP64.
// The model-image entry points run the same kernel on one vector with the
// intermediate images written out.
#include <cuda_runtime.h>

#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <mutex>
#include <new>
#include <vector>

#include "tll.h"
#include "tll_device.cuh"

using namespace tll;

namespace {

constexpr int kThreads = 1024;     // CTA size of k_loglike (64 registers, 32 warps per SM)
constexpr int kHMax = 8;           // in-place row pass holds nx <= 32*kHMax
constexpr int kRedBytes = 32 * 5 * 8;

thread_local char g_err[512] = "";

int fail(int code, const char *fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof g_err, fmt, ap);
    va_end(ap);
    return code;
}

#define CUDA_TRY(expr)                                                        \
    do {                                                                      \
        cudaError_t e_ = (expr);                                              \
        if (e_ != cudaSuccess)                                                \
            return fail(e_ == cudaErrorMemoryAllocation ? TLL_ENOMEM          \
                                                        : TLL_ECUDA,          \
                        "%s: %s", #expr, cudaGetErrorString(e_));             \
    } while (0)

constexpr int kMaxTaps = 32;   // separable PSF factors carried in the parameter block

struct LensDev {
    int nx, ny, npix, sub, K, h, sep, mode;
    float JCX, JCY;   // subpixel index of the grid centre, (n*s - 1)/2
    float inv_s2;
    int W, HL;        // padded layout: row stride, left zero columns
    int img;          // image placement (IMG_*)
    double XC, YC, d; // grid centre and subpixel step (for the prologue)
    const float *psf;    // [K*K] unit sum (direct path)
    const float *pu;     // [K] column factor over PSF rows (separable path)
    const float *pv;     // [K] row factor over PSF columns
    const float4 *wpack; // [npix] (w_hi, w_lo, wd_hi, wd_lo)
    double dWd, lognorm;
    float tu[kMaxTaps], tv[kMaxTaps];   // the separable factors again, by value
};

// Image placement in k_loglike.
enum : int {
    IMG_GLOBAL = 0,   // per-CTA global scratch slot (L2), generic convolution
    IMG_SMEM = 1,     // shared memory, unpadded, generic convolution
    IMG_PADDED = 2    // shared memory with zero halos, convolution compiled per K
};

struct RunArgs {
    const float *kc;     // [B][NCONST]
    int B;
    double *out;         // [B]
    float *gscr;         // global image scratch, 4*npix floats per CTA
    float *wr_unblurred; // WRITE: [2][npix]
    float *wr_blurred;   // WRITE: [2][npix]
    double *wr_res;      // WRITE: [8] All Als Ass bl bs sl ss logL
};

// -------------------------------------------------------------- kernels
__global__ void k_prologue(const float *__restrict__ params, int B,
                           float *__restrict__ kc, double XC, double YC, double d,
                           const double *__restrict__ bn_tab)
{
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b < B)
        decode_vector(params + (size_t)b * NPAR, kc + (size_t)b * NCONST, XC, YC, d,
                      bn_tab);
}

// One thread per node of the b_n table (run once per device).
__global__ void k_bn_table(double *__restrict__ tab)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= 2 * BN_SEG) return;
    const int seg = t / BN_SEG, k = t - seg * BN_SEG - 1;
    tab[t] = sersic_bn_dev(bn_node(seg, k));
}

// One term of the five weighted sums (Sec. 2.3: A = M^T W M, b = M^T W d)
// for one pixel with blurred column values ml, ms; wp = (w_hi, w_lo,
// wd_hi, wd_lo).  Products are formed exactly as float pairs and added
// with TwoSum into double-float accumulators a[0..9].
__device__ __forceinline__ void accum_pixel(float ml, float ms, float4 wp, float *a)
{
    float p1 = wp.x * ml, e1 = fmaf(wp.x, ml, -p1);
    e1 = fmaf(wp.y, ml, e1);
    float p2 = wp.x * ms, e2 = fmaf(wp.x, ms, -p2);
    e2 = fmaf(wp.y, ms, e2);
    float p, e;
    p = p1 * ml; e = fmaf(p1, ml, -p); e = fmaf(e1, ml, e); df_acc(a[0], a[1], p, e);
    p = p1 * ms; e = fmaf(p1, ms, -p); e = fmaf(e1, ms, e); df_acc(a[2], a[3], p, e);
    p = p2 * ms; e = fmaf(p2, ms, -p); e = fmaf(e2, ms, e); df_acc(a[4], a[5], p, e);
    p = wp.z * ml; e = fmaf(wp.z, ml, -p); e = fmaf(wp.w, ml, e); df_acc(a[6], a[7], p, e);
    p = wp.z * ms; e = fmaf(wp.z, ms, -p); e = fmaf(wp.w, ms, e); df_acc(a[8], a[9], p, e);
}

// Amplitudes and log L from the five sums (thread-local, FP64).
// NNLS over two columns: the optimum is the unconstrained minimiser of one
// face {none, lens only, source only, both} that is feasible; chi^2 of a
// face's minimiser s is dWd - s^T b.  Fixed mode: s = (I_e^L, I_e^S) and
// chi^2 = dWd - 2 s^T b + s^T A s.
__device__ __forceinline__ void finish_vector(const LensDev &L, const double *S,
                                              float IeL, float IeS, double *sl_o,
                                              double *ss_o, double *ll_o)
{
    const double All = S[0], Als = S[1], Ass = S[2], bl = S[3], bs = S[4];
    double sl, ss, chi2;
    if (L.mode == TLL_AMP_FIXED) {
        sl = IeL;
        ss = IeS;
        chi2 = L.dWd - 2.0 * (sl * bl + ss * bs) + sl * sl * All +
               2.0 * sl * ss * Als + ss * ss * Ass;
    } else {
        sl = 0.0; ss = 0.0; chi2 = L.dWd;
        if (All > 0.0 && bl > 0.0) {
            const double c = L.dWd - bl * (bl / All);
            if (c < chi2) { chi2 = c; sl = bl / All; ss = 0.0; }
        }
        if (Ass > 0.0 && bs > 0.0) {
            const double c = L.dWd - bs * (bs / Ass);
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
                const double c = L.dWd - 2.0 * (tl * bl + ts * bs) + tl * tl * All +
                                 2.0 * tl * ts * Als + ts * ts * Ass;
                if (c < chi2) { chi2 = c; sl = tl; ss = ts; }
            }
        }
    }
    *sl_o = sl;
    *ss_o = ss;
    *ll_o = -0.5 * chi2 + L.lognorm;
}

// --------------------------------------------------------- trace phase
// Ray-trace + light on the s x s subpixels of every pixel, mean-binned:
// pixel (i, j) of the lens / source image goes to Il / Is [i*stride + off + j].
// Subpixel (J, I) of the supersampled grid has exact integer-or-half
// offsets (fj, fi) = (J - JCX, I - JCY) from the grid centre; every
// coordinate is an affine function of them (see decode_vector).
template <int SUB>
__device__ __forceinline__ void trace_image(const LensDev &L, const VecConst &v,
                                            float *Il, float *Is, int stride, int off,
                                            int tid, int nthr)
{
    const int sub = SUB > 0 ? SUB : L.sub;
    const int nx = L.nx;
    for (int pix = tid; pix < L.npix; pix += nthr) {
        const int i = pix / nx, j = pix - i * nx;
        const float fj0 = (float)(j * sub) - L.JCX;
        const float fi0 = (float)(i * sub) - L.JCY;
        float accl = 0.0f, accs = 0.0f;
#pragma unroll 1
        for (int a = 0; a < sub; ++a) {
            const RowTerms r = row_terms(v, fi0 + (float)a);
#pragma unroll
            for (int c = 0; c < (SUB > 0 ? SUB : 1); ++c) {
                for (int cr = 0; cr < (SUB > 0 ? 1 : sub); ++cr) {
                    float il, is;
                    subpixel(v, r, fj0 + (float)(SUB > 0 ? c : cr), il, is);
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
template <bool INPLACE, bool WRITE>
__device__ __forceinline__ void conv_generic(const LensDev &L, const RunArgs &R,
                                             const float *spsf, float *Il, float *Is,
                                             float *Hl, float *Hs, float *acc, int tid,
                                             int nthr)
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
        __syncthreads();
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
                    R.wr_blurred[npix + pix] = ms;
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
                R.wr_blurred[npix + pix] = ms;
            }
            accum_pixel(ml, ms, L.wpack[pix], acc);
        }
    }
}

// --------------------------------------------------- padded convolution
// Separable PSF with compile-time side K on the zero-padded shared-memory
// layout: image pixel (i, j) at P[(h + i) W + HL + j], HL = h rounded up to
// a multiple of 4; rows [0, h) and [h + ny, ...) and the columns outside
// [HL, HL + nx) hold zeros, so no tap needs a bounds check.
//  Row pass (in place, one warp per row): a lane computes 4 adjacent
//  outputs from one window of K + 3 values read as float4s.
//  Column pass: a warp takes 32 adjacent columns x CR rows; a lane reads
//  CR + K - 1 values of its column and computes CR outputs per channel.
// Taps come from the parameter block (compile-time indices).
constexpr int kCR = 4;

template <int K>
struct PadGeom {
    static constexpr int h = (K - 1) / 2;
    static constexpr int HL = (h + 3) & ~3;
    static constexpr int D = HL - h;                 // window offset in a group
    static constexpr int NW = (D + K + 3 + 3) / 4;   // float4 reads per window
};

// Padded row stride for an image of nx columns and PSF side K (host and
// device): covers every float4 window read of the row pass and the right
// zero halo.
__host__ __device__ inline int padded_stride(int nx, int K)
{
    const int h = (K - 1) / 2, HL = (h + 3) & ~3, D = HL - h;
    const int NW = (D + K + 6) / 4;
    const int W = 4 * ((nx + 3) / 4) + 4 * NW;
    return (W + 3) & ~3;
}

struct Acc10 {
    float a[10];
};

template <int K, bool WRITE>
__device__ __noinline__ Acc10 conv_padded(const LensDev &L, const RunArgs &R, float *Pl,
                                          float *Ps, int tid, int nthr)
{
    Acc10 out;
    float *acc = out.a;
#pragma unroll
    for (int k = 0; k < 10; ++k) acc[k] = 0.0f;
    using G = PadGeom<K>;
    const int nx = L.nx, ny = L.ny, W = L.W;
    const int lane = tid & 31, warp = tid >> 5, nwarp = nthr >> 5;
    const int ngroups = (nx + 3) >> 2;
    // row pass, in place; each lane holds at most 2 groups (nx <= 256)
    for (int row = warp; row < 2 * ny; row += nwarp) {
        float *P = (row < ny ? Pl + (G::h + row) * W : Ps + (G::h + row - ny) * W);
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
    __syncthreads();
    // column pass with the fused weighted sums
    const int ncg = (nx + 31) >> 5, nrb = (ny + kCR - 1) / kCR;
    for (int item = warp; item < ncg * nrb; item += nwarp) {
        const int cg = item % ncg, rb = item / ncg;
        const int j = 32 * cg + lane, i0 = rb * kCR;
        const int jc = min(j, nx - 1);
        float ml[kCR], ms[kCR];
#pragma unroll
        for (int ch = 0; ch < 2; ++ch) {
            const float *col = (ch == 0 ? Pl : Ps) + i0 * W + G::HL + jc;
            float win[kCR + K - 1];
#pragma unroll
            for (int t = 0; t < kCR + K - 1; ++t) win[t] = col[t * W];
#pragma unroll
            for (int r = 0; r < kCR; ++r) {
                float a = 0.0f;
#pragma unroll
                for (int c = 0; c < K; ++c) a = fmaf(L.tu[c], win[r + K - 1 - c], a);
                if (ch == 0) ml[r] = a; else ms[r] = a;
            }
        }
        if (j < nx) {
#pragma unroll
            for (int r = 0; r < kCR; ++r) {
                const int i = i0 + r;
                if (i < ny) {
                    const int pix = i * nx + j;
                    if (WRITE) {
                        R.wr_blurred[pix] = ml[r];
                        R.wr_blurred[L.npix + pix] = ms[r];
                    }
                    accum_pixel(ml[r], ms[r], L.wpack[pix], acc);
                }
            }
        }
    }
    return out;
}

template <bool WRITE>
__device__ __forceinline__ void conv_padded_dispatch(const LensDev &L, const RunArgs &R,
                                                     float *Pl, float *Ps, float *acc,
                                                     int tid, int nthr)
{
    switch (L.K) {
#define TLL_K(k) case k: { const Acc10 r = conv_padded<k, WRITE>(L, R, Pl, Ps, tid, nthr); \
        for (int q = 0; q < 10; ++q) acc[q] = r.a[q]; } break;
        TLL_K(1) TLL_K(3) TLL_K(5) TLL_K(7) TLL_K(9) TLL_K(11) TLL_K(13) TLL_K(15)
        TLL_K(17) TLL_K(19) TLL_K(21) TLL_K(23) TLL_K(25) TLL_K(27) TLL_K(29) TLL_K(31)
#undef TLL_K
        default: break;   // the host selects IMG_PADDED only for odd K <= 31
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
    return img == IMG_PADDED ? 0 : (L.sep ? 2 * L.K : L.K * L.K);
}

template <int IMG>
__device__ __forceinline__ ImgPtrs img_ptrs(const LensDev &L, float *spsf, float *gslot)
{
    ImgPtrs P;
    if (IMG == IMG_PADDED) {
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
template <int IMG>
__device__ __forceinline__ void setup_lens(const LensDev &L, float *spsf, int tid, int nthr)
{
    if (IMG == IMG_PADDED) {
        const int n = 2 * (L.ny + 2 * L.h + kCR) * L.W;
        for (int t = tid; t < n; t += nthr) spsf[t] = 0.0f;
    } else {
        const int K = L.K, nf = psf_smem_floats(L, IMG);
        for (int t = tid; t < nf; t += nthr)
            spsf[t] = L.sep ? (t < K ? L.pu[t] : L.pv[t - K]) : L.psf[t];
    }
}

// One parameter vector (its constant block kc is valid): trace, convolve
// with the fused sums, reduce, finish; log L goes to *outp.  Ends with a
// block barrier.
template <int SUB, int IMG, bool WRITE>
__device__ __forceinline__ void vector_body(const LensDev &L, const RunArgs &R,
                                            const float *kc, double *outp, const ImgPtrs &P,
                                            const float *spsf, double *sred, int tid, int nthr)
{
    const int lane = tid & 31, warp = tid >> 5, nwarp = nthr >> 5;
    const int nx = L.nx, npix = L.npix;
    {
        const VecConst v = load_consts(kc);
        trace_image<SUB>(L, v, P.Il, P.Is, P.stride, P.off, tid, nthr);
    }
    __syncthreads();
    if (WRITE) {
        for (int t = tid; t < npix; t += nthr) {
            const int i = t / nx, j = t - i * nx;
            R.wr_unblurred[t] = P.Il[i * P.stride + P.off + j];
            R.wr_unblurred[npix + t] = P.Is[i * P.stride + P.off + j];
        }
        __syncthreads();
    }

    // (2)+(3) convolution with the fused weighted sums
    float acc[10];
#pragma unroll
    for (int k = 0; k < 10; ++k) acc[k] = 0.0f;
    if (IMG == IMG_PADDED)
        conv_padded_dispatch<WRITE>(L, R, P.Il, P.Is, acc, tid, nthr);
    else
        conv_generic<IMG == IMG_SMEM, WRITE>(L, R, spsf, P.Il, P.Is, P.Hl, P.Hs, acc, tid,
                                             nthr);

    // (3) warp reduction in double-float, block reduction in FP64
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
        for (int k = 0; k < 5; ++k)
            sred[warp * 5 + k] = (double)acc[2 * k] + (double)acc[2 * k + 1];
    }
    __syncthreads();
    if (warp == 0) {
        double sacc = 0.0;
        if (lane < 5)
            for (int w = 0; w < nwarp; ++w) sacc += sred[w * 5 + lane];
        double S[5];
#pragma unroll
        for (int k = 0; k < 5; ++k) S[k] = __shfl_sync(0xffffffffu, sacc, k);
        if (lane == 0) {
            double sl, ss, ll;
            finish_vector(L, S, kc[K_IEL], kc[K_IES], &sl, &ss, &ll);
            *outp = ll;
            if (WRITE) {
                for (int k = 0; k < 5; ++k) R.wr_res[k] = S[k];
                R.wr_res[5] = sl;
                R.wr_res[6] = ss;
                R.wr_res[7] = ll;
            }
        }
    }
    __syncthreads();
}

// ------------------------------------------------------- one-lens kernel
template <int SUB, int IMG, bool WRITE>
__global__ void __launch_bounds__(kThreads)
k_loglike(const __grid_constant__ LensDev L, const __grid_constant__ RunArgs R)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const int tid = threadIdx.x, nthr = blockDim.x;
    double *sred = reinterpret_cast<double *>(smem);
    float *spsf = reinterpret_cast<float *>(smem + kRedBytes);
    const ImgPtrs P =
        img_ptrs<IMG>(L, spsf, IMG == IMG_GLOBAL ? R.gscr + (size_t)blockIdx.x * 4 * L.npix : nullptr);
    setup_lens<IMG>(L, spsf, tid, nthr);
    __syncthreads();
    for (int b = blockIdx.x; b < R.B; b += gridDim.x) {
        const float *kc = R.kc + (size_t)b * NCONST;
        if (kc[K_VALID] == 0.0f) {
            if (tid == 0) {
                R.out[b] = -INFINITY;
                if (WRITE) R.wr_res[7] = -INFINITY;
            }
            continue;
        }
        vector_body<SUB, IMG, WRITE>(L, R, kc, R.out + b, P, spsf, sred, tid, nthr);
    }
}

// ----------------------------------------------------- multi-lens kernel
// One launch over a work list of B_1 + ... + B_n vectors of n lenses
// (different sizes, supersampling, PSFs).  Segment s covers items
// [first, first + count) of lens `lens`, reading params[k] and writing
// out[k].  CTAs take items from an atomic counter (largest lenses first, as
// the host orders them) and copy a lens's descriptor into shared memory when
// they switch lens.
struct Segment {
    int lens, first, count, pad;
    const float *params;
    double *out;
};
struct MultiHdr {
    int total, nseg;
};
struct MultiArgs {
    const LensDev *lenses;
    const Segment *segs;
    const MultiHdr *hdr;
    float *kc;                 // [total][NCONST]
    float *gscr;               // per-CTA global image slots (IMG_GLOBAL lenses)
    long long gslot_floats;
    int *counter;              // work counter, zero at launch
    const double *bn_tab;
};

__device__ __forceinline__ int find_segment(const Segment *segs, int nseg, int t)
{
    int lo = 0, hi = nseg - 1;     // largest s with segs[s].first <= t
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (segs[mid].first <= t) lo = mid; else hi = mid - 1;
    }
    return lo;
}

__global__ void k_prologue_multi(const __grid_constant__ MultiArgs A)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= A.hdr->total) return;
    const Segment &sg = A.segs[find_segment(A.segs, A.hdr->nseg, t)];
    const LensDev &L = A.lenses[sg.lens];
    decode_vector(sg.params + (size_t)(t - sg.first) * NPAR, A.kc + (size_t)t * NCONST, L.XC,
                  L.YC, L.d, A.bn_tab);
}

template <int SUB, int IMG>
__device__ __noinline__ void vector_body_multi(const LensDev &L, const float *kc, double *outp,
                                               float *spsf, float *gslot, double *sred,
                                               int tid, int nthr)
{
    RunArgs R = {};
    const ImgPtrs P = img_ptrs<IMG>(L, spsf, gslot);
    vector_body<SUB, IMG, false>(L, R, kc, outp, P, spsf, sred, tid, nthr);
}

template <int IMG>
__device__ __forceinline__ void body_multi_sub(const LensDev &L, const float *kc, double *outp,
                                               float *spsf, float *gslot, double *sred,
                                               int tid, int nthr)
{
    if (L.sub == 4) vector_body_multi<4, IMG>(L, kc, outp, spsf, gslot, sred, tid, nthr);
    else if (L.sub == 5) vector_body_multi<5, IMG>(L, kc, outp, spsf, gslot, sred, tid, nthr);
    else vector_body_multi<0, IMG>(L, kc, outp, spsf, gslot, sred, tid, nthr);
}

__global__ void __launch_bounds__(kThreads) k_loglike_multi(const __grid_constant__ MultiArgs A)
{
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ LensDev sL;
    __shared__ int s_t, s_seg;
    const int tid = threadIdx.x, nthr = blockDim.x;
    double *sred = reinterpret_cast<double *>(smem);
    float *spsf = reinterpret_cast<float *>(smem + kRedBytes);
    float *gslot = A.gscr ? A.gscr + (size_t)blockIdx.x * A.gslot_floats : nullptr;
    const int total = A.hdr->total, nseg = A.hdr->nseg;
    int cur = -1;
    for (;;) {
        if (tid == 0) {
            const int t = atomicAdd(A.counter, 1);
            s_t = t;
            s_seg = t < total ? find_segment(A.segs, nseg, t) : 0;
        }
        __syncthreads();
        const int t = s_t;
        if (t >= total) break;
        const Segment sg = A.segs[s_seg];
        if (sg.lens != cur) {
            const unsigned *src = reinterpret_cast<const unsigned *>(A.lenses + sg.lens);
            unsigned *dst = reinterpret_cast<unsigned *>(&sL);
            for (int k = tid; k < (int)(sizeof(LensDev) / 4); k += nthr) dst[k] = src[k];
            __syncthreads();
            if (sL.img == IMG_PADDED) setup_lens<IMG_PADDED>(sL, spsf, tid, nthr);
            else if (sL.img == IMG_SMEM) setup_lens<IMG_SMEM>(sL, spsf, tid, nthr);
            else setup_lens<IMG_GLOBAL>(sL, spsf, tid, nthr);
            __syncthreads();
            cur = sg.lens;
        }
        const float *kc = A.kc + (size_t)t * NCONST;
        double *outp = sg.out + (t - sg.first);
        if (kc[K_VALID] == 0.0f) {
            if (tid == 0) *outp = -INFINITY;
            __syncthreads();
            continue;
        }
        if (sL.img == IMG_PADDED)
            body_multi_sub<IMG_PADDED>(sL, kc, outp, spsf, gslot, sred, tid, nthr);
        else if (sL.img == IMG_SMEM)
            body_multi_sub<IMG_SMEM>(sL, kc, outp, spsf, gslot, sred, tid, nthr);
        else
            body_multi_sub<IMG_GLOBAL>(sL, kc, outp, spsf, gslot, sred, tid, nthr);
    }
}

// Model image of one vector: I^m = s_l m_l + s_s m_s (Eq. 7), FP64 then
// rounded.
__global__ void k_combine(const float *__restrict__ blurred,
                          const double *__restrict__ res, int npix,
                          float *__restrict__ img)
{
    const double sl = res[5], ss = res[6];
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < npix;
         t += gridDim.x * blockDim.x)
        img[t] = (float)(sl * (double)blurred[t] + ss * (double)blurred[npix + t]);
}

}  // namespace

// ------------------------------------------------------------ lens object
struct tll_lens {
    int dev = 0;
    int nx = 0, ny = 0, npix = 0, sub = 0, K = 0, flags = 0, mode = 0, sep = 0;
    float dpix = 0, x0 = 0, y0 = 0;
    double dWd = 0, lognorm = 0, psf_sum = 0;
    float *d_psf = nullptr, *d_pu = nullptr, *d_pv = nullptr;
    float4 *d_wpack = nullptr;
    float *d_kc = nullptr;
    int kc_cap = 0;
    float *d_gscr = nullptr;
    float *d_stage_p = nullptr;
    double *d_stage_o = nullptr;
    int stage_cap = 0;
    float *d_p1 = nullptr, *d_kc1 = nullptr, *d_unb = nullptr, *d_blur = nullptr,
          *d_img = nullptr;
    double *d_res = nullptr, *d_out1 = nullptr;
    int img = 0;          // IMG_GLOBAL / IMG_SMEM / IMG_PADDED
    int W = 0, HL = 0;    // padded layout geometry
    std::vector<float> taps_u, taps_v;
    int grid_cap = 0;
    size_t smem_bytes = 0;
    const double *bn_tab = nullptr;   // per-device b_n table (not owned)
    size_t dev_bytes = 0;             // device memory this lens holds
    cudaEvent_t prof_ev[3] = {nullptr, nullptr, nullptr};
    bool prof_on = false, prof_recorded = false;
};

namespace {

// Per-device b_n table, built on first use and kept for the process.
constexpr int kMaxDevices = 64;
double *g_bn_tab[kMaxDevices] = {};
std::mutex g_bn_mu;

int bn_table(int dev, const double **out)
{
    if (dev < 0 || dev >= kMaxDevices) return fail(TLL_ECUDA, "device id %d out of range", dev);
    std::lock_guard<std::mutex> lk(g_bn_mu);
    if (!g_bn_tab[dev]) {
        double *p = nullptr;
        CUDA_TRY(cudaMalloc(&p, 2 * BN_SEG * sizeof(double)));
        k_bn_table<<<(2 * BN_SEG + 127) / 128, 128>>>(p);
        cudaError_t e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaDeviceSynchronize();
        if (e != cudaSuccess) {
            cudaFree(p);
            return fail(TLL_ECUDA, "b_n table: %s", cudaGetErrorString(e));
        }
        g_bn_tab[dev] = p;
    }
    *out = g_bn_tab[dev];
    return TLL_OK;
}

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev)
    {
        if (cudaGetDevice(&prev) == cudaSuccess && prev != dev) cudaSetDevice(dev);
        else prev = -1;
    }
    ~DeviceGuard()
    {
        if (prev >= 0) cudaSetDevice(prev);
    }
};

// Coordinate of the grid centre, x0 + (nx - 1) dpix / 2: subpixel J sits at
// centre + (J - (nx s - 1)/2) dpix/s.
void grid_centre(const tll_lens *L, double *xc, double *yc)
{
    *xc = (double)L->x0 + 0.5 * (L->nx - 1) * (double)L->dpix;
    *yc = (double)L->y0 + 0.5 * (L->ny - 1) * (double)L->dpix;
}

LensDev lens_dev(const tll_lens *L)
{
    LensDev d;
    d.nx = L->nx; d.ny = L->ny; d.npix = L->npix; d.sub = L->sub;
    d.K = L->K; d.h = (L->K - 1) / 2; d.sep = L->sep; d.mode = L->mode;
    d.JCX = 0.5f * (float)(L->nx * L->sub - 1);
    d.JCY = 0.5f * (float)(L->ny * L->sub - 1);
    d.inv_s2 = 1.0f / (float)(L->sub * L->sub);
    d.psf = L->d_psf; d.pu = L->d_pu; d.pv = L->d_pv; d.wpack = L->d_wpack;
    d.dWd = L->dWd; d.lognorm = L->lognorm;
    d.W = L->W; d.HL = L->HL; d.img = L->img;
    grid_centre(L, &d.XC, &d.YC);
    d.d = (double)L->dpix / L->sub;
    for (int k = 0; k < kMaxTaps; ++k) {
        d.tu[k] = k < (int)L->taps_u.size() ? L->taps_u[k] : 0.0f;
        d.tv[k] = k < (int)L->taps_v.size() ? L->taps_v[k] : 0.0f;
    }
    return d;
}

// Kernel variant for (supersampling, image placement, write-out):
// s = 4 and s = 5 are compiled with the subpixel loop unrolled.
template <int IMG, bool WRITE>
void (*pick_kernel(int sub))(const LensDev, const RunArgs)
{
    if (sub == 4) return k_loglike<4, IMG, WRITE>;
    if (sub == 5) return k_loglike<5, IMG, WRITE>;
    return k_loglike<0, IMG, WRITE>;
}

template <bool WRITE>
void (*pick_kernel(int img, int sub))(const LensDev, const RunArgs)
{
    if (img == IMG_PADDED) return pick_kernel<IMG_PADDED, WRITE>(sub);
    if (img == IMG_SMEM) return pick_kernel<IMG_SMEM, WRITE>(sub);
    return pick_kernel<IMG_GLOBAL, WRITE>(sub);
}

int launch_main(const tll_lens *L, const RunArgs &R, int grid, bool write, cudaStream_t st)
{
    auto kern = write ? pick_kernel<true>(L->img, L->sub) : pick_kernel<false>(L->img, L->sub);
    kern<<<grid, kThreads, L->smem_bytes, st>>>(lens_dev(L), R);
    CUDA_TRY(cudaGetLastError());
    return TLL_OK;
}

int run_batch(tll_lens *L, const float *params, int B, double *out, cudaStream_t st,
              bool write, float *kc)
{
    const bool prof = L->prof_on && !write;
    if (prof) CUDA_TRY(cudaEventRecord(L->prof_ev[0], st));
    double xc, yc;
    grid_centre(L, &xc, &yc);
    k_prologue<<<(B + 127) / 128, 128, 0, st>>>(params, B, kc, xc, yc,
                                                (double)L->dpix / L->sub, L->bn_tab);
    CUDA_TRY(cudaGetLastError());
    if (prof) CUDA_TRY(cudaEventRecord(L->prof_ev[1], st));
    RunArgs R;
    R.kc = kc; R.B = B; R.out = out; R.gscr = L->d_gscr;
    R.wr_unblurred = L->d_unb; R.wr_blurred = L->d_blur; R.wr_res = L->d_res;
    const int grid = std::min(B, L->grid_cap);
    if (write) return launch_main(L, R, 1, true, st);
    const int rc = launch_main(L, R, grid, false, st);
    if (rc == TLL_OK && prof) {
        CUDA_TRY(cudaEventRecord(L->prof_ev[2], st));
        L->prof_recorded = true;
    }
    return rc;
}

int ensure_kc(tll_lens *L, int B)
{
    if (B <= L->kc_cap) return TLL_OK;
    int cap = std::max(B, 2 * L->kc_cap);
    float *p = nullptr;
    CUDA_TRY(cudaMalloc(&p, (size_t)cap * NCONST * sizeof(float)));
    if (L->d_kc) cudaFree(L->d_kc);
    L->dev_bytes += ((size_t)cap - L->kc_cap) * NCONST * sizeof(float);
    L->d_kc = p;
    L->kc_cap = cap;
    return TLL_OK;
}

int configure(tll_lens *L)
{
    int nsm = 0, optin = 0;
    CUDA_TRY(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, L->dev));
    CUDA_TRY(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, L->dev));
    // placement: padded shared memory (separable PSF, K <= 31, nx <= 256),
    // else unpadded shared memory, else a global scratch slot per CTA
    const int h = (L->K - 1) / 2;
    const int Wp = padded_stride(L->nx, L->K);
    const size_t padded = kRedBytes + (size_t)2 * (L->ny + 2 * h + kCR) * Wp * sizeof(float);
    const int psf_floats = L->sep ? 2 * L->K : L->K * L->K;
    const size_t fixed = kRedBytes + (size_t)((psf_floats + 3) & ~3) * sizeof(float);
    const size_t plain = fixed + (size_t)2 * L->npix * sizeof(float);
    if (L->sep && L->K <= kMaxTaps - 1 && L->nx <= 256 && padded <= (size_t)optin) {
        L->img = IMG_PADDED;
        L->smem_bytes = padded;
        L->W = Wp;
        L->HL = (h + 3) & ~3;
    } else if (plain <= (size_t)optin && L->nx <= 32 * kHMax) {
        L->img = IMG_SMEM;
        L->smem_bytes = plain;
    } else {
        L->img = IMG_GLOBAL;
        L->smem_bytes = fixed;
    }
    // allow every shared-memory instantiation the device's full opt-in
    // shared memory, so lenses of different sizes can share the kernels
    for (int sb : {0, 4, 5})
        for (int im : {IMG_SMEM, IMG_PADDED}) {
            CUDA_TRY(cudaFuncSetAttribute(pick_kernel<false>(im, sb),
                                          cudaFuncAttributeMaxDynamicSharedMemorySize, optin));
            CUDA_TRY(cudaFuncSetAttribute(pick_kernel<true>(im, sb),
                                          cudaFuncAttributeMaxDynamicSharedMemorySize, optin));
        }
    int per_sm = 0;
    CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(
        &per_sm, pick_kernel<false>(L->img, L->sub), kThreads, L->smem_bytes));
    if (per_sm < 1) return fail(TLL_ECUDA, "k_loglike cannot be resident on an SM");
    L->grid_cap = nsm * per_sm;
    if (L->img == IMG_GLOBAL) {
        const size_t n = (size_t)L->grid_cap * 4 * L->npix;
        CUDA_TRY(cudaMalloc(&L->d_gscr, n * sizeof(float)));
        L->dev_bytes += n * sizeof(float);
    }
    return TLL_OK;
}

void free_lens(tll_lens *L)
{
    if (!L) return;
    void *ptrs[] = {L->d_psf, L->d_pu, L->d_pv, L->d_wpack, L->d_kc, L->d_gscr,
                    L->d_stage_p, L->d_stage_o, L->d_p1, L->d_kc1, L->d_unb,
                    L->d_blur, L->d_img, L->d_res, L->d_out1};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    for (cudaEvent_t ev : L->prof_ev)
        if (ev) cudaEventDestroy(ev);
    delete L;
}

// Run one vector through the WRITE kernel; outputs stay on the device.
int run_one(tll_lens *L, const float *params_host)
{
    if (!params_host) return fail(TLL_EINVAL, "params is NULL");
    CUDA_TRY(cudaMemcpy(L->d_p1, params_host, NPAR * sizeof(float), cudaMemcpyHostToDevice));
    int rc = run_batch(L, L->d_p1, 1, L->d_out1, 0, true, L->d_kc1);
    if (rc) return rc;
    CUDA_TRY(cudaDeviceSynchronize());
    float valid = 0.0f;
    CUDA_TRY(cudaMemcpy(&valid, L->d_kc1 + K_VALID, sizeof(float), cudaMemcpyDeviceToHost));
    if (valid == 0.0f) return fail(TLL_EINVAL, "invalid parameter vector");
    return TLL_OK;
}

}  // namespace

// ------------------------------------------------------- batch context
// Reusable buffers for multi-lens launches (and their CUDA graph).
struct tll_batcher {
    int dev = 0, nsm = 0, optin = 0, dyn_smem = 0;
    bool use_graph = false;
    int cap_lenses = 0, cap_segs = 0, cap_items = 0;
    long long gslot_floats = 0;
    LensDev *d_lenses = nullptr, *h_lenses = nullptr;   // h_*: pinned staging
    Segment *d_segs = nullptr, *h_segs = nullptr;
    MultiHdr *d_hdr = nullptr, *h_hdr = nullptr;
    float *d_kc = nullptr, *d_gscr = nullptr;
    int *d_counter = nullptr;
    const double *bn_tab = nullptr;
    cudaEvent_t staged = nullptr;      // staging may be refilled after this
    bool staged_pending = false;
    cudaGraphExec_t gexec = nullptr;
    cudaStream_t gstream = nullptr;    // stream the graph was captured on
    long long launches = 0;
};

namespace {

void batcher_free_buffers(tll_batcher *b)
{
    void *dev[] = {b->d_lenses, b->d_segs, b->d_hdr, b->d_kc, b->d_gscr, b->d_counter};
    for (void *p : dev)
        if (p) cudaFree(p);
    void *host[] = {b->h_lenses, b->h_segs, b->h_hdr};
    for (void *p : host)
        if (p) cudaFreeHost(p);
    b->d_lenses = b->h_lenses = nullptr;
    b->d_segs = b->h_segs = nullptr;
    b->d_hdr = b->h_hdr = nullptr;
    b->d_kc = b->d_gscr = nullptr;
    b->d_counter = nullptr;
    if (b->gexec) {
        cudaGraphExecDestroy(b->gexec);
        b->gexec = nullptr;
    }
}

// Grow every buffer to hold (lenses, segs, items, gslot); the graph (which
// bakes in the buffer addresses and copy sizes) is dropped when anything grows.
int batcher_reserve(tll_batcher *b, int lenses, int segs, int items, long long gslot)
{
    if (lenses <= b->cap_lenses && segs <= b->cap_segs && items <= b->cap_items &&
        gslot <= b->gslot_floats && b->d_kc)
        return TLL_OK;
    if (b->staged_pending) CUDA_TRY(cudaEventSynchronize(b->staged));
    CUDA_TRY(cudaDeviceSynchronize());
    const int cl = std::max(lenses, std::max(2 * b->cap_lenses, 16));
    const int cs = std::max(segs, std::max(2 * b->cap_segs, 64));
    const int ci = std::max(items, std::max(2 * b->cap_items, 4096));
    const long long cg = std::max(gslot, b->gslot_floats);
    batcher_free_buffers(b);
    CUDA_TRY(cudaMalloc(&b->d_lenses, cl * sizeof(LensDev)));
    CUDA_TRY(cudaMalloc(&b->d_segs, cs * sizeof(Segment)));
    CUDA_TRY(cudaMalloc(&b->d_hdr, sizeof(MultiHdr)));
    CUDA_TRY(cudaMalloc(&b->d_kc, (size_t)ci * NCONST * sizeof(float)));
    CUDA_TRY(cudaMalloc(&b->d_counter, sizeof(int)));
    if (cg > 0) CUDA_TRY(cudaMalloc(&b->d_gscr, (size_t)b->nsm * cg * sizeof(float)));
    CUDA_TRY(cudaMallocHost(&b->h_lenses, cl * sizeof(LensDev)));
    CUDA_TRY(cudaMallocHost(&b->h_segs, cs * sizeof(Segment)));
    CUDA_TRY(cudaMallocHost(&b->h_hdr, sizeof(MultiHdr)));
    b->cap_lenses = cl;
    b->cap_segs = cs;
    b->cap_items = ci;
    b->gslot_floats = cg;
    return TLL_OK;
}

MultiArgs batcher_args(const tll_batcher *b)
{
    MultiArgs A;
    A.lenses = b->d_lenses;
    A.segs = b->d_segs;
    A.hdr = b->d_hdr;
    A.kc = b->d_kc;
    A.gscr = b->d_gscr;
    A.gslot_floats = b->gslot_floats;
    A.counter = b->d_counter;
    A.bn_tab = b->bn_tab;
    return A;
}

// The launch sequence: stage descriptors, reset the counter, prologue,
// multi-lens kernel.  `full` copies whole staging buffers (graph form,
// fixed sizes); otherwise only what this call uses.
int batcher_enqueue(tll_batcher *b, int nl, int ns, int total, bool full, cudaStream_t st)
{
    const int cl = full ? b->cap_lenses : nl, cs = full ? b->cap_segs : ns;
    const int items = full ? b->cap_items : total;
    CUDA_TRY(cudaMemcpyAsync(b->d_lenses, b->h_lenses, cl * sizeof(LensDev),
                             cudaMemcpyHostToDevice, st));
    CUDA_TRY(cudaMemcpyAsync(b->d_segs, b->h_segs, cs * sizeof(Segment),
                             cudaMemcpyHostToDevice, st));
    CUDA_TRY(cudaMemcpyAsync(b->d_hdr, b->h_hdr, sizeof(MultiHdr), cudaMemcpyHostToDevice, st));
    CUDA_TRY(cudaMemsetAsync(b->d_counter, 0, sizeof(int), st));
    const MultiArgs A = batcher_args(b);
    k_prologue_multi<<<(items + 127) / 128, 128, 0, st>>>(A);
    CUDA_TRY(cudaGetLastError());
    k_loglike_multi<<<b->nsm, kThreads, b->dyn_smem, st>>>(A);
    CUDA_TRY(cudaGetLastError());
    return TLL_OK;
}

}  // namespace

// ------------------------------------------- no-allocation entry point
// Scratch for tll_loglike_batch_noalloc: the per-vector constant blocks
// that tll_loglike_batch keeps in a lens-owned buffer it may grow.  A fixed
// array in the module instead, so the call itself allocates nothing; every
// GPU that loads this library holds it (3 MiB) until the process exits.
constexpr int kNoAllocMaxB = 16384;
static __device__ __align__(256) float g_noalloc_kc[kNoAllocMaxB * NCONST];

namespace {
float *g_noalloc_ptr[kMaxDevices] = {};
std::mutex g_noalloc_mu;

// Device address of g_noalloc_kc on device `dev` (current), looked up once
// per device: host code sees only a host-side stand-in for the symbol.
int noalloc_scratch(int dev, float **out)
{
    if (dev < 0 || dev >= kMaxDevices) return fail(TLL_ECUDA, "device id %d out of range", dev);
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
        void *p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_kc);
        if (e != cudaSuccess || !p)
            return fail(TLL_ECUDA, "cudaGetSymbolAddress(no-allocation scratch): %s",
                        cudaGetErrorString(e));
        g_noalloc_ptr[dev] = static_cast<float *>(p);
    }
    *out = g_noalloc_ptr[dev];
    return TLL_OK;
}
}  // namespace

// ------------------------------------------------------------------ C ABI
extern "C" {

int tll_batcher_create(int use_graph, tll_batcher **out)
{
    if (!out) return fail(TLL_EINVAL, "out is NULL");
    *out = nullptr;
    int ndev = 0;
    cudaError_t e = cudaGetDeviceCount(&ndev);
    if (e != cudaSuccess || ndev < 1)
        return fail(TLL_ECUDA, "no CUDA device: %s", cudaGetErrorString(e));
    tll_batcher *b = new (std::nothrow) tll_batcher;
    if (!b) return fail(TLL_ENOMEM, "host allocation failed");
    int rc = TLL_OK;
    auto bad = [&](int code) { delete b; return code; };
    if (cudaGetDevice(&b->dev) != cudaSuccess) return bad(fail(TLL_ECUDA, "cudaGetDevice"));
    if (cudaDeviceGetAttribute(&b->nsm, cudaDevAttrMultiProcessorCount, b->dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&b->optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, b->dev) !=
            cudaSuccess)
        return bad(fail(TLL_ECUDA, "device attributes"));
    {   // dynamic shared memory = the opt-in maximum minus the static part
        cudaFuncAttributes fa;
        if (cudaFuncGetAttributes(&fa, k_loglike_multi) != cudaSuccess)
            return bad(fail(TLL_ECUDA, "k_loglike_multi attributes"));
        b->dyn_smem = b->optin - (int)fa.sharedSizeBytes;
        if (cudaFuncSetAttribute(k_loglike_multi, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 b->dyn_smem) != cudaSuccess)
            return bad(fail(TLL_ECUDA, "k_loglike_multi shared memory"));
    }
    if ((rc = bn_table(b->dev, &b->bn_tab))) return bad(rc);
    if (cudaEventCreateWithFlags(&b->staged, cudaEventDisableTiming) != cudaSuccess)
        return bad(fail(TLL_ECUDA, "cudaEventCreate"));
    b->use_graph = use_graph != 0;
    *out = b;
    return TLL_OK;
}

void tll_batcher_destroy(tll_batcher *b)
{
    if (!b) return;
    DeviceGuard gd(b->dev);
    if (b->staged_pending) cudaEventSynchronize(b->staged);
    batcher_free_buffers(b);
    if (b->staged) cudaEventDestroy(b->staged);
    delete b;
}

int tll_batcher_run(tll_batcher *b, tll_lens *const *lenses, const float *const *params,
                    const int *counts, double *const *outs, int n, void *stream)
{
    if (!b) return fail(TLL_EINVAL, "batcher is NULL");
    if (n < 0) return fail(TLL_EINVAL, "negative lens count");
    if (n == 0) return TLL_OK;
    if (!lenses || !params || !counts || !outs) return fail(TLL_EINVAL, "NULL array");
    DeviceGuard gd(b->dev);
    cudaStream_t st = (cudaStream_t)stream;
    // distinct lenses, segments ordered by cost (largest lenses first)
    std::vector<tll_lens *> uniq;
    std::vector<int> lid(n), order(n);
    long long total = 0, gslot = 0;
    for (int k = 0; k < n; ++k) {
        tll_lens *L = lenses[k];
        if (!L) return fail(TLL_EINVAL, "lens %d is NULL", k);
        if (L->dev != b->dev) return fail(TLL_EINVAL, "lens %d is on another device", k);
        if (counts[k] < 0) return fail(TLL_EINVAL, "negative count for lens %d", k);
        if (counts[k] > 0 && (!params[k] || !outs[k]))
            return fail(TLL_EINVAL, "NULL params/out for lens %d", k);
        int u = 0;
        while (u < (int)uniq.size() && uniq[u] != L) ++u;
        if (u == (int)uniq.size()) uniq.push_back(L);
        lid[k] = u;
        order[k] = k;
        total += counts[k];
        if (L->img == IMG_GLOBAL) gslot = std::max(gslot, (long long)4 * L->npix);
        if (L->smem_bytes > (size_t)b->dyn_smem)
            return fail(TLL_EINVAL, "lens %d needs more shared memory than the batch kernel has", k);
    }
    if (total == 0) return TLL_OK;
    if (total > (1LL << 30)) return fail(TLL_EINVAL, "batch too large");
    std::stable_sort(order.begin(), order.end(), [&](int a, int c) {
        const long long wa = (long long)lenses[a]->npix * lenses[a]->sub * lenses[a]->sub;
        const long long wc = (long long)lenses[c]->npix * lenses[c]->sub * lenses[c]->sub;
        return wa > wc;
    });
    int rc = batcher_reserve(b, (int)uniq.size(), n, (int)total, gslot);
    if (rc) return rc;
    if (b->staged_pending) CUDA_TRY(cudaEventSynchronize(b->staged));
    for (size_t u = 0; u < uniq.size(); ++u) b->h_lenses[u] = lens_dev(uniq[u]);
    int first = 0, ns = 0;
    for (int k : order) {
        if (counts[k] == 0) continue;
        Segment &sg = b->h_segs[ns++];
        sg.lens = lid[k];
        sg.first = first;
        sg.count = counts[k];
        sg.pad = 0;
        sg.params = params[k];
        sg.out = outs[k];
        first += counts[k];
    }
    b->h_hdr->total = (int)total;
    b->h_hdr->nseg = ns;
    const bool graph = b->use_graph && st != nullptr;
    if (graph) {
        if (!b->gexec || b->gstream != st) {
            if (b->gexec) {
                cudaGraphExecDestroy(b->gexec);
                b->gexec = nullptr;
            }
            cudaGraph_t g = nullptr;
            CUDA_TRY(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
            rc = batcher_enqueue(b, 0, 0, 0, true, st);
            const cudaError_t ce = cudaStreamEndCapture(st, &g);
            if (rc) {
                if (g) cudaGraphDestroy(g);
                return rc;
            }
            if (ce != cudaSuccess) return fail(TLL_ECUDA, "graph capture: %s", cudaGetErrorString(ce));
            const cudaError_t ie = cudaGraphInstantiate(&b->gexec, g, 0);
            cudaGraphDestroy(g);
            if (ie != cudaSuccess)
                return fail(TLL_ECUDA, "graph instantiate: %s", cudaGetErrorString(ie));
            b->gstream = st;
        }
        CUDA_TRY(cudaGraphLaunch(b->gexec, st));
    } else {
        rc = batcher_enqueue(b, (int)uniq.size(), ns, (int)total, false, st);
        if (rc) return rc;
    }
    CUDA_TRY(cudaEventRecord(b->staged, st));
    b->staged_pending = true;
    ++b->launches;
    return TLL_OK;
}

int tll_loglike_batch_noalloc(tll_lens *L, const float *params, int B, double *out,
                              void *stream)
{
    if (!L) return fail(TLL_EINVAL, "lens is NULL");
    if (B < 0) return fail(TLL_EINVAL, "negative batch size");
    if (B > kNoAllocMaxB)
        return fail(TLL_EINVAL,
                    "batch of %d vectors exceeds the no-allocation limit of %d per call",
                    B, kNoAllocMaxB);
    if (B == 0) return TLL_OK;
    if (!params || !out) return fail(TLL_EINVAL, "NULL params or out");
    DeviceGuard gd(L->dev);
    float *kc = nullptr;
    const int rc = noalloc_scratch(L->dev, &kc);
    if (rc) return rc;
    // k_prologue writes all NCONST entries of each of the B blocks before
    // k_loglike reads them on the same stream, so nothing needs clearing.
    return run_batch(L, params, B, out, (cudaStream_t)stream, false, kc);
}


const char *tll_last_error(void) { return g_err; }

int tll_version(void) { return 100; }

int tll_create_lens(const float *image, const float *noise, const float *psf,
                    int psf_size, const tll_grid_t *grid, int flags, tll_lens **out)
{
    g_err[0] = 0;
    if (!out) return fail(TLL_EINVAL, "out is NULL");
    *out = nullptr;
    if (!image || !noise || !psf || !grid) return fail(TLL_EINVAL, "NULL input pointer");
    const tll_grid_t g = *grid;
    if (g.nx < 1 || g.ny < 1 || g.nx > TLL_MAX_SIDE || g.ny > TLL_MAX_SIDE)
        return fail(TLL_EINVAL, "image size %d x %d out of range", g.ny, g.nx);
    if (g.sub < 1 || g.sub > TLL_MAX_SUB)
        return fail(TLL_EINVAL, "supersampling %d out of range", g.sub);
    if (!(g.pixel_scale > 0.0f) || !isfinite(g.pixel_scale) || !isfinite(g.x0) ||
        !isfinite(g.y0))
        return fail(TLL_EINVAL, "bad grid geometry");
    if (psf_size < 1 || psf_size > TLL_MAX_PSF || psf_size % 2 == 0)
        return fail(TLL_EINVAL, "PSF side %d must be odd and <= %d", psf_size, TLL_MAX_PSF);
    const int mode = flags & 0xff;
    if (mode != TLL_AMP_LINEAR && mode != TLL_AMP_FIXED)
        return fail(TLL_EINVAL, "unknown amplitude mode %d", mode);
    const int K = psf_size, npix = g.nx * g.ny;
    double psum = 0.0;
    for (int t = 0; t < K * K; ++t) {
        if (!isfinite(psf[t])) return fail(TLL_EINVAL, "non-finite PSF entry");
        psum += psf[t];
    }
    if (!(psum > 0.0)) return fail(TLL_EINVAL, "PSF sum must be > 0");

    int dev = 0;
    {
        int ndev = 0;
        cudaError_t e = cudaGetDeviceCount(&ndev);
        if (e != cudaSuccess || ndev < 1)
            return fail(TLL_ECUDA, "no CUDA device: %s", cudaGetErrorString(e));
        CUDA_TRY(cudaGetDevice(&dev));
    }
    tll_lens *L = new (std::nothrow) tll_lens;
    if (!L) return fail(TLL_ENOMEM, "host allocation failed");
    L->dev = dev;
    L->nx = g.nx; L->ny = g.ny; L->npix = npix; L->sub = g.sub; L->K = K;
    L->flags = flags; L->mode = mode;
    L->dpix = g.pixel_scale; L->x0 = g.x0; L->y0 = g.y0; L->psf_sum = psum;

    // PSF, unit sum (Eq. 3); separable if it is an outer product to rounding
    std::vector<float> pn(K * K), pu(K), pv(K);
    for (int t = 0; t < K * K; ++t) pn[t] = (float)((double)psf[t] / psum);
    int sep = 0;
    if (!(flags & TLL_FLAG_DIRECT_CONV)) {
        int r0 = 0, c0 = 0;
        float best = -1.0f;
        for (int r = 0; r < K; ++r)
            for (int c = 0; c < K; ++c)
                if (fabsf(pn[r * K + c]) > best) { best = fabsf(pn[r * K + c]); r0 = r; c0 = c; }
        if (best > 0.0f) {
            sep = 1;
            std::vector<double> u(K), v(K);
            for (int r = 0; r < K; ++r) u[r] = pn[r * K + c0];
            for (int c = 0; c < K; ++c) v[c] = (double)pn[r0 * K + c] / (double)pn[r0 * K + c0];
            for (int r = 0; r < K && sep; ++r)
                for (int c = 0; c < K; ++c) {
                    const double kv = pn[r * K + c], uv = u[r] * v[c];
                    if (fabs(kv - uv) > 4.8e-7 * fabs(kv) + 1e-37) { sep = 0; break; }
                }
            for (int r = 0; r < K; ++r) pu[r] = (float)u[r];
            for (int c = 0; c < K; ++c) pv[c] = (float)v[c];
        }
    }
    L->sep = sep;
    if (sep) {
        L->taps_u = pu;
        L->taps_v = pv;
    }

    // weights (Eq. 5): w = 1/sigma^2 as a float pair, w*d likewise; masked
    // pixels get 0.  dWd = sum w d^2, lognorm = -sum log(2 pi sigma^2)/2.
    std::vector<float4> wp(npix);
    double dWd = 0.0, lognorm = 0.0;
    for (int t = 0; t < npix; ++t) {
        const double s = noise[t], d = image[t];
        float4 q = make_float4(0.f, 0.f, 0.f, 0.f);
        if (isfinite(s) && s > 0.0 && isfinite(d)) {
            const double w = 1.0 / (s * s), wd = w * d;
            q.x = (float)w; q.y = (float)(w - (double)q.x);
            q.z = (float)wd; q.w = (float)(wd - (double)q.z);
            dWd += wd * d;
            lognorm -= 0.5 * log(2.0 * M_PI * s * s);
        }
        wp[t] = q;
    }
    L->dWd = dWd;
    L->lognorm = lognorm;

    int rc = TLL_OK;
    auto alloc = [&](void **p, size_t bytes) -> int {
        cudaError_t e = cudaMalloc(p, bytes);
        if (e != cudaSuccess)
            return fail(e == cudaErrorMemoryAllocation ? TLL_ENOMEM : TLL_ECUDA,
                        "cudaMalloc(%zu): %s", bytes, cudaGetErrorString(e));
        L->dev_bytes += bytes;
        return TLL_OK;
    };
    if ((rc = alloc((void **)&L->d_psf, K * K * sizeof(float))) ||
        (rc = alloc((void **)&L->d_pu, K * sizeof(float))) ||
        (rc = alloc((void **)&L->d_pv, K * sizeof(float))) ||
        (rc = alloc((void **)&L->d_wpack, npix * sizeof(float4))) ||
        (rc = alloc((void **)&L->d_p1, NPAR * sizeof(float))) ||
        (rc = alloc((void **)&L->d_kc1, NCONST * sizeof(float))) ||
        (rc = alloc((void **)&L->d_unb, 2 * npix * sizeof(float))) ||
        (rc = alloc((void **)&L->d_blur, 2 * npix * sizeof(float))) ||
        (rc = alloc((void **)&L->d_img, npix * sizeof(float))) ||
        (rc = alloc((void **)&L->d_res, 8 * sizeof(double))) ||
        (rc = alloc((void **)&L->d_out1, sizeof(double)))) {
        free_lens(L);
        return rc;
    }
    cudaError_t e = cudaSuccess;
    if (e == cudaSuccess) e = cudaMemcpy(L->d_psf, pn.data(), K * K * sizeof(float), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(L->d_pu, pu.data(), K * sizeof(float), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(L->d_pv, pv.data(), K * sizeof(float), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(L->d_wpack, wp.data(), npix * sizeof(float4), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        free_lens(L);
        return fail(TLL_ECUDA, "cudaMemcpy: %s", cudaGetErrorString(e));
    }
    if ((rc = configure(L)) || (rc = ensure_kc(L, 1024)) || (rc = bn_table(dev, &L->bn_tab))) {
        free_lens(L);
        return rc;
    }
    *out = L;
    return TLL_OK;
}

void tll_destroy_lens(tll_lens *L)
{
    if (!L) return;
    DeviceGuard gd(L->dev);
    free_lens(L);
}

int tll_lens_footprint(const tll_lens *L, size_t *bytes)
{
    if (!L || !bytes) return fail(TLL_EINVAL, "NULL argument");
    *bytes = L->dev_bytes;
    return TLL_OK;
}

int tll_lens_info(const tll_lens *L, int *nx, int *ny, int *sub, int *psf_size,
                  int *flags, int *separable)
{
    if (!L) return fail(TLL_EINVAL, "lens is NULL");
    if (nx) *nx = L->nx;
    if (ny) *ny = L->ny;
    if (sub) *sub = L->sub;
    if (psf_size) *psf_size = L->K;
    if (flags) *flags = L->flags;
    if (separable) *separable = L->sep;
    return TLL_OK;
}

int tll_profile_enable(tll_lens *L, int on)
{
    if (!L) return fail(TLL_EINVAL, "lens is NULL");
    DeviceGuard gd(L->dev);
    if (on && !L->prof_ev[0])
        for (auto &ev : L->prof_ev) CUDA_TRY(cudaEventCreate(&ev));
    L->prof_on = on != 0;
    L->prof_recorded = false;
    return TLL_OK;
}

int tll_profile_last(tll_lens *L, float *prologue_ms, float *main_ms)
{
    if (!L) return fail(TLL_EINVAL, "lens is NULL");
    if (!L->prof_on || !L->prof_recorded)
        return fail(TLL_EINVAL, "profiling not enabled or no batch recorded");
    DeviceGuard gd(L->dev);
    CUDA_TRY(cudaEventSynchronize(L->prof_ev[2]));
    float a = 0.f, b = 0.f;
    CUDA_TRY(cudaEventElapsedTime(&a, L->prof_ev[0], L->prof_ev[1]));
    CUDA_TRY(cudaEventElapsedTime(&b, L->prof_ev[1], L->prof_ev[2]));
    if (prologue_ms) *prologue_ms = a;
    if (main_ms) *main_ms = b;
    return TLL_OK;
}

int tll_loglike_batch(tll_lens *L, const float *params, int B, double *out, void *stream)
{
    if (!L) return fail(TLL_EINVAL, "lens is NULL");
    if (B < 0) return fail(TLL_EINVAL, "negative batch size");
    if (B == 0) return TLL_OK;
    if (!params || !out) return fail(TLL_EINVAL, "NULL params or out");
    DeviceGuard gd(L->dev);
    int rc = ensure_kc(L, B);
    if (rc) return rc;
    return run_batch(L, params, B, out, (cudaStream_t)stream, false, L->d_kc);
}

int tll_loglike_batch_host(tll_lens *L, const float *params, int B, double *out,
                           void *stream)
{
    if (!L) return fail(TLL_EINVAL, "lens is NULL");
    if (B < 0) return fail(TLL_EINVAL, "negative batch size");
    if (B == 0) return TLL_OK;
    if (!params || !out) return fail(TLL_EINVAL, "NULL params or out");
    DeviceGuard gd(L->dev);
    cudaStream_t st = (cudaStream_t)stream;
    if (B > L->stage_cap) {
        const int cap = std::max(B, 2 * L->stage_cap);
        float *p = nullptr;
        double *o = nullptr;
        CUDA_TRY(cudaMalloc(&p, (size_t)cap * NPAR * sizeof(float)));
        cudaError_t e = cudaMalloc(&o, (size_t)cap * sizeof(double));
        if (e != cudaSuccess) {
            cudaFree(p);
            return fail(TLL_ENOMEM, "cudaMalloc: %s", cudaGetErrorString(e));
        }
        if (L->d_stage_p) cudaFree(L->d_stage_p);
        if (L->d_stage_o) cudaFree(L->d_stage_o);
        L->dev_bytes += ((size_t)cap - L->stage_cap) * (NPAR * sizeof(float) + sizeof(double));
        L->d_stage_p = p;
        L->d_stage_o = o;
        L->stage_cap = cap;
    }
    int rc = ensure_kc(L, B);
    if (rc) return rc;
    CUDA_TRY(cudaMemcpyAsync(L->d_stage_p, params, (size_t)B * NPAR * sizeof(float),
                             cudaMemcpyHostToDevice, st));
    rc = run_batch(L, L->d_stage_p, B, L->d_stage_o, st, false, L->d_kc);
    if (rc) return rc;
    CUDA_TRY(cudaMemcpyAsync(out, L->d_stage_o, (size_t)B * sizeof(double),
                             cudaMemcpyDeviceToHost, st));
    CUDA_TRY(cudaStreamSynchronize(st));
    return TLL_OK;
}

int tll_model_columns(tll_lens *L, const float *params, float *lens_out, float *src_out,
                      int blurred)
{
    if (!L) return fail(TLL_EINVAL, "lens is NULL");
    if (!lens_out || !src_out) return fail(TLL_EINVAL, "NULL output");
    DeviceGuard gd(L->dev);
    int rc = run_one(L, params);
    if (rc) return rc;
    const float *src = blurred ? L->d_blur : L->d_unb;
    const size_t n = (size_t)L->npix * sizeof(float);
    CUDA_TRY(cudaMemcpy(lens_out, src, n, cudaMemcpyDeviceToHost));
    CUDA_TRY(cudaMemcpy(src_out, src + L->npix, n, cudaMemcpyDeviceToHost));
    return TLL_OK;
}

int tll_model_image(tll_lens *L, const float *params, float *image_out, float *amps_out,
                    double *loglike_out)
{
    if (!L) return fail(TLL_EINVAL, "lens is NULL");
    if (!image_out) return fail(TLL_EINVAL, "NULL output");
    DeviceGuard gd(L->dev);
    int rc = run_one(L, params);
    if (rc) return rc;
    k_combine<<<std::max(1, std::min(1024, (L->npix + 255) / 256)), 256>>>(
        L->d_blur, L->d_res, L->npix, L->d_img);
    CUDA_TRY(cudaGetLastError());
    CUDA_TRY(cudaMemcpy(image_out, L->d_img, (size_t)L->npix * sizeof(float),
                        cudaMemcpyDeviceToHost));
    double res[8];
    CUDA_TRY(cudaMemcpy(res, L->d_res, sizeof res, cudaMemcpyDeviceToHost));
    if (amps_out) {
        amps_out[0] = (float)res[5];
        amps_out[1] = (float)res[6];
    }
    if (loglike_out) *loglike_out = res[7];
    return TLL_OK;
}

}  // extern "C"
