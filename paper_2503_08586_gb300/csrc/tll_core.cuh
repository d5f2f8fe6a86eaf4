// tll_core.cuh -- types and helpers shared by the likelihood kernels and
// the compiled convolutions (separate translation units, relocatable
// device code).
#pragma once

#include <cuda_runtime.h>

#include "tll.h"
#include "tll_device.cuh"
#include "tll_stretch.cuh"

namespace tll {

constexpr int kThreads = 1024;     // CTA size of k_loglike (64 registers, 32 warps per SM)
constexpr int kHMax = 8;           // in-place row pass holds nx <= 32*kHMax
constexpr int kRedBytes = 32 * 5 * 8;   // the warps' five partial sums, a float pair each

constexpr int kMaxTaps = 32;   // separable PSF factors carried in the parameter block
constexpr int kMaxK = 31;      // largest PSF side of the compiled convolutions

// Row stride of the full PSF in LensDev::tk: K + 1 for the odd sides K,
// so that every row starts on an 8-byte boundary and its taps are read in
// pairs; the extra entry of a row is zero.
__host__ __device__ constexpr int tap_stride(int K) { return K + 1; }

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
    int band_rows;    // IMG_BANDED: output rows per shared-memory band
    int epl;          // elliptical power-law mass: 22 parameters per vector
    // Pixels the batched kernels trace: tlist[0 .. ntrace) (row-major pixel
    // indices) when masked pixels leave some pixels out of reach of every
    // unmasked one through the PSF, else tlist = null (all npix pixels).
    const int *tlist;
    int ntrace;
    int nc_smem;      // multi-column kernel: dynamic shared memory of the launch
    // n / nx as __umulhi(n, nx_mul), nx_mul = ceil(2^32 / nx): exact for
    // n < 2^32 / nx, which nx_fast records for every index a kernel divides
    // (pixel indices and column-pass units, n < nx (ny + 8)); 0 for nx = 1
    unsigned nx_mul;
    int nx_fast;
    float tu[kMaxTaps], tv[kMaxTaps];   // the separable factors again, by value
    // the full PSF (direct convolution), row r at tk[r * tap_stride(K)]
    alignas(8) float tk[kMaxK * (kMaxK + 1)];
};

// Asynchronous global -> shared copies (cp.async): the copies of a thread
// complete at its cp_async_wait_all (or the group's wait), visible to the
// other threads after a barrier.  cp_async4_zfill with valid = false reads
// nothing from src and writes 0.
__device__ __forceinline__ void cp_async4_zfill(float *dst, const float *src, bool valid)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(
                     (unsigned)__cvta_generic_to_shared(dst)),
                 "l"(src), "r"(valid ? 4 : 0)
                 : "memory");
}
__device__ __forceinline__ void cp_async4(float *dst, const float *src)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(
                     (unsigned)__cvta_generic_to_shared(dst)),
                 "l"(src)
                 : "memory");
}
__device__ __forceinline__ void cp_async16(float4 *dst, const float4 *src)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(
                     (unsigned)__cvta_generic_to_shared(dst)),
                 "l"(src)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// Barrier over the threads taking part in a phase: BAR 0 is the whole CTA
// (__syncthreads); BAR > 0 is named barrier BAR over the first nthr threads
// (a multiple of 32), which leaves the other warps free for other work.
template <int BAR>
__device__ __forceinline__ void phase_sync(int nthr)
{
    if constexpr (BAR == 0)
        __syncthreads();
    else
        asm volatile("bar.sync %0, %1;" ::"n"(BAR), "r"(nthr) : "memory");
}

// Row of index n in a row-major image of L.nx columns.
__device__ __forceinline__ int div_nx(const LensDev &L, int n)
{
    return L.nx_fast ? (int)__umulhi((unsigned)n, L.nx_mul) : n / L.nx;
}

// Image placement in k_loglike.
enum : int {
    IMG_GLOBAL = 0,   // per-CTA global scratch slot (L2), generic convolution
    IMG_SMEM = 1,     // shared memory, unpadded, generic convolution
    IMG_PADDED = 2,   // shared memory with zero halos, convolution compiled per K
    IMG_BANDED = 3    // global slot, convolved band by band through a zero-padded
                      // shared-memory buffer, convolution compiled per K
};

struct RunArgs {
    const float *kc;     // [B][NCONST]
    // fused: the kernel decodes its own vectors into kc (each CTA at most
    // one vector: batches no larger than the grid) from params [B][np]
    // (grid centre XC, YC, subpixel step d, b_n table), no separate prologue
    int fused, epl, np;
    const float *params;
    double XC, YC, d;
    const double *bn_tab;
    int B;
    double *out;         // [B]
    float *gscr;         // global image scratch, gslot floats per CTA
    long long gslot;
    float *wr_unblurred; // WRITE: [2][npix]
    float *wr_blurred;   // WRITE: [2][npix]
    float *wr_blurred_s; // WRITE: the second column there instead, when not null
    double *wr_res;      // WRITE: [8] All Als Ass bl bs sl ss logL
    // fused (only): a stretch-move half step around the likelihood -- each
    // vector's walker proposed into its params row before the decode,
    // accepted or rejected after its log L (smp_on)
    StretchStep smp;
    int smp_on;
};

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

// --------------------------------------------------- padded convolution
// Separable PSF with compile-time side K on the zero-padded shared-memory
// layout: image pixel (i, j) at P[(h + i) W + HL + j], HL = h rounded up to
// a multiple of 4; rows [0, h) and [h + ny, ...) and the columns outside
// [HL, HL + nx) hold zeros, so no tap needs a bounds check.
//  Row pass (in place, one warp per row): a lane computes 4 adjacent
//  outputs from one window of K + 3 values read as float4s.
//  Column pass: a thread takes one column x CR rows (CR = 4 or 5, whichever
//  needs fewer rounds of the CTA's threads), reads CR + K - 1 values of its
//  column and computes CR outputs per channel.
// Taps come from the parameter block (compile-time indices).  kCR: the
// largest CR, the zero rows kept below the image for the last row block.
constexpr int kCR = 5;

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

// Multi-lens work list: segment s covers items [first, first + count) of
// lens `lens`, reading params[k] and writing out[k]; segments are grouped
// (same supersampling and convolution class) and each group is one launch.
struct Segment {
    int lens, first, count, pad;
    const float *params;
    double *out;
};
struct MultiHdr {        // one group: items [first, first + total), segments [seg0, seg0 + nseg)
    int first, total, seg0, nseg;
};
constexpr int kMaxComps = 32;       // components (columns) per lens
constexpr int kPassMax = 8;         // components of one trace pass (lens-plane Gaussians)
constexpr int kMaxPasses = 16;      // trace passes per vector

// A multi-column lens's component list and its trace schedule (kernel
// parameter; tll_multi.cuh).
struct MultiDev {
    int nc, npar, npass;
    int type[kMaxComps], plane[kMaxComps], flags[kMaxComps];
    float scale[kMaxComps], index[kMaxComps];
    // pass p: plane, component count, Gaussian-only (up to kPassMax
    // components) or mixed (up to kPassMix), component indices
    int pass_plane[kMaxPasses], pass_n[kMaxPasses], pass_gauss[kMaxPasses];
    int pass_comp[kMaxPasses][kPassMax];
};

// The lenses of one multi-lens launch, by value in the kernel's
// parameters (constant bank) rather than copied to shared memory: read
// through a block-uniform slot index, the lens constants (the PSF taps of
// the convolutions' inner loops above all) stay operands of the arithmetic
// instead of shared-memory loads.  Slot s: lens[s], its vectors are items
// [first[s], first[s] + count[s]) of the work list, handed out by counter
// A.counter[kMultiCounters + g kMultiSlots + s]; CTAs [cta_end[s-1],
// cta_end[s]) start on slot s (in proportion to its work) and move on to
// the following slots when it runs dry.  Multi-column lenses also carry
// their component lists (md[s]; 28.8 KB in all of the 32 KB the parameters
// may take).
constexpr int kMultiSlots = 5;
constexpr int kMultiCounters = 1024;   // groups per run; slot counters follow
struct LensSlots {
    int n;
    int cta_end[kMultiSlots];
    int first[kMultiSlots], count[kMultiSlots];
    LensDev lens[kMultiSlots];
    MultiDev md[kMultiSlots];
};
struct MultiArgs {
    const LensDev *lenses;
    const MultiDev *mdevs;     // per lens: its component list (nc = 0: two columns)
    const Segment *segs;
    const MultiHdr *groups;
    const MultiHdr *all;       // the whole work list (prologue)
    float *kc;                 // [total][NCONST]
    float *gscr;               // per-CTA global image slots
    long long gslot_floats;
    int *counter;              // one work counter per group, zero at launch
    const double *bn_tab;
};

// Largest s in [s0, s0 + n) with segs[s].first <= t.
__host__ __device__ inline int find_segment(const Segment *segs, int s0, int n, int t)
{
    int lo = s0, hi = s0 + n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (segs[mid].first <= t) lo = mid; else hi = mid - 1;
    }
    return lo;
}

}  // namespace tll
