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
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <new>
#include <vector>

#include "tll.h"
#include "tll_internal.h"
#include "tll_multi.cuh"
#include "tll_split.cuh"

using namespace tll;

namespace {

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

// -------------------------------------------------------------- kernels
// Block (32, 4): warp y decodes part y (decode_vector) of vectors
// 32 blockIdx.x + [0, 32).  The FP64 work of a vector is split four ways
// over four warps (four sub-partitions) rather than run by one thread:
// GB300's FP64 pipe takes a warp instruction every 64 cycles or so, so a
// vector's decode time is set by its longest serial FP64 chain.
constexpr int kPrologueVectors = 32;
__global__ void __launch_bounds__(128) k_prologue(const float *__restrict__ params, int B,
                                                  float *__restrict__ kc, double XC, double YC,
                                                  double d, const double *__restrict__ bn_tab,
                                                  int epl)
{
    const int b = blockIdx.x * kPrologueVectors + threadIdx.x;
    if (b < B)
        decode_vector(params + (size_t)b * (epl ? NPAR_EPL : NPAR), kc + (size_t)b * NCONST,
                      XC, YC, d, bn_tab, epl != 0, threadIdx.y);
}

// One thread per node of the b_n table (run once per device).
__global__ void k_bn_table(double *__restrict__ tab)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= 2 * BN_SEG) return;
    const int seg = t / BN_SEG, k = t - seg * BN_SEG - 1;
    tab[t] = sersic_bn_dev(bn_node(seg, k));
}

// ------------------------------------------------- multi-lens prologue
// Block (32, 4) as k_prologue: a two-column vector's four parts on four
// warps; a multi-component vector decoded whole by warp 0.
__global__ void __launch_bounds__(128) k_prologue_multi(const __grid_constant__ MultiArgs A)
{
    const int t = blockIdx.x * kPrologueVectors + threadIdx.x;
    if (t >= A.all->total) return;
    const Segment &sg = A.segs[find_segment(A.segs, 0, A.all->nseg, t)];
    const LensDev &L = A.lenses[sg.lens];
    const MultiDev &M = A.mdevs[sg.lens];
    if (M.nc > 0) {
        if (threadIdx.y == 0)
            decode_multi(sg.params + (size_t)(t - sg.first) * M.npar, A.kc + (size_t)t * NCONST,
                         L, M, A.bn_tab);
    } else {
        decode_vector(sg.params + (size_t)(t - sg.first) * (L.epl ? NPAR_EPL : NPAR),
                      A.kc + (size_t)t * NCONST, L.XC, L.YC, L.d, A.bn_tab, L.epl != 0,
                      threadIdx.y);
    }
}

// Multi-component prologue: one thread per vector.
__global__ void k_prologue_nc(const float *__restrict__ params, int B, float *__restrict__ kc,
                              const __grid_constant__ LensDev L, const __grid_constant__ MultiDev M,
                              const double *__restrict__ bn_tab)
{
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b < B) decode_multi(params + (size_t)b * M.npar, kc + (size_t)b * NCONST, L, M, bn_tab);
}

// Model image of one multi-component vector: sum_k s_k M_k (Eq. 7), FP64
// then rounded; res holds the amplitudes.
__global__ void k_combine_nc(const float *__restrict__ cols, const double *__restrict__ res,
                             int nc, int npix, float *__restrict__ img)
{
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < npix;
         t += gridDim.x * blockDim.x) {
        double v = 0.0;
        for (int k = 0; k < nc; ++k) v += res[k] * (double)cols[(size_t)k * npix + t];
        img[t] = (float)v;
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
namespace {
// Launch shape of the likelihood kernels for one lens: CTA size, CTAs
// resident per SM, where the two images live, and what that costs.
struct Shape {
    int threads = kThreads;   // CTA size (multiple of 32, <= kThreads)
    int per_sm = 1;           // resident CTAs per SM at this shared memory
    int img = IMG_GLOBAL;     // IMG_*
    int band_rows = 0;        // IMG_BANDED output rows per band
    size_t smem = 0;          // dynamic shared memory per CTA
    int grid_cap = 0;         // nsm * per_sm: persistent CTAs of one launch
    long long gslot = 0;      // floats of global image slot per CTA (0: none)
    float ms = 0.0f;          // tuning time per launch (0: not timed)
};
}  // namespace

struct tll_lens {
    int dev = 0;
    int nx = 0, ny = 0, npix = 0, sub = 0, K = 0, flags = 0, mode = 0, sep = 0;
    int epl = 0, nparam = NPAR;   // mass model: SIE (21 parameters) or EPL (22)
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
    Shape shape;          // launch shape of the batched likelihood kernels
    bool tuned = false;   // shape chosen by tll_autotune (or its cache)
    int img_write = 0;    // placement of the write-out (model image) launches
    size_t smem_write = 0;
    int W = 0, HL = 0;    // padded layout geometry
    std::vector<float> taps_u, taps_v, psf_norm;
    long long gscr_floats = 0;   // size of d_gscr
    // split pipeline (tll_set_conv): image buffers for split_cap vectors,
    // Toeplitz tiles, the tensor-core kernel's status word
    int conv_variant = TLL_CONV_FUSED;
    float *d_unbl = nullptr, *d_sblur = nullptr, *d_tiles = nullptr;
    float *d_thi = nullptr, *d_tlo = nullptr;   // TF32 parts, chunk-major (Toeplitz)
    CUtensorMap tm_hi, tm_lo;                   // their tensor maps
    void *d_bpart[3] = {nullptr, nullptr, nullptr};   // BF16 parts (split-BF16 Toeplitz)
    CUtensorMap tm_b[3];                        // their tensor maps
    uint16_t *d_btiles = nullptr;               // BF16 Toeplitz tiles
    size_t bf_part_bytes_each = 0;
    int *d_tc_status = nullptr;
    int split_cap = 0;
    size_t tc_part_bytes = 0;
    const double *bn_tab = nullptr;   // per-device b_n table (not owned)
    size_t dev_bytes = 0;             // device memory this lens holds
    cudaEvent_t prof_ev[3] = {nullptr, nullptr, nullptr};
    bool prof_on = false, prof_recorded = false;
    // multi-component light (tll_set_light): nc > 0 columns, their list and
    // trace schedule, the multi-column kernel's shape and per-CTA slots
    // pixels the batched kernels trace (masked lenses; null: all)
    int *d_tlist = nullptr;
    int ntrace = 0;
    int nc = 0;
    MultiDev md = {};
    Shape nc_shape;
    float *d_nscr = nullptr;
    long long nscr_floats = 0;
    double *d_nres = nullptr;   // amplitudes and log L of the model-image launch
};

namespace {

// Largest parameter vector of any model: 15 + 2 per component + the slope.
constexpr int kMaxParams = kMultiHead + 2 * kMaxComps + 1;

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
    d.W = L->W; d.HL = L->HL; d.img = L->shape.img; d.band_rows = L->shape.band_rows;
    d.epl = L->epl;
    if (L->nc) {   // the multi-column kernels' placement
        d.img = L->nc_shape.img;
        d.band_rows = L->nc_shape.band_rows;
        d.nc_smem = (int)L->nc_shape.smem;
    }
    d.tlist = L->d_tlist;
    d.ntrace = L->d_tlist ? L->ntrace : L->npix;
    d.nx_mul = (unsigned)(((1ULL << 32) + (unsigned long long)L->nx - 1) / L->nx);
    // (nx = 1: ceil(2^32 / nx) does not fit 32 bits; the division is used)
    d.nx_fast = L->nx > 1 && (unsigned long long)L->nx * L->nx * (L->ny + 8) < (1ULL << 32) ? 1 : 0;
    for (int k = 0; k < kMaxK * (kMaxK + 1); ++k) d.tk[k] = 0.0f;
    if (L->K <= kMaxK) {
        const int ts = tap_stride(L->K);
        for (int r = 0; r < L->K; ++r)
            for (int c = 0; c < L->K; ++c) d.tk[r * ts + c] = L->psf_norm[r * L->K + c];
    }
    grid_centre(L, &d.XC, &d.YC);
    d.d = (double)L->dpix / L->sub;
    for (int k = 0; k < kMaxTaps; ++k) {
        d.tu[k] = k < (int)L->taps_u.size() ? L->taps_u[k] : 0.0f;
        d.tv[k] = k < (int)L->taps_v.size() ? L->taps_v[k] : 0.0f;
    }
    return d;
}

// ------------------------------------------------------------ registry
}  // namespace

namespace tll {
extern const KernelSet kernel_set_generic, kernel_set_k01, kernel_set_k05, kernel_set_k09,
    kernel_set_k13, kernel_set_k17, kernel_set_k21, kernel_set_k25, kernel_set_k29;
}

namespace {

const KernelSet *const kSets[] = {&kernel_set_generic, &kernel_set_k01, &kernel_set_k05,
                                  &kernel_set_k09, &kernel_set_k13, &kernel_set_k17,
                                  &kernel_set_k21, &kernel_set_k25, &kernel_set_k29};

// Convolution class of a placement: the compiled side K, or 0 (generic).
int conv_class(int img, int K) { return (img == IMG_PADDED || img == IMG_BANDED) ? K : 0; }

SingleKernel find_single(int sub, int Kc, bool write)
{
    for (const KernelSet *ks : kSets)
        if (SingleKernel f = ks->single(sub, Kc, write)) return f;
    return nullptr;
}

MultiKernel find_multi(int sub, int Kc)
{
    for (const KernelSet *ks : kSets)
        if (MultiKernel f = ks->multi(sub, Kc)) return f;
    return nullptr;
}

NcKernel find_nc(int sub, int Kc)
{
    for (const KernelSet *ks : kSets)
        if (NcKernel f = ks->nc(sub, Kc)) return f;
    return nullptr;
}

MultiKernel find_nc_multi(int sub, int Kc)
{
    for (const KernelSet *ks : kSets)
        if (MultiKernel f = ks->nc_multi(sub, Kc)) return f;
    return nullptr;
}

int launch_main(const tll_lens *L, const RunArgs &R, int grid, bool write, cudaStream_t st)
{
    LensDev d = lens_dev(L);
    if (write) d.img = L->img_write;
    const SingleKernel kern = write ? find_single(L->sub, 0, true)
                                    : find_single(L->sub, conv_class(L->shape.img, L->K), false);
    if (!kern) return fail(TLL_ECUDA, "no kernel for s=%d K=%d", L->sub, L->K);
    kern<<<grid, write ? kThreads : L->shape.threads, write ? L->smem_write : L->shape.smem,
           st>>>(d, R);
    CUDA_TRY(cudaGetLastError());
    return TLL_OK;
}

// The split pipeline for B vectors whose constants are in kc: in chunks of
// split_cap vectors, trace -> convolution (direct or Toeplitz on the tensor
// cores) -> sums, with the images in the lens's split buffers.
int run_split(tll_lens *L, const float *kc, int B, double *out, cudaStream_t st)
{
    int nsm = 0;
    CUDA_TRY(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, L->dev));
    const LensDev d = lens_dev(L);
    for (int b0 = 0; b0 < B; b0 += L->split_cap) {
        const int nb = std::min(L->split_cap, B - b0);
        const float *k = kc + (size_t)b0 * NCONST;
        CUDA_TRY(launch_trace_split(d, k, nb, L->d_unbl, std::min(nb, nsm), st));
        if (L->conv_variant == TLL_CONV_SPLIT_TOEPLITZ_TC)
            CUDA_TRY(launch_conv_tc(d, L->d_unbl, nb, L->d_thi, L->d_tlo, L->tm_hi, L->tm_lo,
                                    L->d_sblur, L->d_tiles, L->d_tc_status, nsm, st));
        else if (L->conv_variant == TLL_CONV_SPLIT_TOEPLITZ_BF16)
            CUDA_TRY(launch_conv_bf(d, L->d_unbl, nb, L->d_bpart, L->tm_b, L->d_sblur,
                                    L->d_btiles, L->d_tc_status, nsm, st));
        else
            CUDA_TRY(launch_conv_direct_split(d, L->d_unbl, nb, L->d_sblur,
                                              std::min(2 * nb, nsm), st));
        CUDA_TRY(launch_sums_split(d, k, L->d_sblur, nb, out + b0, std::min(nb, nsm), st));
    }
    return TLL_OK;
}

int run_batch(tll_lens *L, const float *params, int B, double *out, cudaStream_t st,
              bool write, float *kc, const StretchStep *ss = nullptr)
{
    const bool prof = L->prof_on && !write;
    if (prof) CUDA_TRY(cudaEventRecord(L->prof_ev[0], st));
    double xc, yc;
    grid_centre(L, &xc, &yc);
    const double d = (double)L->dpix / L->sub;
    // a batch no larger than the grid (each CTA one vector) is decoded by the
    // likelihood kernel itself: one launch instead of two, which is most of
    // the gain for small batches (a sampler's few hundred walkers)
    const bool fused = !write && B <= L->shape.grid_cap && L->conv_variant == TLL_CONV_FUSED;
    if (ss && !fused) return fail(TLL_EINVAL, "a fused sampler step needs a batch within the grid");
    if (!fused) {
        k_prologue<<<(B + kPrologueVectors - 1) / kPrologueVectors, dim3(kPrologueVectors, 4),
                     0, st>>>(params, B, kc, xc, yc, d, L->bn_tab, L->epl);
        CUDA_TRY(cudaGetLastError());
    }
    if (prof) CUDA_TRY(cudaEventRecord(L->prof_ev[1], st));
    RunArgs R = {};
    R.kc = kc; R.B = B; R.out = out; R.gscr = L->d_gscr; R.gslot = L->shape.gslot;
    R.wr_unblurred = L->d_unb; R.wr_blurred = L->d_blur; R.wr_res = L->d_res;
    R.fused = fused ? 1 : 0;
    R.epl = L->epl;
    R.np = L->epl ? NPAR_EPL : NPAR;
    R.params = params;
    R.XC = xc; R.YC = yc; R.d = d;
    R.bn_tab = L->bn_tab;
    if (ss) {
        R.smp = *ss;
        R.smp_on = 1;
    }
    const int grid = std::min(B, L->shape.grid_cap);
    if (write) return launch_main(L, R, 1, true, st);
    const int rc = L->conv_variant == TLL_CONV_FUSED ? launch_main(L, R, grid, false, st)
                                                     : run_split(L, kc, B, out, st);
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

// Shared memory kept free for the kernels' static part (the multi-lens
// kernel's copy of a lens descriptor, the EPL series' table), so every lens
// also fits that kernel.
constexpr int kSmemReserve = 12288;

// Let kernel k use all the dynamic shared memory the opt-in limit leaves
// beside its static part.
int allow_dynamic_smem(const void *k, int optin)
{
    cudaFuncAttributes fa;
    CUDA_TRY(cudaFuncGetAttributes(&fa, k));
    CUDA_TRY(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  optin - (int)fa.sharedSizeBytes));
    return TLL_OK;
}

struct DevLimits {
    int nsm = 0, optin = 0, per_sm_smem = 0, reserved = 0;
};

int dev_limits(int dev, DevLimits *D)
{
    CUDA_TRY(cudaDeviceGetAttribute(&D->nsm, cudaDevAttrMultiProcessorCount, dev));
    CUDA_TRY(cudaDeviceGetAttribute(&D->optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    CUDA_TRY(cudaDeviceGetAttribute(&D->per_sm_smem, cudaDevAttrMaxSharedMemoryPerMultiprocessor,
                                    dev));
    CUDA_TRY(cudaDeviceGetAttribute(&D->reserved, cudaDevAttrReservedSharedMemoryPerBlock, dev));
    return TLL_OK;
}

// The shape of running lens L with CTAs of `threads` threads, `per_sm` of
// them per SM: each CTA gets an equal share of the SM's shared memory (less
// the multi-lens kernel's static part).  Placement: for PSF side <= 31 and
// nx <= 256 the compiled convolutions, on the whole zero-padded image in
// shared memory if it fits, else band by band (bands of equal height) from
// a global slot; otherwise the generic convolution on unpadded shared
// memory or a global slot.  S->per_sm is the occupancy actually reached.
int make_shape(const tll_lens *L, const DevLimits &D, int threads, int per_sm, Shape *out)
{
    if (threads < 32 || threads > kThreads || threads % 32 || per_sm < 1)
        return fail(TLL_EINVAL, "bad launch shape %d x %d", threads, per_sm);
    Shape S;
    S.threads = threads;
    const long long share =
        std::min<long long>(D.optin, D.per_sm_smem / per_sm - D.reserved);
    const long long avail = share - kSmemReserve;
    const int h = (L->K - 1) / 2;
    S.img = -1;
    if (L->K <= kMaxK && L->nx <= 256) {
        const size_t row_bytes = (size_t)2 * L->W * sizeof(float);
        const size_t whole = kRedBytes + (size_t)(L->ny + 2 * h + kCR) * row_bytes;
        const long long br = (avail - kRedBytes) / (long long)row_bytes - 2 * h - kCR;
        if ((long long)whole <= avail) {
            S.img = IMG_PADDED;
            S.smem = whole;
        } else if (br >= 8) {
            const long long nb = (L->ny + br - 1) / br;
            S.img = IMG_BANDED;
            S.band_rows = (int)((L->ny + nb - 1) / nb);
            S.smem = kRedBytes + (size_t)(S.band_rows + 2 * h + kCR) * row_bytes;
            S.gslot = 2LL * L->npix;
        }
    }
    if (S.img < 0) {
        const int psf_floats = L->sep ? 2 * L->K : L->K * L->K;
        const size_t fixed = kRedBytes + (size_t)((psf_floats + 3) & ~3) * sizeof(float);
        const size_t plain = fixed + (size_t)2 * L->npix * sizeof(float);
        if ((long long)plain <= avail && L->nx <= 32 * kHMax) {
            S.img = IMG_SMEM;
            S.smem = plain;
        } else if ((long long)fixed <= avail) {
            S.img = IMG_GLOBAL;
            S.smem = fixed;
            S.gslot = 4LL * L->npix;
        } else {
            return fail(TLL_EINVAL, "no placement for %d CTAs per SM", per_sm);
        }
    }
    const SingleKernel k = find_single(L->sub, conv_class(S.img, L->K), false);
    if (!k) return fail(TLL_ECUDA, "no kernel for s=%d K=%d", L->sub, L->K);
    if (int rc = allow_dynamic_smem((const void *)k, D.optin)) return rc;
    int n = 0;
    CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k, threads, S.smem));
    if (n < 1) return fail(TLL_EINVAL, "k_loglike cannot be resident at %d threads", threads);
    S.per_sm = n;
    S.grid_cap = D.nsm * n;
    *out = S;
    return TLL_OK;
}

// Tuned shapes by lens signature (device, nx, ny, s, K, separable): lenses
// created later with a tuned signature start with its shape.
struct TuneKey {
    int dev, nx, ny, sub, K, sep;
    bool operator<(const TuneKey &o) const
    {
        return std::tie(dev, nx, ny, sub, K, sep) < std::tie(o.dev, o.nx, o.ny, o.sub, o.K, o.sep);
    }
};
std::map<TuneKey, std::pair<int, int>> g_tuned;   // -> (threads, CTAs per SM asked)
std::mutex g_tune_mu;

TuneKey tune_key(const tll_lens *L) { return TuneKey{L->dev, L->nx, L->ny, L->sub, L->K, L->sep}; }

int configure(tll_lens *L)
{
    DevLimits D;
    int rc = dev_limits(L->dev, &D);
    if (rc) return rc;
    L->W = padded_stride(L->nx, L->K);
    L->HL = (((L->K - 1) / 2) + 3) & ~3;
    {   // the write-out (model image) launches: generic placement, one CTA
        const int psf_floats = L->sep ? 2 * L->K : L->K * L->K;
        const size_t fixed = kRedBytes + (size_t)((psf_floats + 3) & ~3) * sizeof(float);
        const size_t plain = fixed + (size_t)2 * L->npix * sizeof(float);
        const size_t avail = (size_t)D.optin - kSmemReserve;
        if (plain <= avail && L->nx <= 32 * kHMax) {
            L->img_write = IMG_SMEM;
            L->smem_write = plain;
        } else {
            L->img_write = IMG_GLOBAL;
            L->smem_write = fixed;
        }
        const SingleKernel kw = find_single(L->sub, 0, true);
        if (!kw) return fail(TLL_ECUDA, "no kernel for s=%d", L->sub);
        if (int rc = allow_dynamic_smem((const void *)kw, D.optin)) return rc;
    }
    int threads = kThreads, per_sm = 1;
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        auto it = g_tuned.find(tune_key(L));
        if (it != g_tuned.end()) {
            threads = it->second.first;
            per_sm = it->second.second;
            L->tuned = true;
        }
    }
    rc = make_shape(L, D, threads, per_sm, &L->shape);
    if (rc && L->tuned) {
        L->tuned = false;
        rc = make_shape(L, D, kThreads, 1, &L->shape);
    }
    return rc;
}

long long gscr_need(const tll_lens *L)
{
    long long n = (long long)L->shape.grid_cap * L->shape.gslot;
    if (L->img_write == IMG_GLOBAL) n = std::max(n, 4LL * L->npix);
    return n;
}

// The one-lens kernel's per-CTA global image slots (shapes that keep the
// images in global memory, and the generic write-out).  Allocated at
// creation, except for lenses created TLL_FLAG_BATCH_ONLY (evaluated
// through a batcher, which has its own slots); for those the allocating
// one-lens entry points allocate on first use.  Grows (never shrinks
// here) when the shape changes.
int ensure_gscr(tll_lens *L)
{
    const long long need = gscr_need(L);
    if (need <= L->gscr_floats) return TLL_OK;
    if (L->d_gscr) {
        CUDA_TRY(cudaDeviceSynchronize());
        cudaFree(L->d_gscr);
        L->d_gscr = nullptr;
        L->dev_bytes -= (size_t)L->gscr_floats * sizeof(float);
        L->gscr_floats = 0;
    }
    CUDA_TRY(cudaMalloc(&L->d_gscr, (size_t)need * sizeof(float)));
    L->gscr_floats = need;
    L->dev_bytes += (size_t)need * sizeof(float);
    return TLL_OK;
}

void free_lens(tll_lens *L)
{
    if (!L) return;
    void *ptrs[] = {L->d_psf, L->d_pu, L->d_pv, L->d_wpack, L->d_kc, L->d_gscr,
                    L->d_stage_p, L->d_stage_o, L->d_p1, L->d_kc1, L->d_unb,
                    L->d_blur, L->d_img, L->d_res, L->d_out1, L->d_unbl, L->d_sblur,
                    L->d_tiles, L->d_tc_status, L->d_thi, L->d_tlo, L->d_nscr, L->d_nres,
                    L->d_tlist, L->d_bpart[0], L->d_bpart[1], L->d_bpart[2], L->d_btiles};
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
    {
        const int rc = ensure_gscr(L);
        if (rc) return rc;
    }
    CUDA_TRY(cudaMemcpy(L->d_p1, params_host, L->nparam * sizeof(float), cudaMemcpyHostToDevice));
    int rc = run_batch(L, L->d_p1, 1, L->d_out1, 0, true, L->d_kc1);
    if (rc) return rc;
    CUDA_TRY(cudaDeviceSynchronize());
    float valid = 0.0f;
    CUDA_TRY(cudaMemcpy(&valid, L->d_kc1 + K_VALID, sizeof(float), cudaMemcpyDeviceToHost));
    if (valid == 0.0f) return fail(TLL_EINVAL, "invalid parameter vector");
    return TLL_OK;
}

// ------------------------------------------------- multi-column lenses
// Shape of the multi-column kernel: 1024-thread CTAs, one per SM.  For PSF
// side <= 31 and nx <= 256 the compiled band convolution, with the tallest
// equal bands the shared memory allows (the whole image when it fits);
// otherwise the generic convolution with the PSF taps in shared memory.
// Per-CTA global slot: U [nc], M [nc + 1] and H [2] images of npix floats.
int nc_configure(tll_lens *L)
{
    DevLimits D;
    if (int rc = dev_limits(L->dev, &D)) return rc;
    Shape S;
    S.threads = kThreads;
    const int h = (L->K - 1) / 2;
    const long long share = std::min<long long>(D.optin, D.per_sm_smem - D.reserved);
    NcKernel k = nullptr;
    if (L->K <= kMaxK && L->nx <= 256) {
        k = find_nc(L->sub, L->K);
        const MultiKernel km = find_nc_multi(L->sub, L->K);
        if (!k || !km) return fail(TLL_ECUDA, "no multi-column kernel for s=%d K=%d", L->sub, L->K);
        // the band must fit both the one-lens kernel and the batcher's
        // multi-lens one (their static shared memory differs)
        cudaFuncAttributes fa, fm;
        CUDA_TRY(cudaFuncGetAttributes(&fa, (const void *)k));
        CUDA_TRY(cudaFuncGetAttributes(&fm, (const void *)km));
        const long long avail =
            share - (long long)std::max(fa.sharedSizeBytes, fm.sharedSizeBytes);
        const size_t row_bytes = (size_t)2 * L->W * sizeof(float);
        const long long rows = avail / (long long)row_bytes - 2 * h - kCR;
        if (rows >= 8) {
            const long long nb = (L->ny + std::min<long long>(rows, L->ny) - 1) /
                                 std::min<long long>(rows, L->ny);
            S.img = IMG_BANDED;
            S.band_rows = (int)((L->ny + nb - 1) / nb);
            S.smem = (size_t)(S.band_rows + 2 * h + kCR) * row_bytes;
        } else {
            k = nullptr;
        }
    }
    if (!k) {
        k = find_nc(L->sub, 0);
        if (!k) return fail(TLL_ECUDA, "no multi-column kernel for s=%d", L->sub);
        S.img = IMG_GLOBAL;
        S.band_rows = 0;
        const int psf_floats = L->sep ? 2 * L->K : L->K * L->K;
        S.smem = (size_t)((psf_floats + 3) & ~3) * sizeof(float);
    }
    // the normal equations' pixel tiles reuse the dynamic shared memory:
    // at least 256 pixels of every column per tile, and room for one FP64
    // partial per thread after the last tile
    {
        cudaFuncAttributes fa;
        CUDA_TRY(cudaFuncGetAttributes(&fa, (const void *)k));
        const size_t tile = std::max((size_t)nc_tile_bytes(L->nc, 256) + 64,
                                     (size_t)kThreads * sizeof(double));
        const size_t cap = (size_t)(share - (long long)fa.sharedSizeBytes);
        S.smem = std::max(S.smem, std::min(tile, cap));
    }
    // the kernel is shared by every lens of its (s, K) class: allow the
    // most any of them can ask for, never less
    if (int rc = allow_dynamic_smem((const void *)k, D.optin)) return rc;
    int n = 0;
    CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k, S.threads, S.smem));
    if (n < 1) return fail(TLL_EINVAL, "multi-column kernel cannot be resident");
    S.per_sm = 1;
    S.grid_cap = D.nsm;
    S.gslot = (2LL * L->nc + 3) * L->npix;
    L->nc_shape = S;
    return TLL_OK;
}

int nc_ensure_scr(tll_lens *L)
{
    const long long need = (long long)L->nc_shape.grid_cap * L->nc_shape.gslot;
    if (need <= L->nscr_floats) return TLL_OK;
    if (L->d_nscr) {
        CUDA_TRY(cudaDeviceSynchronize());
        cudaFree(L->d_nscr);
        L->dev_bytes -= (size_t)L->nscr_floats * sizeof(float);
        L->d_nscr = nullptr;
        L->nscr_floats = 0;
    }
    CUDA_TRY(cudaMalloc(&L->d_nscr, (size_t)need * sizeof(float)));
    L->nscr_floats = need;
    L->dev_bytes += (size_t)need * sizeof(float);
    return TLL_OK;
}

// Prologue and multi-column kernel for B vectors; wres != null: one CTA,
// amplitudes and log L of vector 0 to wres, its columns stay in slot 0.
int run_batch_nc(tll_lens *L, const float *params, int B, double *out, cudaStream_t st,
                 float *kc, double *wres)
{
    const bool prof = L->prof_on && !wres;
    if (prof) CUDA_TRY(cudaEventRecord(L->prof_ev[0], st));
    LensDev d = lens_dev(L);
    d.img = L->nc_shape.img;
    d.band_rows = L->nc_shape.band_rows;
    d.nc_smem = (int)L->nc_shape.smem;
    k_prologue_nc<<<(B + 127) / 128, 128, 0, st>>>(params, B, kc, d, L->md, L->bn_tab);
    CUDA_TRY(cudaGetLastError());
    if (prof) CUDA_TRY(cudaEventRecord(L->prof_ev[1], st));
    const NcKernel k = find_nc(L->sub, d.img == IMG_BANDED ? L->K : 0);
    if (!k) return fail(TLL_ECUDA, "no multi-column kernel for s=%d K=%d", L->sub, L->K);
    NcArgs R;
    R.kc = kc; R.B = B; R.out = out; R.gscr = L->d_nscr; R.gslot = L->nc_shape.gslot;
    R.wr_res = wres;
    const int grid = wres ? 1 : std::min(B, L->nc_shape.grid_cap);
    k<<<grid, L->nc_shape.threads, L->nc_shape.smem, st>>>(d, L->md, R);
    CUDA_TRY(cudaGetLastError());
    if (prof) {
        CUDA_TRY(cudaEventRecord(L->prof_ev[2], st));
        L->prof_recorded = true;
    }
    return TLL_OK;
}

// One multi-column vector with its columns and amplitudes kept (model
// image entry points); synchronous.
int run_one_nc(tll_lens *L, const float *params_host)
{
    if (!params_host) return fail(TLL_EINVAL, "params is NULL");
    if (int rc = nc_ensure_scr(L)) return rc;
    CUDA_TRY(cudaMemcpy(L->d_p1, params_host, L->nparam * sizeof(float), cudaMemcpyHostToDevice));
    int rc = run_batch_nc(L, L->d_p1, 1, L->d_out1, 0, L->d_kc1, L->d_nres);
    if (rc) return rc;
    CUDA_TRY(cudaDeviceSynchronize());
    float valid = 0.0f;
    CUDA_TRY(cudaMemcpy(&valid, L->d_kc1 + K_VALID, sizeof(float), cudaMemcpyDeviceToHost));
    if (valid == 0.0f) return fail(TLL_EINVAL, "invalid parameter vector");
    return TLL_OK;
}

int reject_nc(const tll_lens *L, const char *what)
{
    return L && L->nc ? fail(TLL_EINVAL, "%s: not available for multi-component lenses", what)
                      : TLL_OK;
}

}  // namespace

// ------------------------------------------- internal entry points
namespace tll {

int lens_prepare(tll_lens *L)
{
    DeviceGuard gd(L->dev);
    return L->nc ? nc_ensure_scr(L) : ensure_gscr(L);
}

int lens_eval(tll_lens *L, const float *params, int B, double *out, cudaStream_t st, float *kc)
{
    if (B <= 0) return TLL_OK;
    return L->nc ? run_batch_nc(L, params, B, out, st, kc, nullptr)
                 : run_batch(L, params, B, out, st, false, kc);
}

bool lens_eval_fuses(const tll_lens *L, int B)
{
    return !L->nc && B > 0 && B <= L->shape.grid_cap && L->conv_variant == TLL_CONV_FUSED;
}

int lens_eval_stretch(tll_lens *L, float *params, int B, double *out, cudaStream_t st,
                      float *kc, const StretchStep &ss)
{
    if (!lens_eval_fuses(L, B)) return fail(TLL_EINVAL, "no fused sampler step for this batch");
    return run_batch(L, params, B, out, st, false, kc, &ss);
}

int lens_nparam(const tll_lens *L) { return L->nparam; }
int lens_device(const tll_lens *L) { return L->dev; }
int const_block_floats() { return NCONST; }

int set_error(int code, const char *fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof g_err, fmt, ap);
    va_end(ap);
    return code;
}

}  // namespace tll

// ------------------------------------------------------- batch context
// Reusable buffers for multi-lens launches (and their CUDA graph).  The
// entries of a run are grouped by (supersampling class, convolution class,
// launch shape) and at most kMultiSlots lenses; each group is one launch of
// its k_loglike_multi<SUB, K> (two-column lenses) or k_loglike_nc_multi<SUB,
// K>, the lenses' descriptors in the launch's parameters (LensSlots).
constexpr int kMaxGroups = kMultiCounters;
constexpr int kCounterInts = kMultiCounters * (1 + kMultiSlots);

namespace {
// One group's launch: kernel, CTA size, grid and dynamic shared memory.
struct GroupLaunch {
    MultiKernel kern = nullptr;
    int threads = 0, grid = 0;
    size_t smem = 0;
    bool operator==(const GroupLaunch &o) const
    {
        return kern == o.kern && threads == o.threads && grid == o.grid && smem == o.smem;
    }
};
}  // namespace

struct tll_batcher {
    int dev = 0, nsm = 0, optin = 0, dyn_smem = 0;
    bool use_graph = false;
    int cap_lenses = 0, cap_segs = 0, cap_items = 0, cap_ctas = 0;
    long long gslot_floats = 0;
    LensDev *d_lenses = nullptr, *h_lenses = nullptr;   // h_*: pinned staging
    MultiDev *d_mdevs = nullptr, *h_mdevs = nullptr;   // per lens: component list
    Segment *d_segs = nullptr, *h_segs = nullptr;
    MultiHdr *d_groups = nullptr, *h_groups = nullptr; // [kMaxGroups] + the whole list
    float *d_kc = nullptr, *d_gscr = nullptr;
    int *d_counter = nullptr;   // [kMaxGroups] group counters, then kMultiSlots per group
    const double *bn_tab = nullptr;
    cudaEvent_t staged = nullptr;      // staging may be refilled after this
    bool staged_pending = false;
    std::vector<GroupLaunch> glaunch;  // this run's group launches
    std::vector<LensSlots> gslots;     // ... and their lens slots
    std::vector<MultiKernel> kern_ready;  // kernels whose shared-memory limit is set
    int dyn_smem_nc = 0;              // dynamic shared memory of the multi-column kernels
    cudaGraphExec_t gexec = nullptr;
    cudaStream_t gstream = nullptr;    // stream the graph was captured on
    std::vector<GroupLaunch> gcaptured;   // group launches baked into the graph
    long long launches = 0;
};

namespace {

void batcher_free_buffers(tll_batcher *b)
{
    void *dev[] = {b->d_lenses, b->d_segs, b->d_groups, b->d_kc, b->d_gscr, b->d_counter,
                   b->d_mdevs};
    for (void *p : dev)
        if (p) cudaFree(p);
    void *host[] = {b->h_lenses, b->h_segs, b->h_groups, b->h_mdevs};
    for (void *p : host)
        if (p) cudaFreeHost(p);
    b->d_lenses = b->h_lenses = nullptr;
    b->d_mdevs = b->h_mdevs = nullptr;
    b->d_segs = b->h_segs = nullptr;
    b->d_groups = b->h_groups = nullptr;
    b->d_kc = b->d_gscr = nullptr;
    b->d_counter = nullptr;
    if (b->gexec) {
        cudaGraphExecDestroy(b->gexec);
        b->gexec = nullptr;
    }
}

// Grow every buffer to hold (lenses, segs, items, gslot floats for each of
// ctas CTAs); the graph (which bakes in the buffer addresses and copy
// sizes) is dropped when anything grows.
int batcher_reserve(tll_batcher *b, int lenses, int segs, int items, long long gslot, int ctas)
{
    if (lenses <= b->cap_lenses && segs <= b->cap_segs && items <= b->cap_items &&
        gslot <= b->gslot_floats && (gslot == 0 || ctas <= b->cap_ctas) && b->d_kc)
        return TLL_OK;
    if (b->staged_pending) CUDA_TRY(cudaEventSynchronize(b->staged));
    CUDA_TRY(cudaDeviceSynchronize());
    const int cl = std::max(lenses, std::max(2 * b->cap_lenses, 16));
    const int cs = std::max(segs, std::max(2 * b->cap_segs, 64));
    const int ci = std::max(items, std::max(2 * b->cap_items, 4096));
    const long long cg = std::max(gslot, b->gslot_floats);
    const int cc = std::max(ctas, b->cap_ctas);
    batcher_free_buffers(b);
    CUDA_TRY(cudaMalloc(&b->d_lenses, cl * sizeof(LensDev)));
    CUDA_TRY(cudaMalloc(&b->d_mdevs, cl * sizeof(MultiDev)));
    CUDA_TRY(cudaMallocHost(&b->h_mdevs, cl * sizeof(MultiDev)));
    CUDA_TRY(cudaMalloc(&b->d_segs, cs * sizeof(Segment)));
    CUDA_TRY(cudaMalloc(&b->d_groups, (kMaxGroups + 1) * sizeof(MultiHdr)));
    CUDA_TRY(cudaMalloc(&b->d_kc, (size_t)ci * NCONST * sizeof(float)));
    CUDA_TRY(cudaMalloc(&b->d_counter, kCounterInts * sizeof(int)));
    if (cg > 0) CUDA_TRY(cudaMalloc(&b->d_gscr, (size_t)cc * cg * sizeof(float)));
    CUDA_TRY(cudaMallocHost(&b->h_lenses, cl * sizeof(LensDev)));
    CUDA_TRY(cudaMallocHost(&b->h_segs, cs * sizeof(Segment)));
    CUDA_TRY(cudaMallocHost(&b->h_groups, (kMaxGroups + 1) * sizeof(MultiHdr)));
    b->cap_lenses = cl;
    b->cap_segs = cs;
    b->cap_items = ci;
    b->gslot_floats = cg;
    b->cap_ctas = cc;
    return TLL_OK;
}

MultiArgs batcher_args(const tll_batcher *b)
{
    MultiArgs A;
    A.lenses = b->d_lenses;
    A.mdevs = b->d_mdevs;
    A.segs = b->d_segs;
    A.groups = b->d_groups;
    A.all = b->d_groups + kMaxGroups;
    A.kc = b->d_kc;
    A.gscr = b->d_gscr;
    A.gslot_floats = b->gslot_floats;
    A.counter = b->d_counter;
    A.bn_tab = b->bn_tab;
    return A;
}

// The launch sequence: stage descriptors, reset the counters, prologue,
// one multi-lens launch per group.  `full` copies whole staging buffers
// (graph form, fixed sizes); otherwise only what this run uses.
int batcher_enqueue(tll_batcher *b, int nl, int ns, int total, bool full, cudaStream_t st)
{
    const int cl = full ? b->cap_lenses : nl, cs = full ? b->cap_segs : ns;
    const int items = full ? b->cap_items : total;
    CUDA_TRY(cudaMemcpyAsync(b->d_lenses, b->h_lenses, cl * sizeof(LensDev),
                             cudaMemcpyHostToDevice, st));
    CUDA_TRY(cudaMemcpyAsync(b->d_mdevs, b->h_mdevs, cl * sizeof(MultiDev),
                             cudaMemcpyHostToDevice, st));
    CUDA_TRY(cudaMemcpyAsync(b->d_segs, b->h_segs, cs * sizeof(Segment),
                             cudaMemcpyHostToDevice, st));
    CUDA_TRY(cudaMemcpyAsync(b->d_groups, b->h_groups, (kMaxGroups + 1) * sizeof(MultiHdr),
                             cudaMemcpyHostToDevice, st));
    CUDA_TRY(cudaMemsetAsync(b->d_counter, 0, kCounterInts * sizeof(int), st));
    const MultiArgs A = batcher_args(b);
    k_prologue_multi<<<(items + kPrologueVectors - 1) / kPrologueVectors,
                       dim3(kPrologueVectors, 4), 0, st>>>(A);
    CUDA_TRY(cudaGetLastError());
    for (int g = 0; g < (int)b->glaunch.size(); ++g) {
        const GroupLaunch &gl = b->glaunch[g];
        gl.kern<<<gl.grid, gl.threads, gl.smem, st>>>(A, g, b->gslots[g]);
        CUDA_TRY(cudaGetLastError());
    }
    return TLL_OK;
}

}  // namespace

// ------------------------------------------- no-allocation entry point
// Scratch for tll_loglike_batch_noalloc: the per-vector constant blocks
// that tll_loglike_batch keeps in a lens-owned buffer it may grow.  A fixed
// array in this module instead, so the call itself allocates nothing.  The
// module's globals are placed on a device when the module is loaded there
// (lazily, at the first use of one of its kernels or symbols, by default
// since CUDA 12.2); tll_create_lens launches k_bn_table from this module,
// so every device with a lens holds the array (22 MB) from then until the
// process exits.
constexpr int kNoAllocMaxB = TLL_NOALLOC_MAX_B;
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
        // (a lens descriptor), the same for every multi-lens kernel
        cudaFuncAttributes fa;
        const MultiKernel k0 = find_multi(4, 0);
        if (!k0 || cudaFuncGetAttributes(&fa, k0) != cudaSuccess)
            return bad(fail(TLL_ECUDA, "k_loglike_multi attributes"));
        b->dyn_smem = b->optin - (int)fa.sharedSizeBytes;
        const MultiKernel k1 = find_nc_multi(4, 0);
        if (!k1 || cudaFuncGetAttributes(&fa, k1) != cudaSuccess)
            return bad(fail(TLL_ECUDA, "k_loglike_nc_multi attributes"));
        b->dyn_smem_nc = b->optin - (int)fa.sharedSizeBytes;
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
    // distinct lenses; entries ordered by group key, then cost (largest first)
    std::vector<tll_lens *> uniq;
    std::vector<int> lid(n), order;
    std::vector<long long> key(n);
    long long total = 0, gslot = 0;
    int ctas = 0;
    for (int k = 0; k < n; ++k) {
        tll_lens *L = lenses[k];
        if (!L) return fail(TLL_EINVAL, "lens %d is NULL", k);
        if (L->dev != b->dev) return fail(TLL_EINVAL, "lens %d is on another device", k);
        if (counts[k] < 0) return fail(TLL_EINVAL, "negative count for lens %d", k);
        if (counts[k] > 0 && (!params[k] || !outs[k]))
            return fail(TLL_EINVAL, "NULL params/out for lens %d", k);
        const Shape &S = L->nc ? L->nc_shape : L->shape;
        if (S.smem > (size_t)(L->nc ? b->dyn_smem_nc : b->dyn_smem))
            return fail(TLL_EINVAL, "lens %d needs more shared memory than the batch kernel has", k);
        int u = 0;
        while (u < (int)uniq.size() && uniq[u] != L) ++u;
        if (u == (int)uniq.size()) uniq.push_back(L);
        lid[k] = u;
        // group key: kind (two columns / multi-column), supersampling class,
        // convolution class, CTA size, CTAs per SM
        key[k] = ((((long long)(L->nc ? 1 : 0) * 8 + sub_class(L->sub)) * 1000 +
                   conv_class(S.img, L->K)) * 2048 + S.threads) * 64 + std::min(S.per_sm, 63);
        if (counts[k] > 0) {
            order.push_back(k);
            if (S.gslot > 0) {
                gslot = std::max(gslot, S.gslot);
                ctas = std::max(ctas, b->nsm * S.per_sm);
            }
        }
        total += counts[k];
    }
    if (total == 0) return TLL_OK;
    if (total > (1LL << 30)) return fail(TLL_EINVAL, "batch too large");
    // per-vector cost estimate (subpixels) orders a group's lenses (largest
    // first) and splits its CTAs among lens slots; ties by lens, so that a
    // lens's segments are adjacent
    auto cost = [&](int k) {
        return (long long)lenses[k]->npix * lenses[k]->sub * lenses[k]->sub;
    };
    std::stable_sort(order.begin(), order.end(), [&](int a, int c) {
        if (key[a] != key[c]) return key[a] < key[c];
        if (cost(a) != cost(c)) return cost(a) > cost(c);
        return lid[a] < lid[c];
    });
    int rc = batcher_reserve(b, (int)uniq.size(), n, (int)total, gslot, ctas);
    if (rc) return rc;
    if (b->staged_pending) CUDA_TRY(cudaEventSynchronize(b->staged));
    for (size_t u = 0; u < uniq.size(); ++u) {
        b->h_lenses[u] = lens_dev(uniq[u]);
        b->h_mdevs[u] = uniq[u]->md;
        if (!uniq[u]->nc) b->h_mdevs[u].nc = 0;
    }
    b->glaunch.clear();
    b->gslots.clear();
    int first = 0, ns = 0, ng = 0;
    for (size_t q = 0; q < order.size(); ++q) {
        const int k = order[q];
        const bool ncl = lenses[k]->nc > 0;
        const Shape &S = ncl ? lenses[k]->nc_shape : lenses[k]->shape;
        // a new group at a new key, or at a (kMultiSlots + 1)-th lens
        bool fresh = q == 0 || key[k] != key[order[q - 1]];
        if (!fresh) {
            const LensSlots &ls = b->gslots.back();
            fresh = lid[k] != lid[order[q - 1]] && ls.n == kMultiSlots;
        }
        if (fresh) {
            if (ng == kMaxGroups) return fail(TLL_EINVAL, "more than %d kernel groups", kMaxGroups);
            const int Kc = conv_class(S.img, lenses[k]->K);
            const MultiKernel mk = ncl ? find_nc_multi(lenses[k]->sub, Kc)
                                       : find_multi(lenses[k]->sub, Kc);
            if (!mk) return fail(TLL_ECUDA, "no multi-lens kernel for s=%d K=%d", lenses[k]->sub,
                                 Kc);
            if (std::find(b->kern_ready.begin(), b->kern_ready.end(), mk) == b->kern_ready.end()) {
                CUDA_TRY(cudaFuncSetAttribute(mk, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                              ncl ? b->dyn_smem_nc : b->dyn_smem));
                b->kern_ready.push_back(mk);
            }
            GroupLaunch gl;
            gl.kern = mk;
            gl.threads = S.threads;
            gl.grid = b->nsm * S.per_sm;
            b->glaunch.push_back(gl);
            b->gslots.emplace_back();
            b->gslots.back().n = 0;
            b->h_groups[ng] = MultiHdr{first, 0, ns, 0};
            ++ng;
        }
        b->glaunch.back().smem = std::max(b->glaunch.back().smem, S.smem);
        {
            // the lens's slot in the group: a new one, or the previous
            // segment's (a lens's segments are adjacent)
            LensSlots &ls = b->gslots.back();
            if (ls.n == 0 || lid[k] != lid[order[q - 1]]) {
                ls.lens[ls.n] = b->h_lenses[lid[k]];
                ls.md[ls.n] = b->h_mdevs[lid[k]];
                ls.first[ls.n] = first;
                ls.count[ls.n] = 0;
                ls.cta_end[ls.n] = 0;
                ++ls.n;
            }
            ls.count[ls.n - 1] += counts[k];
        }
        Segment &sg = b->h_segs[ns++];
        sg.lens = lid[k];
        sg.first = first;
        sg.count = counts[k];
        sg.pad = 0;
        sg.params = params[k];
        sg.out = outs[k];
        first += counts[k];
        b->h_groups[ng - 1].total += counts[k];
        b->h_groups[ng - 1].nseg += 1;
    }
    b->h_groups[kMaxGroups] = MultiHdr{0, (int)total, 0, ns};
    // each group's CTAs split among its lens slots in proportion to their
    // cost (vectors x subpixels x columns), at least one each
    for (int g = 0; g < ng; ++g) {
        LensSlots &ls = b->gslots[g];
        if (ls.n == 0) continue;
        const int grid = b->glaunch[g].grid;
        double w[kMultiSlots], wsum = 0.0;
        for (int s2 = 0; s2 < ls.n; ++s2) {
            w[s2] = (double)ls.count[s2] * (double)ls.lens[s2].npix * ls.lens[s2].sub *
                    ls.lens[s2].sub * (ls.md[s2].nc > 0 ? ls.md[s2].nc : 2);
            wsum += w[s2];
        }
        int end = 0;
        for (int s2 = 0; s2 < ls.n; ++s2) {
            const int left = ls.n - 1 - s2;   // slots after this one keep >= 1 CTA each
            int c = (int)((double)grid * w[s2] / std::max(wsum, 1.0));
            c = std::max(1, std::min(c, grid - end - left));
            end = s2 + 1 == ls.n ? grid : end + c;
            ls.cta_end[s2] = end;
        }
    }
    const bool graph = b->use_graph && st != nullptr;
    if (graph) {
        // the lens slots are launch parameters: captured anew every run and
        // the instantiated graph updated in place (same topology while the
        // group launches are the same), instantiated again otherwise
        cudaGraph_t g = nullptr;
        CUDA_TRY(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
        rc = batcher_enqueue(b, 0, 0, 0, true, st);
        const cudaError_t ce = cudaStreamEndCapture(st, &g);
        if (rc) {
            if (g) cudaGraphDestroy(g);
            return rc;
        }
        if (ce != cudaSuccess) return fail(TLL_ECUDA, "graph capture: %s", cudaGetErrorString(ce));
        bool updated = false;
        if (b->gexec && b->gstream == st && b->gcaptured == b->glaunch) {
            cudaGraphExecUpdateResultInfo info;
            updated = cudaGraphExecUpdate(b->gexec, g, &info) == cudaSuccess;
            if (!updated) cudaGetLastError();
        }
        if (!updated) {
            if (b->gexec) {
                cudaGraphExecDestroy(b->gexec);
                b->gexec = nullptr;
            }
            const cudaError_t ie = cudaGraphInstantiate(&b->gexec, g, 0);
            if (ie != cudaSuccess) {
                cudaGraphDestroy(g);
                return fail(TLL_ECUDA, "graph instantiate: %s", cudaGetErrorString(ie));
            }
        }
        cudaGraphDestroy(g);
        b->gstream = st;
        b->gcaptured = b->glaunch;
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
    if (!L->nc && L->gscr_floats < gscr_need(L))
        return fail(TLL_EINVAL, "lens was created TLL_FLAG_BATCH_ONLY and has no one-lens "
                                "image slots; evaluate it with tll_loglike_batch once first");
    DeviceGuard gd(L->dev);
    float *kc = nullptr;
    const int rc = noalloc_scratch(L->dev, &kc);
    if (rc) return rc;
    // a multi-component lens's image slots come from tll_set_light (or a
    // first allocating one-lens call for a TLL_FLAG_BATCH_ONLY lens)
    if (L->nc) {
        if (L->nscr_floats < (long long)L->nc_shape.grid_cap * L->nc_shape.gslot)
            return fail(TLL_EINVAL, "lens was created TLL_FLAG_BATCH_ONLY and has no one-lens "
                                    "image slots; evaluate it with tll_loglike_batch once first");
        return run_batch_nc(L, params, B, out, (cudaStream_t)stream, kc, nullptr);
    }
    // k_prologue writes all NCONST entries of each of the B blocks before
    // k_loglike reads them on the same stream, so nothing needs clearing.
    return run_batch(L, params, B, out, (cudaStream_t)stream, false, kc);
}


static_assert((int)TLL_PLACE_GLOBAL == (int)IMG_GLOBAL && (int)TLL_PLACE_SMEM == (int)IMG_SMEM &&
                  (int)TLL_PLACE_PADDED == (int)IMG_PADDED &&
                  (int)TLL_PLACE_BANDED == (int)IMG_BANDED,
              "placement codes");

namespace {
void shape_out(const Shape &S, tll_shape_t *o)
{
    o->threads = S.threads;
    o->ctas_per_sm = S.per_sm;
    o->placement = S.img;
    o->band_rows = S.band_rows;
    o->smem_bytes = S.smem;
    o->ms = S.ms;
    o->tuned = 0;
}

// Parameter vectors for timing when the caller gives none: a fixed set
// spanning both SIE forms (q near 1 and q well below it), both Sersic
// extremes of the usual prior, and sources inside and outside the caustic.
void default_tuning_vectors(int B, int nparam, std::vector<float> &p)
{
    p.assign((size_t)B * nparam, 0.0f);
    for (int b = 0; b < B; ++b) {
        float *v = &p[(size_t)b * nparam];
        if (nparam > NPAR) v[21] = (b & 1) ? 1.8f : 2.2f;   // EPL slope
        const int k = b % 8;
        v[0] = 0.7f + 0.1f * (float)k;              // theta_E
        v[1] = (k & 1) ? 0.25f : 0.04f;             // e1 (q = 0.6 or 0.92)
        v[2] = 0.02f;
        v[3] = 0.01f; v[4] = -0.02f;                // centre
        v[5] = 0.03f; v[6] = -0.02f;                // shear
        v[7] = 1.0f; v[8] = 0.6f; v[9] = (k & 2) ? 4.0f : 1.0f;
        v[10] = 0.1f; v[11] = -0.05f;
        v[12] = v[3]; v[13] = v[4];
        v[14] = 1.0f; v[15] = 0.25f; v[16] = (k & 4) ? 3.0f : 1.2f;
        v[17] = -0.1f; v[18] = 0.08f;
        v[19] = (k & 1) ? 0.05f : 0.2f; v[20] = -0.03f;
    }
}
}  // namespace

extern "C" int tll_lens_shape(const tll_lens *L, tll_shape_t *out)
{
    if (!L || !out) return fail(TLL_EINVAL, "NULL argument");
    shape_out(L->nc ? L->nc_shape : L->shape, out);
    out->tuned = L->tuned && !L->nc ? 1 : 0;
    return TLL_OK;
}

extern "C" int tll_set_conv(tll_lens *L, int variant, int chunk)
{
    if (!L) return fail(TLL_EINVAL, "lens is NULL");
    if (variant != TLL_CONV_FUSED && variant != TLL_CONV_SPLIT_DIRECT &&
        variant != TLL_CONV_SPLIT_TOEPLITZ_TC && variant != TLL_CONV_SPLIT_TOEPLITZ_BF16)
        return fail(TLL_EINVAL, "unknown convolution variant %d", variant);
    if (chunk < 0 || chunk > (1 << 20)) return fail(TLL_EINVAL, "chunk %d out of range", chunk);
    if (int rc = reject_nc(L, "tll_set_conv")) return rc;
    DeviceGuard gd(L->dev);
    CUDA_TRY(cudaDeviceSynchronize());   // no launch using the old buffers in flight
    if (variant == TLL_CONV_FUSED) {
        L->conv_variant = variant;
        return TLL_OK;
    }
    DevLimits D;
    int rc = dev_limits(L->dev, &D);
    if (rc) return rc;
    const LensDev d = lens_dev(L);
    if (variant == TLL_CONV_SPLIT_DIRECT && conv_direct_split_smem(d) > (size_t)D.optin)
        return fail(TLL_EINVAL, "padded %d x %d image does not fit shared memory", L->ny, L->nx);
    const bool toeplitz = variant == TLL_CONV_SPLIT_TOEPLITZ_TC ||
                          variant == TLL_CONV_SPLIT_TOEPLITZ_BF16;
    if (toeplitz && L->K > kTcMaxK)
        return fail(TLL_EINVAL, "Toeplitz tiles hold PSF sides up to %d", kTcMaxK);
    const int cap = chunk > 0 ? chunk : 1024;
    const bool regrow = cap != L->split_cap || !L->d_unbl;
    if (regrow) {
        const size_t bytes = (size_t)cap * 2 * L->npix * sizeof(float);
        float *u = nullptr, *b = nullptr;
        cudaError_t e = cudaMalloc(&u, bytes);
        if (e == cudaSuccess) e = cudaMalloc(&b, bytes);
        if (e != cudaSuccess) {
            if (u) cudaFree(u);
            return fail(TLL_ENOMEM, "split image buffers (%zu bytes): %s", 2 * bytes,
                        cudaGetErrorString(e));
        }
        if (L->d_unbl) {
            cudaFree(L->d_unbl);
            cudaFree(L->d_sblur);
            L->dev_bytes -= (size_t)L->split_cap * 2 * L->npix * sizeof(float) * 2;
        }
        L->d_unbl = u;
        L->d_sblur = b;
        L->split_cap = cap;
        L->dev_bytes += 2 * bytes;
    }
    if (variant == TLL_CONV_SPLIT_TOEPLITZ_TC && (regrow || !L->d_thi)) {
        const size_t pf = tc_part_floats(2 * cap, L->ny, L->nx);
        if (L->d_thi) {
            cudaFree(L->d_thi);
            cudaFree(L->d_tlo);
            L->d_thi = L->d_tlo = nullptr;
            L->dev_bytes -= L->tc_part_bytes * 2;
            L->tc_part_bytes = 0;
        }
        CUDA_TRY(cudaMalloc(&L->d_thi, pf * sizeof(float)));
        CUDA_TRY(cudaMalloc(&L->d_tlo, pf * sizeof(float)));
        L->tc_part_bytes = pf * sizeof(float);
        L->dev_bytes += 2 * L->tc_part_bytes;
        if (make_tc_maps(L->d_thi, L->d_tlo, 2 * cap, L->ny, L->nx, L->K, &L->tm_hi, &L->tm_lo))
            return fail(TLL_ECUDA, "cuTensorMapEncodeTiled failed for the Toeplitz operands");
    }
    if (variant == TLL_CONV_SPLIT_TOEPLITZ_TC && !L->d_tiles) {
        std::vector<float> t(tc_tile_floats(L->K));
        build_tc_tiles(L->psf_norm.data(), L->K, t.data());
        CUDA_TRY(cudaMalloc(&L->d_tiles, t.size() * sizeof(float)));
        L->dev_bytes += t.size() * sizeof(float);
        CUDA_TRY(cudaMemcpy(L->d_tiles, t.data(), t.size() * sizeof(float),
                            cudaMemcpyHostToDevice));
    }
    if (variant == TLL_CONV_SPLIT_TOEPLITZ_BF16 && (regrow || !L->d_bpart[0])) {
        const size_t pb = bf_part_bytes(2 * cap, L->ny, L->nx);
        for (int q = 0; q < 3; ++q)
            if (L->d_bpart[q]) {
                cudaFree(L->d_bpart[q]);
                L->d_bpart[q] = nullptr;
                L->dev_bytes -= L->bf_part_bytes_each;
            }
        L->bf_part_bytes_each = 0;
        for (int q = 0; q < 3; ++q) {
            CUDA_TRY(cudaMalloc(&L->d_bpart[q], pb));
            L->dev_bytes += pb;
        }
        L->bf_part_bytes_each = pb;
        if (make_bf_maps(L->d_bpart, 2 * cap, L->ny, L->nx, L->K, L->tm_b))
            return fail(TLL_ECUDA, "cuTensorMapEncodeTiled failed for the BF16 Toeplitz operands");
    }
    if (variant == TLL_CONV_SPLIT_TOEPLITZ_BF16 && !L->d_btiles) {
        std::vector<uint16_t> t(bf_tile_elems(L->K));
        build_bf_tiles(L->psf_norm.data(), L->K, t.data());
        CUDA_TRY(cudaMalloc(&L->d_btiles, t.size() * sizeof(uint16_t)));
        L->dev_bytes += t.size() * sizeof(uint16_t);
        CUDA_TRY(cudaMemcpy(L->d_btiles, t.data(), t.size() * sizeof(uint16_t),
                            cudaMemcpyHostToDevice));
    }
    if (toeplitz && !L->d_tc_status) {
        CUDA_TRY(cudaMalloc(&L->d_tc_status, sizeof(int)));
        L->dev_bytes += sizeof(int);
        CUDA_TRY(cudaMemset(L->d_tc_status, 0, sizeof(int)));
    }
    L->conv_variant = variant;
    return TLL_OK;
}

extern "C" int tll_conv_check(tll_lens *L)
{
    if (!L) return fail(TLL_EINVAL, "lens is NULL");
    if (!L->d_tc_status) return TLL_OK;
    DeviceGuard gd(L->dev);
    CUDA_TRY(cudaDeviceSynchronize());
    int st = 0;
    CUDA_TRY(cudaMemcpy(&st, L->d_tc_status, sizeof(int), cudaMemcpyDeviceToHost));
    if (st == 0) return TLL_OK;
    CUDA_TRY(cudaMemset(L->d_tc_status, 0, sizeof(int)));
    return fail(TLL_ETIMEOUT, "tensor-core convolution: a bounded wait ran out (status %d); "
                              "its outputs are not valid", st);
}

extern "C" int tll_set_shape(tll_lens *L, int threads, int ctas_per_sm)
{
    if (!L) return fail(TLL_EINVAL, "lens is NULL");
    if (int rc = reject_nc(L, "tll_set_shape")) return rc;
    DeviceGuard gd(L->dev);
    DevLimits D;
    int rc = dev_limits(L->dev, &D);
    if (rc) return rc;
    Shape S;
    if ((rc = make_shape(L, D, threads, ctas_per_sm, &S))) return rc;
    CUDA_TRY(cudaDeviceSynchronize());   // no launch of the old shape in flight
    const Shape keep = L->shape;
    L->shape = S;
    if (!(L->flags & TLL_FLAG_BATCH_ONLY) && (rc = ensure_gscr(L))) {
        L->shape = keep;
        return rc;
    }
    return TLL_OK;
}

extern "C" int tll_autotune(tll_lens *L, const float *params, int B, void *stream,
                            tll_shape_t *chosen, tll_shape_t *tried, int max_tried,
                            int *n_tried)
{
    if (!L) return fail(TLL_EINVAL, "lens is NULL");
    if (B < 0 || (B > 0 && !params)) return fail(TLL_EINVAL, "bad tuning batch");
    if (max_tried < 0 || (max_tried > 0 && !tried)) return fail(TLL_EINVAL, "bad tried array");
    if (int rc = reject_nc(L, "tll_autotune")) return rc;
    DeviceGuard gd(L->dev);
    cudaStream_t st = (cudaStream_t)stream;
    DevLimits D;
    int rc = dev_limits(L->dev, &D);
    if (rc) return rc;
    // candidates: 1024 threads resident per SM as 1 x 1024, 2 x 512, 4 x 256
    static const int kCand[][2] = {{1024, 1}, {512, 2}, {256, 4}};
    std::vector<Shape> cand;
    std::vector<int> ask;   // CTAs per SM each candidate was made for
    for (const auto &c : kCand) {
        Shape S;
        if (make_shape(L, D, c[0], c[1], &S) == TLL_OK) {
            cand.push_back(S);
            ask.push_back(c[1]);
        }
    }
    g_err[0] = 0;
    if (cand.empty()) return fail(TLL_ECUDA, "no launch shape fits this lens");
    int grid_max = 0;
    for (const Shape &S : cand) grid_max = std::max(grid_max, S.grid_cap);
    // tuning batch: at least two vectors per CTA of the largest grid; the
    // caller's vectors repeated, or the default set
    const int Bt = std::max(B, 2 * grid_max);
    float *d_p = nullptr;
    double *d_o = nullptr;
    cudaEvent_t ev[2] = {nullptr, nullptr};
    auto cleanup = [&]() {
        if (d_p) cudaFree(d_p);
        if (d_o) cudaFree(d_o);
        for (cudaEvent_t e : ev)
            if (e) cudaEventDestroy(e);
    };
    auto bail = [&](int code) { cleanup(); return code; };
    if (cudaMalloc(&d_p, (size_t)Bt * L->nparam * sizeof(float)) != cudaSuccess ||
        cudaMalloc(&d_o, (size_t)Bt * sizeof(double)) != cudaSuccess)
        return bail(fail(TLL_ENOMEM, "tuning buffers"));
    if (B > 0) {
        for (int off = 0; off < Bt; off += B) {
            const int n = std::min(B, Bt - off);
            if (cudaMemcpyAsync(d_p + (size_t)off * L->nparam, params,
                                (size_t)n * L->nparam * sizeof(float),
                                cudaMemcpyDeviceToDevice, st) != cudaSuccess)
                return bail(fail(TLL_ECUDA, "tuning batch copy"));
        }
    } else {
        std::vector<float> hp;
        default_tuning_vectors(Bt, L->nparam, hp);
        if (cudaMemcpyAsync(d_p, hp.data(), hp.size() * sizeof(float), cudaMemcpyHostToDevice,
                            st) != cudaSuccess ||
            cudaStreamSynchronize(st) != cudaSuccess)
            return bail(fail(TLL_ECUDA, "tuning batch copy"));
    }
    if (cudaEventCreate(&ev[0]) != cudaSuccess || cudaEventCreate(&ev[1]) != cudaSuccess)
        return bail(fail(TLL_ECUDA, "cudaEventCreate"));
    if ((rc = ensure_kc(L, Bt))) return bail(rc);
    const Shape keep = L->shape;
    int best = -1;
    for (size_t c = 0; c < cand.size(); ++c) {
        L->shape = cand[c];
        if ((rc = ensure_gscr(L))) break;
        // one warm-up launch, then three timed
        if ((rc = run_batch(L, d_p, Bt, d_o, st, false, L->d_kc))) break;
        if (cudaEventRecord(ev[0], st) != cudaSuccess) { rc = fail(TLL_ECUDA, "event"); break; }
        for (int r = 0; r < 3 && !rc; ++r) rc = run_batch(L, d_p, Bt, d_o, st, false, L->d_kc);
        if (rc) break;
        float ms = 0.0f;
        if (cudaEventRecord(ev[1], st) != cudaSuccess || cudaEventSynchronize(ev[1]) != cudaSuccess ||
            cudaEventElapsedTime(&ms, ev[0], ev[1]) != cudaSuccess) {
            rc = fail(TLL_ECUDA, "tuning launch: %s", cudaGetErrorString(cudaGetLastError()));
            break;
        }
        cand[c].ms = ms / 3.0f;
        if (best < 0 || cand[c].ms < cand[best].ms) best = (int)c;
    }
    if (rc) {
        L->shape = keep;
        return bail(rc);
    }
    L->shape = cand[best];
    L->tuned = true;
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        g_tuned[tune_key(L)] = {cand[best].threads, ask[best]};
    }
    // keep the slots the chosen shape needs, no more
    if (L->d_gscr && L->gscr_floats > gscr_need(L)) {
        if (cudaStreamSynchronize(st) != cudaSuccess) return bail(fail(TLL_ECUDA, "sync"));
        cudaFree(L->d_gscr);
        L->d_gscr = nullptr;
        L->dev_bytes -= (size_t)L->gscr_floats * sizeof(float);
        L->gscr_floats = 0;
        if (!(L->flags & TLL_FLAG_BATCH_ONLY) && (rc = ensure_gscr(L))) return bail(rc);
    }
    if (chosen) {
        shape_out(L->shape, chosen);
        chosen->tuned = 1;
    }
    if (n_tried) *n_tried = (int)cand.size();
    for (int c = 0; c < (int)cand.size() && c < max_tried; ++c) shape_out(cand[c], &tried[c]);
    cleanup();
    return TLL_OK;
}

const char *tll_last_error(void) { return g_err; }

int tll_version(void) { return 200; }

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
    L->epl = (flags & TLL_MASS_EPL) ? 1 : 0;
    L->nparam = L->epl ? NPAR_EPL : NPAR;
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
    L->psf_norm = pn;

    // weights (Eq. 5): w = 1/sigma^2 as a float pair, w*d likewise; masked
    // pixels get 0.  dWd = sum w d^2, lognorm = -sum log(2 pi sigma^2)/2.
    std::vector<float4> wp(npix);
    std::vector<unsigned char> used(npix, 0);
    double dWd = 0.0, lognorm = 0.0;
    for (int t = 0; t < npix; ++t) {
        const double s = noise[t], d = image[t];
        float4 q = make_float4(0.f, 0.f, 0.f, 0.f);
        if (isfinite(s) && s > 0.0 && isfinite(d)) {
            used[t] = 1;
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
    // Pixels within the PSF's reach of an unmasked pixel: the unmasked set
    // dilated by the K x K box (rows, then columns).  Only they can change
    // an unmasked blurred pixel (Eq. 3), so the batched kernels trace only
    // them when that leaves any pixel out.
    std::vector<int> tlist;
    {
        const int h = (K - 1) / 2, nx = g.nx, ny = g.ny;
        std::vector<unsigned char> rowd(npix, 0);
        for (int i = 0; i < ny; ++i) {
            int last = -1000000;   // column of the last unmasked pixel at or left of j + h
            for (int j = 0; j < nx + h; ++j) {
                if (j < nx && used[i * nx + j]) last = j;
                const int c = j - h;   // output column
                if (c >= 0 && c < nx) {
                    bool any = last >= c - h;
                    rowd[i * nx + c] = any ? 1 : 0;
                }
            }
        }
        for (int j = 0; j < nx; ++j) {
            int last = -1000000;
            for (int i = 0; i < ny + h; ++i) {
                if (i < ny && rowd[i * nx + j]) last = i;
                const int r = i - h;
                if (r >= 0 && r < ny && last >= r - h) tlist.push_back(r * nx + j);
            }
        }
        std::sort(tlist.begin(), tlist.end());
    }
    const bool listed = (int)tlist.size() < npix;   // some pixel left out (or all)

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
        (rc = alloc((void **)&L->d_p1, kMaxParams * sizeof(float))) ||
        (rc = alloc((void **)&L->d_kc1, NCONST * sizeof(float))) ||
        (rc = alloc((void **)&L->d_unb, 2 * npix * sizeof(float))) ||
        (rc = alloc((void **)&L->d_blur, 2 * npix * sizeof(float))) ||
        (rc = alloc((void **)&L->d_img, npix * sizeof(float))) ||
        (rc = alloc((void **)&L->d_res, 8 * sizeof(double))) ||
        (rc = alloc((void **)&L->d_out1, sizeof(double)))) {
        free_lens(L);
        return rc;
    }
    L->ntrace = listed ? (int)tlist.size() : npix;
    if (listed && (rc = alloc((void **)&L->d_tlist, std::max<size_t>(1, tlist.size()) * sizeof(int)))) {
        free_lens(L);
        return rc;
    }
    cudaError_t e = cudaSuccess;
    if (listed && !tlist.empty())
        e = cudaMemcpy(L->d_tlist, tlist.data(), tlist.size() * sizeof(int),
                       cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(L->d_psf, pn.data(), K * K * sizeof(float), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(L->d_pu, pu.data(), K * sizeof(float), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(L->d_pv, pv.data(), K * sizeof(float), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(L->d_wpack, wp.data(), npix * sizeof(float4), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        free_lens(L);
        return fail(TLL_ECUDA, "cudaMemcpy: %s", cudaGetErrorString(e));
    }
    if ((rc = configure(L)) || (rc = ensure_kc(L, 1024)) || (rc = bn_table(dev, &L->bn_tab)) ||
        (!(flags & TLL_FLAG_BATCH_ONLY) && (rc = ensure_gscr(L)))) {
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

// ---------------------------------------------------- autotune cache
// Text file: a header line "tll-autotune 1", then one line per tuned
// signature: "<GPU name, spaces as _> nx ny sub K separable threads ctas_per_sm".
namespace {
std::string gpu_name(int dev)
{
    cudaDeviceProp p;
    if (cudaGetDeviceProperties(&p, dev) != cudaSuccess) return std::string();
    std::string n(p.name);
    for (char &c : n)
        if (c == ' ' || c == '\t') c = '_';
    return n;
}
}  // namespace

int tll_autotune_save(const char *path)
{
    if (!path) return fail(TLL_EINVAL, "path is NULL");
    std::vector<std::pair<TuneKey, std::pair<int, int>>> all;
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        all.assign(g_tuned.begin(), g_tuned.end());
    }
    FILE *f = fopen(path, "w");
    if (!f) return fail(TLL_EINVAL, "cannot write %s", path);
    fprintf(f, "tll-autotune 1\n");
    for (const auto &e : all) {
        const std::string n = gpu_name(e.first.dev);
        fprintf(f, "%s %d %d %d %d %d %d %d\n", n.empty() ? "unknown" : n.c_str(), e.first.nx,
                e.first.ny, e.first.sub, e.first.K, e.first.sep, e.second.first, e.second.second);
    }
    const bool ok = fflush(f) == 0;
    fclose(f);
    return ok ? TLL_OK : fail(TLL_EINVAL, "cannot write %s", path);
}

int tll_autotune_load(const char *path)
{
    if (!path) return fail(TLL_EINVAL, "path is NULL");
    FILE *f = fopen(path, "r");
    if (!f) return fail(TLL_EINVAL, "cannot read %s", path);
    char line[512];
    int version = 0;
    if (!fgets(line, sizeof line, f) || sscanf(line, "tll-autotune %d", &version) != 1 ||
        version != 1) {
        fclose(f);
        return fail(TLL_EINVAL, "%s is not a tll autotune file", path);
    }
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev < 1) {
        fclose(f);
        return fail(TLL_ECUDA, "no CUDA device");
    }
    std::vector<std::string> names(ndev);
    for (int d = 0; d < ndev; ++d) names[d] = gpu_name(d);
    std::vector<std::pair<TuneKey, std::pair<int, int>>> add;
    int lineno = 1;
    while (fgets(line, sizeof line, f)) {
        ++lineno;
        char name[256];
        int nx, ny, sub, K, sep, threads, per_sm;
        if (sscanf(line, "%255s %d %d %d %d %d %d %d", name, &nx, &ny, &sub, &K, &sep, &threads,
                   &per_sm) != 8 ||
            nx < 1 || ny < 1 || sub < 1 || K < 1 || (sep != 0 && sep != 1) || threads < 32 ||
            threads > kThreads || threads % 32 || per_sm < 1) {
            fclose(f);
            return fail(TLL_EINVAL, "%s line %d is malformed", path, lineno);
        }
        for (int d = 0; d < ndev; ++d)
            if (names[d] == name)
                add.push_back({TuneKey{d, nx, ny, sub, K, sep}, {threads, per_sm}});
    }
    fclose(f);
    std::lock_guard<std::mutex> lk(g_tune_mu);
    for (const auto &e : add) g_tuned[e.first] = e.second;
    return TLL_OK;
}

void tll_autotune_clear(void)
{
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tuned.clear();
}

int tll_lens_ntrace(const tll_lens *L)
{
    if (!L) return fail(TLL_EINVAL, "lens is NULL"), -1;
    return L->d_tlist ? L->ntrace : L->npix;
}

int tll_lens_nparam(const tll_lens *L)
{
    if (!L) return fail(TLL_EINVAL, "lens is NULL"), -1;
    return L->nparam;
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
    if (L->nc) {
        if (!rc) rc = nc_ensure_scr(L);
        if (rc) return rc;
        return run_batch_nc(L, params, B, out, (cudaStream_t)stream, L->d_kc, nullptr);
    }
    if (!rc) rc = ensure_gscr(L);
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
        CUDA_TRY(cudaMalloc(&p, (size_t)cap * L->nparam * sizeof(float)));
        cudaError_t e = cudaMalloc(&o, (size_t)cap * sizeof(double));
        if (e != cudaSuccess) {
            cudaFree(p);
            return fail(TLL_ENOMEM, "cudaMalloc: %s", cudaGetErrorString(e));
        }
        if (L->d_stage_p) cudaFree(L->d_stage_p);
        if (L->d_stage_o) cudaFree(L->d_stage_o);
        L->dev_bytes += ((size_t)cap - L->stage_cap) * (L->nparam * sizeof(float) + sizeof(double));
        L->d_stage_p = p;
        L->d_stage_o = o;
        L->stage_cap = cap;
    }
    int rc = ensure_kc(L, B);
    if (!rc) rc = L->nc ? nc_ensure_scr(L) : ensure_gscr(L);
    if (rc) return rc;
    CUDA_TRY(cudaMemcpyAsync(L->d_stage_p, params, (size_t)B * L->nparam * sizeof(float),
                             cudaMemcpyHostToDevice, st));
    rc = L->nc ? run_batch_nc(L, L->d_stage_p, B, L->d_stage_o, st, L->d_kc, nullptr)
               : run_batch(L, L->d_stage_p, B, L->d_stage_o, st, false, L->d_kc);
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
    if (int rc = reject_nc(L, "tll_model_columns (use tll_model_columns_n)")) return rc;
    DeviceGuard gd(L->dev);
    int rc = run_one(L, params);
    if (rc) return rc;
    const float *src = blurred ? L->d_blur : L->d_unb;
    if (L->conv_variant != TLL_CONV_FUSED) {
        // the columns of the lens's split pipeline (its convolution variant)
        rc = run_split(L, L->d_kc1, 1, L->d_out1, 0);
        if (rc) return rc;
        CUDA_TRY(cudaDeviceSynchronize());
        if ((rc = tll_conv_check(L))) return rc;
        src = blurred ? L->d_sblur : L->d_unbl;
    }
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
    if (L->nc) {
        int rc = run_one_nc(L, params);
        if (rc) return rc;
        const float *cols = L->d_nscr + (size_t)L->nc * L->npix;   // slot 0, blurred
        k_combine_nc<<<std::max(1, std::min(1024, (L->npix + 255) / 256)), 256>>>(
            cols, L->d_nres, L->nc, L->npix, L->d_img);
        CUDA_TRY(cudaGetLastError());
        CUDA_TRY(cudaMemcpy(image_out, L->d_img, (size_t)L->npix * sizeof(float),
                            cudaMemcpyDeviceToHost));
        double res[kMaxComps + 1];
        CUDA_TRY(cudaMemcpy(res, L->d_nres, (L->nc + 1) * sizeof(double),
                            cudaMemcpyDeviceToHost));
        if (amps_out)
            for (int k = 0; k < L->nc; ++k) amps_out[k] = (float)res[k];
        if (loglike_out) *loglike_out = res[L->nc];
        return TLL_OK;
    }
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

int tll_set_light(tll_lens *L, const tll_comp_t *comps, int ncomp)
{
    if (!L) return fail(TLL_EINVAL, "lens is NULL");
    if (ncomp < 0 || ncomp > TLL_MAX_COMPS)
        return fail(TLL_EINVAL, "component count %d out of range [0, %d]", ncomp, TLL_MAX_COMPS);
    if (ncomp > 0 && !comps) return fail(TLL_EINVAL, "comps is NULL");
    if (ncomp > 0 && L->mode != TLL_AMP_LINEAR)
        return fail(TLL_EINVAL, "multi-component light needs TLL_AMP_LINEAR amplitudes");
    if (ncomp > 0 && L->conv_variant != TLL_CONV_FUSED)
        return fail(TLL_EINVAL, "multi-component light runs the fused pipeline only");
    MultiDev md = {};
    int npar = kMultiHead;
    for (int c = 0; c < ncomp; ++c) {
        const tll_comp_t &q = comps[c];
        if (q.type != TLL_COMP_SERSIC && q.type != TLL_COMP_GAUSSIAN)
            return fail(TLL_EINVAL, "component %d: unknown type %d", c, q.type);
        if (q.plane != TLL_PLANE_LENS && q.plane != TLL_PLANE_SOURCE)
            return fail(TLL_EINVAL, "component %d: unknown plane %d", c, q.plane);
        if (q.flags & ~(TLL_COMP_FREE_SCALE | TLL_COMP_FREE_INDEX))
            return fail(TLL_EINVAL, "component %d: unknown flags 0x%x", c, q.flags);
        if (!(q.flags & TLL_COMP_FREE_SCALE) && !(q.scale > 0.0f && isfinite(q.scale)))
            return fail(TLL_EINVAL, "component %d: fixed scale must be finite and > 0", c);
        const bool free_n = q.type == TLL_COMP_SERSIC && (q.flags & TLL_COMP_FREE_INDEX);
        if (q.type == TLL_COMP_SERSIC && !free_n && !(q.index >= 0.2f && q.index <= 10.0f))
            return fail(TLL_EINVAL, "component %d: fixed Sersic index must be in [0.2, 10]", c);
        md.type[c] = q.type == TLL_COMP_SERSIC ? COMP_SERSIC : COMP_GAUSS;
        md.plane[c] = q.plane == TLL_PLANE_LENS ? PLANE_LENS : PLANE_SOURCE;
        md.flags[c] = ((q.flags & TLL_COMP_FREE_SCALE) ? FREE_SCALE : 0) | (free_n ? FREE_INDEX : 0);
        md.scale[c] = q.scale;
        md.index[c] = q.index;
        npar += ((q.flags & TLL_COMP_FREE_SCALE) ? 1 : 0) + (free_n ? 1 : 0);
    }
    DeviceGuard gd(L->dev);
    CUDA_TRY(cudaDeviceSynchronize());
    if (ncomp == 0) {   // back to the two-column model
        if (L->d_nscr) {
            cudaFree(L->d_nscr);
            L->dev_bytes -= (size_t)L->nscr_floats * sizeof(float);
            L->d_nscr = nullptr;
            L->nscr_floats = 0;
        }
        L->nc = 0;
        L->nparam = L->epl ? NPAR_EPL : NPAR;
        return TLL_OK;
    }
    // trace schedule: lens-plane passes, then source-plane passes; per plane
    // the Gaussians in passes of up to kPassMax (lens plane) or kPassSrcG
    // (source plane), then the Sersics in passes of up to kPassMix, each in
    // list order
    for (int pl = 0; pl < 2; ++pl) {
        const int plane = pl == 0 ? PLANE_LENS : PLANE_SOURCE;
        for (int kind = 0; kind < 2; ++kind) {   // 0: Gaussians, 1: Sersics
            const int want = kind == 0 ? COMP_GAUSS : COMP_SERSIC;
            const int cap = kind == 1 ? kPassMix : plane == PLANE_LENS ? kPassMax : kPassSrcG;
            bool open = false;
            for (int c = 0; c < ncomp; ++c) {
                if (md.plane[c] != plane || md.type[c] != want) continue;
                if (!open || md.pass_n[md.npass - 1] == cap) {
                    md.pass_plane[md.npass] = plane;
                    md.pass_gauss[md.npass] = kind == 0;
                    md.pass_n[md.npass] = 0;
                    ++md.npass;
                    open = true;
                }
                md.pass_comp[md.npass - 1][md.pass_n[md.npass - 1]++] = c;
            }
        }
    }
    md.nc = ncomp;
    md.npar = npar + (L->epl ? 1 : 0);
    const int old_nc = L->nc;
    const MultiDev old_md = L->md;
    L->nc = ncomp;
    L->md = md;
    int rc = nc_configure(L);
    if (!rc && !L->d_nres) {
        cudaError_t e = cudaMalloc(&L->d_nres, (kMaxComps + 1) * sizeof(double));
        if (e != cudaSuccess) rc = fail(TLL_ENOMEM, "cudaMalloc: %s", cudaGetErrorString(e));
        else L->dev_bytes += (kMaxComps + 1) * sizeof(double);
    }
    // the one-lens image slots; a TLL_FLAG_BATCH_ONLY lens (evaluated through
    // a batcher or the server) gets them on first one-lens use instead
    if (!rc && !(L->flags & TLL_FLAG_BATCH_ONLY)) rc = nc_ensure_scr(L);
    if (rc) {
        L->nc = old_nc;
        L->md = old_md;
        return rc;
    }
    L->nparam = md.npar;
    return TLL_OK;
}

int tll_lens_ncols(const tll_lens *L)
{
    if (!L) return fail(TLL_EINVAL, "lens is NULL"), -1;
    return L->nc ? L->nc : 2;
}

int tll_model_columns_n(tll_lens *L, const float *params, float *cols_out, int blurred)
{
    if (!L) return fail(TLL_EINVAL, "lens is NULL");
    if (!cols_out) return fail(TLL_EINVAL, "NULL output");
    if (!L->nc)
        return tll_model_columns(L, params, cols_out, cols_out + L->npix, blurred);
    DeviceGuard gd(L->dev);
    int rc = run_one_nc(L, params);
    if (rc) return rc;
    const float *src = L->d_nscr + (blurred ? (size_t)L->nc * L->npix : 0);
    CUDA_TRY(cudaMemcpy(cols_out, src, (size_t)L->nc * L->npix * sizeof(float),
                        cudaMemcpyDeviceToHost));
    return TLL_OK;
}

}  // extern "C"
