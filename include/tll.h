/*
 * tll.h -- C ABI of the GB300 (sm_103a) lens log-likelihood library, libtll.so.
 *
 * The library evaluates, for a batch of parameter vectors against one
 * observed strong-lens image, the forward model and Gaussian log-likelihood
 * of arXiv:2503.08586 (TinyLensGpu):
 *   - lens equation beta = theta - alpha(theta) (Sec. 2.1, Eq. 1) with an
 *     SIE (Sec. 2.4, Eq. 12 at gamma = 2) or, for lenses created with
 *     TLL_MASS_EPL, the elliptical power law of Eq. 12 at any slope, plus
 *     external shear (Eqs. 13, 14);
 *   - image formation I = I_L(theta) + I_S(beta) (Eq. 2) with elliptical
 *     Sersic light (Eqs. 8-11), on an s x s supersampled grid binned back to
 *     pixels (Sec. 2.1, text after Eq. 2);
 *   - PSF convolution (Eq. 3);
 *   - non-negative linear amplitudes of the lens and source columns
 *     (Sec. 2.3, Eq. 7 and the penalty after it; Sec. 2.2, Eq. 6);
 *   - the Gaussian log-likelihood (Sec. 2.2, Eq. 5).
 * All arithmetic runs in this library's CUDA kernels.  There is no CPU
 * fallback: every entry point returns TLL_ECUDA when no usable GPU exists.
 *
 * Conventions shared by all entry points
 *   Grid: pixel (i row, j column) has its centre at (x0 + j*pixel_scale,
 *     y0 + i*pixel_scale) arcsec; subpixel (a, c) of its s x s grid sits at
 *     offset ((c + 1/2)/s - 1/2, (a + 1/2)/s - 1/2) * pixel_scale.  Images are
 *     float32, row-major [ny][nx].
 *   Parameter vector (TLL_NPARAM = 21 float32, row-major [B][21]):
 *     [0] theta_E  [1] eps1_m [2] eps2_m [3] x_m [4] y_m [5] gamma_1
 *     [6] gamma_2  [7] I_e^L [8] r_e^L [9] n^L [10] eps1_L [11] eps2_L
 *     [12] x_L [13] y_L [14] I_e^S [15] r_e^S [16] n^S [17] eps1_S
 *     [18] eps2_S [19] x_S [20] y_S
 *     Lenses created with TLL_MASS_EPL take TLL_NPARAM_EPL = 22 entries,
 *     [21] the mass slope gamma of Eq. 12 (valid in (1, 3); kappa =
 *     (3 - gamma)/2 (theta_E/R_p)^(gamma - 1) with the Eq. 10 radius).
 *     (ellipticities as Eq. 11; shear components with
 *     psi_ext = gamma_1 (x^2 - y^2)/2 + gamma_2 x y about the origin, which is
 *     Eq. 13 on the branch gamma_1 = -gamma cos 2phi of Eq. 14; I_e slots
 *     are used only with TLL_AMP_FIXED.)
 *   Invalid vectors (|eps| >= 1, r_e <= 0, n outside [0.2, 10],
 *     theta_E < 0, an EPL slope outside (1, 3), a non-finite entry) give
 *     log L = -INFINITY; the rest of the batch is unaffected.
 *   Masking: a pixel whose noise sigma is not finite and > 0, or whose datum
 *     is not finite, has weight 0 and no normalisation term.  Unmasked
 *     pixels need 1/sigma^2 and d/sigma^2 within the FP32 range (sigma above
 *     about 1e-19 for data of order 1): the weights are stored as FP32 pairs.  (The paper fits
 *     only a region of the image, Appendix A; give the other pixels an
 *     infinite sigma.)  The batched kernels trace only the pixels within the
 *     PSF's reach of an unmasked pixel (the unmasked set dilated by the
 *     PSF box), since no other pixel can change an unmasked blurred pixel
 *     (Eq. 3); the model-image calls trace every pixel.
 *   log L = -chi^2/2 - sum_{unmasked} log(2 pi sigma_i^2)/2, in FP64.
 *   Errors: every int-returning call returns TLL_OK (0) or a TLL_E* code and
 *     never aborts; tll_last_error() gives a message for the calling thread.
 */
#ifndef TLL_H
#define TLL_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

#define TLL_NPARAM 21
#define TLL_NPARAM_EPL 22
#define TLL_MAX_SUB 8      /* largest supersampling factor s */
#define TLL_MAX_PSF 63     /* largest PSF side */
#define TLL_MAX_SIDE 4096  /* largest image side */

enum {
    TLL_OK = 0,
    TLL_EINVAL = 1,   /* invalid argument (null pointer, bad size, ...) */
    TLL_ENOMEM = 2,   /* device or host allocation failed */
    TLL_ECUDA = 3,    /* CUDA runtime error or no usable GPU */
    TLL_ETIMEOUT = 4, /* a bounded wait ran out */
    TLL_EBUSY = 5     /* no capacity right now (server admission) */
};

/* Amplitude modes (the `flags` of tll_create_lens, low bits). */
enum {
    TLL_AMP_LINEAR = 0, /* amplitudes by non-negative least squares (Sec. 2.3) */
    TLL_AMP_FIXED = 1   /* amplitudes are the I_e slots [7], [14] */
};
/* Extra flag bit: never take the separable-PSF fast path (testing). */
#define TLL_FLAG_DIRECT_CONV 0x100
/* Extra flag bit: the lens is evaluated through a tll_batcher / tll_server;
 * skip the one-lens kernel's per-CTA image slots for images that do not fit
 * shared memory (8 or 16 B per pixel per resident CTA), allocated on first
 * use by the allocating one-lens entry points if it is evaluated alone
 * after all. */
#define TLL_FLAG_BATCH_ONLY 0x200
/* Extra flag bit: the mass is the elliptical power law of Eq. 12 with a free
 * slope (parameter vectors of TLL_NPARAM_EPL entries) instead of the SIE.
 * Its deflection is the closed form of Tessore & Metcalf (2015), a
 * hypergeometric series summed per vector to 1e-9 of its leading term (at
 * most 64 terms: axis ratios down to ~0.25 at that accuracy). */
#define TLL_MASS_EPL 0x400

typedef struct tll_lens tll_lens; /* opaque; owns device copies of its data */

typedef struct {
    int nx, ny;          /* image size in pixels */
    float pixel_scale;   /* arcsec per pixel, > 0 */
    int sub;             /* supersampling factor s, 1..TLL_MAX_SUB */
    float x0, y0;        /* arcsec coordinates of pixel (0, 0)'s centre */
} tll_grid_t;

/*
 * tll_create_lens -- copy one observed lens to the current CUDA device.
 *   image  host float32 [ny][nx], the data d (Sec. 2.3)
 *   noise  host float32 [ny][nx], sigma per pixel (Eq. 5); see Masking
 *   psf    host float32 [psf_size][psf_size], odd side <= TLL_MAX_PSF, finite,
 *          positive sum; the library normalises it to unit sum (Eq. 3)
 *   grid   image geometry (see Grid)
 *   flags  TLL_AMP_LINEAR or TLL_AMP_FIXED, optionally | TLL_FLAG_DIRECT_CONV
 *          | TLL_FLAG_BATCH_ONLY
 *   out    receives the new lens
 * The caller keeps ownership of all input buffers.  The lens owns its device
 * memory and per-launch scratch; destroy it with tll_destroy_lens.
 * Errors: TLL_EINVAL (null pointer, bad size, non-finite PSF, zero PSF sum),
 * TLL_ENOMEM, TLL_ECUDA.
 */
int tll_create_lens(const float *image, const float *noise, const float *psf,
                    int psf_size, const tll_grid_t *grid, int flags,
                    tll_lens **out);

/*
 * tll_loglike_batch -- log L of B parameter vectors (Eqs. 1-3, 5-12).
 *   params  DEVICE float32 [B][tll_lens_nparam(L)] (see Parameter vector)
 *   B       number of vectors, >= 0 (0: no work, TLL_OK)
 *   out     DEVICE float64 [B]
 *   stream  cudaStream_t to launch on (NULL: the legacy default stream)
 * Asynchronous: returns after enqueueing; the caller synchronises the
 * stream before reading out.  params and out stay owned by the caller and
 * must not be touched until the stream reaches this work.  Calls on one lens
 * must not overlap on different streams (they share the lens's scratch).
 * Errors: TLL_EINVAL, TLL_ENOMEM (scratch growth), TLL_ECUDA (launch).
 */
int tll_loglike_batch(tll_lens *L, const float *params, int B, double *out,
                      void *stream);

/*
 * tll_loglike_batch_host -- tll_loglike_batch from HOST buffers: copies
 * params (host float32 [B][tll_lens_nparam(L)]) to the device, runs the batch and copies the
 * log-likelihoods back to out (host float64 [B]), all on `stream`, and
 * waits for the stream.  Pinned host buffers make the copies asynchronous
 * DMA.  Errors: as tll_loglike_batch.
 */
int tll_loglike_batch_host(tll_lens *L, const float *params, int B,
                           double *out, void *stream);

/*
 * tll_batcher -- one launch over parameter batches of several lenses.
 * A ragged multi-lens batch (lenses of different sizes, supersampling and
 * PSFs, each with its own number of vectors) runs as one persistent launch:
 * CTAs take vectors from a shared work counter, largest lenses first, and
 * switch lens descriptors on the fly.  This is the batching of Sec. 3.1.4
 * ("batched likelihood evaluations") extended across lenses.
 *
 * tll_batcher_create -- a reusable context on the current device.
 *   use_graph  != 0: each run replays a captured CUDA graph (descriptor
 *              uploads, counter reset, prologue, kernel) on a non-default
 *              stream; the graph is re-captured when buffers grow or the
 *              stream changes.  0: plain launches.
 * tll_batcher_run -- enqueue n (lens, params, count, out) entries on stream.
 *   lenses  n lens handles (repeats allowed), all on the batcher's device
 *   params  n DEVICE pointers, float32 [count_k][21]
 *   counts  n batch sizes (0 allowed)
 *   outs    n DEVICE pointers, float64 [count_k]
 *   Asynchronous; results as tll_loglike_batch for each entry.  The lens
 *   handles' scratch is not used (the batcher owns its own), but the
 *   params/out buffers must stay valid until the stream reaches the work.
 *   Runs on one batcher are ordered by its internal staging fence.
 * Errors: TLL_EINVAL, TLL_ENOMEM, TLL_ECUDA.
 */
typedef struct tll_batcher tll_batcher;
int tll_batcher_create(int use_graph, tll_batcher **out);
int tll_batcher_run(tll_batcher *b, tll_lens *const *lenses,
                    const float *const *params, const int *counts,
                    double *const *outs, int n, void *stream);
void tll_batcher_destroy(tll_batcher *b);

/*
 * Continuous-batching server.  The paper's sampler calls the likelihood in
 * batches of proposals (Sec. 3.1.4) and names host-device transfers and
 * one-lens-at-a-time GPU use as its bottleneck (Sec. 3.1.4, 4.2); serving
 * many lenses at once on one GPU has no counterpart in the paper and is a
 * deployment layer over tll_batcher.
 *
 * A job is one observed lens kept on the device; it is admitted if its
 * device footprint fits the remaining budget (else TLL_EBUSY: retry after
 * another job closes).  A request is one parameter batch of one job, from
 * host memory.  A launcher thread merges all pending requests (of any job)
 * into one multi-lens launch per free slot; up to max_inflight launches run
 * on their own streams, so work that arrives while others run joins the
 * next launch and overlaps on the GPU.  Each result is the same as the
 * job's own tll_loglike_batch (one vector never depends on another).
 */
typedef struct tll_server tll_server;
typedef struct {
    size_t hbm_budget_bytes;    /* device bytes open jobs may hold; 0: no limit */
    int max_jobs;               /* job slots */
    int max_vectors_per_launch; /* merge cap per launch, and the largest request */
    int max_inflight;           /* launches in flight, 1..4 */
    int coalesce;               /* 1: merge pending requests; 0: one per launch */
    int use_graph;              /* replay each launch as a CUDA graph */
    int autotune;               /* 1: tll_autotune (built-in vectors) each job
                                   whose lens signature is not tuned yet, at
                                   admission, on a stream of its own */
} tll_server_config_t;
typedef struct {
    long long launches, vectors, requests, admissions_refused, pending, inflight;
    size_t hbm_used_bytes;
    int open_jobs;
    double latency_p50_ms, latency_p99_ms, latency_max_ms; /* submit -> result,
                                                              last 65536 requests */
} tll_server_stats_t;

/* Create a server on the current device (starts two host threads). */
int tll_server_create(const tll_server_config_t *cfg, tll_server **out);
/* Admit a lens (arguments as tll_create_lens); *job_id >= 0 on success,
 * TLL_EBUSY when the budget or the job slots are exhausted. */
int tll_server_open_job(tll_server *S, const float *image, const float *noise,
                        const float *psf, int psf_size, const tll_grid_t *grid,
                        int flags, int *job_id);
/* Release a job; TLL_EBUSY while it has requests not yet completed. */
int tll_server_close_job(tll_server *S, int job_id);
/* Queue B vectors (host float32 [B][nparam of the job's lens]) of a job; results go to out (host
 * float64 [B]).  Both buffers must stay valid until the request completes.
 * 1 <= B <= max_vectors_per_launch. */
int tll_server_submit(tll_server *S, int job_id, const float *params, int B,
                      double *out, long long *request_id);
/* *done = 1 once the request's results are in out. */
int tll_server_poll(tll_server *S, long long request_id, int *done);
/* Wait for a request (timeout_ms < 0: no limit; TLL_ETIMEOUT when it runs
 * out, the request stays valid); on success the request is released and
 * *latency_ms (may be NULL) is its submit-to-result time. */
int tll_server_wait(tll_server *S, long long request_id, int timeout_ms,
                    double *latency_ms);
int tll_server_stats(tll_server *S, tll_server_stats_t *st);
/* Finish queued work, stop the threads, release every job. */
void tll_server_destroy(tll_server *S);
/* Message for the last server error on the calling thread. */
const char *tll_server_last_error(void);

/*
 * tll_loglike_batch_noalloc -- tll_loglike_batch for callers that must not
 * allocate device memory during the call: for example a process whose
 * device memory is entirely reserved by another allocator (a framework's
 * caching allocator, a fixed per-job budget), where cudaMalloc would fail,
 * or a latency-critical sampler loop that cannot accept cudaMalloc/cudaFree
 * stalls.  (tll_loglike_batch grows a lens-owned scratch buffer with
 * cudaMalloc when B exceeds what it has seen.)  There is no counterpart in
 * the paper; this is a deployment variant of the same computation.
 *   Same arguments, results and asynchrony as tll_loglike_batch.
 *   B must be <= TLL_NOALLOC_MAX_B; larger batches give TLL_EINVAL (split
 *     them into several calls).
 *   Scratch: a fixed array (TLL_NOALLOC_MAX_B constant blocks, 22 MB)
 *     compiled into the library.  A device holds it from the first use of
 *     the library's kernels there (module loading is lazy by default; the
 *     lens's tll_create_lens already loaded it) until the process exits.
 *     All calls share it and it
 *     keeps the last call's contents; each call rewrites the part it reads
 *     before reading it.  Calls that overlap on the GPU (different streams,
 *     different lenses) race on it: order them on one stream or synchronise.
 *   Set-up: the first call on each device looks up the array's device
 *     address (cudaGetSymbolAddress) with that device current; make that
 *     first call before any stream capture.
 *   The call itself makes no cudaMalloc, cudaFree or other allocating call;
 *   the lens must already exist (tll_create_lens allocates).
 */
#define TLL_NOALLOC_MAX_B 16384
int tll_loglike_batch_noalloc(tll_lens *L, const float *params, int B,
                              double *out, void *stream);

/*
 * tll_model_image -- the blurred model image I^m (Eq. 3) of one vector with
 * its amplitudes: linear (NNLS) or fixed, per the lens's mode.
 *   params     host float32 [tll_lens_nparam(L)]
 *   image_out  host float32 [ny][nx]
 *   amps_out   host float32 [tll_lens_ncols(L)] (lens, source amplitude;
 *              or one per component) or NULL
 *   loglike_out host float64 [1] or NULL
 * Synchronous.  An invalid vector gives TLL_EINVAL.
 */
int tll_model_image(tll_lens *L, const float *params, float *image_out,
                    float *amps_out, double *loglike_out);

/*
 * tll_model_columns -- the two unit-amplitude columns of L (Eq. 7) for one
 * vector: lens light and lensed source, binned, before (blurred = 0) or after
 * (blurred = 1) the PSF.  params host [21]; lens_out, src_out host float32
 * [ny][nx].  Synchronous.  An invalid vector gives TLL_EINVAL.
 */
int tll_model_columns(tll_lens *L, const float *params, float *lens_out,
                      float *src_out, int blurred);

/*
 * tll_profile_enable / tll_profile_last -- per-launch timing for profiling.
 * While enabled (on != 0), each tll_loglike_batch / _host call records CUDA
 * events on its stream before the prologue launch, between the two launches
 * and after the main launch.  tll_profile_last waits for the last call's
 * events and returns the prologue and main-kernel durations in ms.  The
 * events belong to the lens.  Errors: TLL_EINVAL (not enabled, no call yet),
 * TLL_ECUDA.
 */
int tll_profile_enable(tll_lens *L, int on);
int tll_profile_last(tll_lens *L, float *prologue_ms, float *main_ms);

/* Device memory a lens currently holds, in bytes (its data, the model
 * buffers, and the scratch it has grown). */
int tll_lens_footprint(const tll_lens *L, size_t *bytes);

/*
 * Launch shapes and the autotuner.
 * A lens's batched likelihood kernels (tll_loglike_batch*, and the lens's
 * group in tll_batcher_run / the server) run persistent CTAs, each taking
 * one parameter vector at a time (ray-trace + light of every subpixel,
 * binning, PSF convolution, weighted sums; Sec. 2.1-2.4).  Its shape is the
 * CTA size, how many CTAs share an SM, and where each CTA keeps the two
 * binned images:
 *   TLL_PLACE_PADDED  whole zero-padded images in shared memory, convolution
 *                     compiled for the PSF side (PSF side <= 31, nx <= 256)
 *   TLL_PLACE_BANDED  images in a per-CTA global slot (L2-resident),
 *                     convolved band by band through a padded shared buffer
 *                     (same compiled convolution; images too large to pad)
 *   TLL_PLACE_SMEM    unpadded images in shared memory, generic convolution
 *   TLL_PLACE_GLOBAL  images in a per-CTA global slot, generic convolution
 * A new lens takes 1024-thread CTAs, one per SM, and the first placement
 * that fits -- or the tuned shape of an earlier lens with the same
 * signature (device, nx, ny, s, PSF side, separable PSF) in this process.
 */
enum {
    TLL_PLACE_GLOBAL = 0,
    TLL_PLACE_SMEM = 1,
    TLL_PLACE_PADDED = 2,
    TLL_PLACE_BANDED = 3
};
typedef struct {
    int threads;        /* CTA size */
    int ctas_per_sm;    /* CTAs resident per SM; a launch has SMs x this CTAs */
    int placement;      /* TLL_PLACE_* */
    int band_rows;      /* output rows per band (TLL_PLACE_BANDED), else 0 */
    size_t smem_bytes;  /* dynamic shared memory per CTA */
    float ms;           /* mean time of one tuning batch (0: not timed) */
    int tuned;          /* 1: chosen by tll_autotune (here or for an earlier
                           lens of the same signature) */
} tll_shape_t;

/* The lens's current launch shape (for a multi-component lens, the
 * multi-column kernel's: 1024-thread CTAs, one per SM, its band rows and
 * shared memory; never tuned). Errors: TLL_EINVAL (NULL argument). */
int tll_lens_shape(const tll_lens *L, tll_shape_t *out);

/*
 * Convolution variants (Eq. 3) of a lens's one-lens batched entry points
 * (tll_loglike_batch*, tll_model_columns); the batcher and the server always
 * use the fused kernels.
 *   TLL_CONV_FUSED        the default: trace, convolution and sums in one
 *                         kernel (separable or direct FP32 FMAs)
 *   TLL_CONV_SPLIT_DIRECT a split pipeline -- trace kernel, convolution
 *                         kernel, sums kernel, images of `chunk` vectors in
 *                         device memory -- with a direct FP32 convolution
 *                         (whole padded image in shared memory)
 *   TLL_CONV_SPLIT_TOEPLITZ_TC  the same pipeline with the convolution of
 *                         each PSF row as a GEMM with a banded Toeplitz
 *                         matrix on the tensor cores (tcgen05, TF32 with
 *                         three products per term for FP32-level accuracy);
 *                         PSF side <= 33
 *   TLL_CONV_SPLIT_TOEPLITZ_BF16  the same GEMM with both operands split
 *                         into three BF16 parts (hi + mid + lo, every FP32
 *                         mantissa bit) and the six products down to 2^-24
 *                         relative (tcgen05 kind::f16); PSF side <= 33
 * The split variants exist to compare the two convolutions on the same
 * inputs.  chunk: vectors per pass of the split pipeline (0: 1024); it holds
 * 16 B per pixel per vector of device memory.  Waits for the device first.
 * Errors: TLL_EINVAL (unknown variant, image or PSF too large), TLL_ENOMEM,
 * TLL_ECUDA.
 */
enum {
    TLL_CONV_FUSED = 0,
    TLL_CONV_SPLIT_DIRECT = 1,
    TLL_CONV_SPLIT_TOEPLITZ_TC = 2,
    TLL_CONV_SPLIT_TOEPLITZ_BF16 = 3
};
int tll_set_conv(tll_lens *L, int variant, int chunk);

/* Wait for the device and report whether the tensor-core convolution's
 * bounded waits ran out since the last check (TLL_ETIMEOUT: the affected
 * outputs are not valid), else TLL_OK. */
int tll_conv_check(tll_lens *L);

/*
 * tll_set_shape -- give the lens the shape of `threads`-thread CTAs (a
 * multiple of 32, <= 1024) with ctas_per_sm of them per SM, and the
 * placement that share of shared memory allows.  Waits for the device to
 * be idle first.  Errors: TLL_EINVAL (no such shape fits), TLL_ENOMEM,
 * TLL_ECUDA (the lens keeps its shape).
 */
int tll_set_shape(tll_lens *L, int threads, int ctas_per_sm);

/*
 * tll_autotune -- time the candidate shapes (1 x 1024, 2 x 512 and 4 x 256
 * threads per SM, each with the placement its shared-memory share allows)
 * on the device and give the lens the fastest; later lenses with the same
 * signature start with it.
 *   params     DEVICE float32 [B][tll_lens_nparam(L)] vectors to time with, repeated
 *              to at least two per CTA; or NULL with B = 0 for a built-in
 *              set covering both SIE branches and steep and shallow Sersics
 *   stream     cudaStream_t the tuning launches run on (NULL: default)
 *   chosen     receives the chosen shape (may be NULL)
 *   tried      receives up to max_tried candidate shapes with their times
 *   n_tried    receives the number of candidates timed (may be NULL)
 * Blocks until the tuning launches end.  Allocates temporary device buffers;
 * the lens's one-lens image slots are resized to the chosen shape.  Must
 * not run while other calls use the same lens.  Results of the likelihood
 * do not depend on the shape beyond rounding (the sums' order changes).
 * Errors: TLL_EINVAL, TLL_ENOMEM, TLL_ECUDA (the lens keeps its shape).
 */
int tll_autotune(tll_lens *L, const float *params, int B, void *stream,
                 tll_shape_t *chosen, tll_shape_t *tried, int max_tried,
                 int *n_tried);

/*
 * The autotuner's choices outlive the process in a cache file:
 * tll_autotune_save writes every tuned signature of this process (GPU name,
 * nx, ny, s, PSF side, separable PSF -> CTA size, CTAs per SM) as text;
 * tll_autotune_load adds a file's entries for the GPUs present with the same
 * name, so lenses created afterwards start with those shapes (a restarted
 * server skips re-tuning); tll_autotune_clear forgets every tuned shape.
 * Errors: TLL_EINVAL (NULL path, unreadable / unwritable or malformed
 * file), TLL_ECUDA (load: no CUDA device).
 */
int tll_autotune_save(const char *path);
int tll_autotune_load(const char *path);
void tll_autotune_clear(void);

/* Entries per parameter vector of this lens: TLL_NPARAM, or TLL_NPARAM_EPL
 * for a TLL_MASS_EPL lens, or the multi-component layout's count after
 * tll_set_light (-1 for NULL). */
int tll_lens_nparam(const tll_lens *L);

/*
 * Multi-component light (Sec. 2.3, Eq. 7: the lens light and the source
 * light are superpositions of N_l and N_s profiles, each a column of
 * L = [L_l | L_s] with its own non-negative amplitude, solved by FNNLS).
 * Sec. 3.2 fits SLACS lenses with two Sersics per galaxy sharing one centre
 * and one ellipticity, indices fixed at 1 and 4; Sec. 4.3 names the
 * Gaussian expansion.  A component is an elliptical Sersic (Eq. 8, unit
 * I_e) or an elliptical Gaussian of unit central intensity,
 * exp(-R_p^2 / (2 sigma^2)) with the R_p of Eq. 10, placed in the lens plane
 * (evaluated at theta) or the source plane (at beta of Eq. 1).  All
 * components of one plane share that plane's centre and ellipticity.
 *
 * Parameter vector of a multi-component lens (float32):
 *   [0] theta_E [1] eps1_m [2] eps2_m [3] x_m [4] y_m [5] gamma_1 [6] gamma_2
 *   [7] eps1_L [8] eps2_L [9] x_L [10] y_L      (lens-plane geometry)
 *   [11] eps1_S [12] eps2_S [13] x_S [14] y_S   (source-plane geometry)
 *   then, component by component, its scale (r_e or sigma, arcsec) if
 *   TLL_COMP_FREE_SCALE, then its Sersic index if TLL_COMP_FREE_INDEX;
 *   a TLL_MASS_EPL lens appends the mass slope last.  Values that are not
 *   free come from the component list.  Invalid vectors (scale <= 0, index
 *   outside [0.2, 10], |eps| >= 1, theta_E < 0, a slope outside (1, 3),
 *   non-finite entries) give log L = -INFINITY.
 * The amplitudes are the non-negative least-squares solution over all
 * columns (FNNLS, Bro & de Jong 1997, in FP64 per vector); log L as above.
 */
#define TLL_MAX_COMPS 32
enum { TLL_COMP_SERSIC = 0, TLL_COMP_GAUSSIAN = 1 };
enum { TLL_PLANE_LENS = 0, TLL_PLANE_SOURCE = 1 };
#define TLL_COMP_FREE_SCALE 1   /* scale read from the parameter vector */
#define TLL_COMP_FREE_INDEX 2   /* Sersic index read from the parameter vector */
typedef struct {
    int type;     /* TLL_COMP_SERSIC or TLL_COMP_GAUSSIAN */
    int plane;    /* TLL_PLANE_LENS or TLL_PLANE_SOURCE */
    int flags;    /* TLL_COMP_FREE_SCALE | TLL_COMP_FREE_INDEX */
    float scale;  /* fixed r_e or sigma (arcsec) when not free */
    float index;  /* fixed Sersic index when not free */
} tll_comp_t;

/*
 * tll_set_light -- give lens L the multi-component light model `comps`
 * (1..TLL_MAX_COMPS components; columns in list order), or with ncomp = 0
 * return it to the two-column Sersic model of TLL_NPARAM.  The lens must
 * use TLL_AMP_LINEAR and the fused convolution.  Allocates the model's
 * per-CTA image slots ((2 ncomp + 3) x 4 bytes per pixel per SM) and waits
 * for the device first.  Afterwards tll_loglike_batch, _host, _noalloc,
 * tll_model_image (amps_out receives ncomp amplitudes) and
 * tll_model_columns_n, the batcher (its multi-column lenses run in their
 * own multi-lens launches) and the server (tll_server_set_light) evaluate
 * the new model; tll_model_columns, tll_set_shape, tll_set_conv and
 * tll_autotune refuse the lens with TLL_EINVAL.  A lens created with
 * TLL_FLAG_BATCH_ONLY gets its one-lens image slots on first one-lens use.
 * Errors: TLL_EINVAL (bad list), TLL_ENOMEM, TLL_ECUDA (the lens keeps its
 * previous model).
 */
int tll_set_light(tll_lens *L, const tll_comp_t *comps, int ncomp);

/* Give a server job's lens a multi-component light model (as tll_set_light;
 * its requests then take that model's parameter layout).  Only while the job
 * has no request outstanding (else TLL_EBUSY).  Errors as tll_set_light. */
int tll_server_set_light(tll_server *S, int job_id, const tll_comp_t *comps, int ncomp);

/* Columns of the lens's model: 2 (lens, source) or its component count. */
int tll_lens_ncols(const tll_lens *L);

/*
 * tll_model_columns_n -- every unit-amplitude column of L (Eq. 7) for one
 * vector (params host [tll_lens_nparam(L)]), binned, before (blurred = 0)
 * or after (blurred = 1) the PSF, to cols_out (host float32
 * [tll_lens_ncols(L)][ny][nx]).  Synchronous.  An invalid vector gives
 * TLL_EINVAL.
 */
int tll_model_columns_n(tll_lens *L, const float *params, float *cols_out, int blurred);

/* Pixels the batched kernels trace per vector: npix, or fewer for a lens
 * with masked pixels (see Masking); -1 for NULL. */
int tll_lens_ntrace(const tll_lens *L);

/*
 * Device-side sampler loop.  The paper's sampler runs on the CPU and calls
 * the GPU likelihood for each batch of proposals; it names those host round
 * trips as the bottleneck and proposes moving the sampler to the GPU
 * (Sec. 4.2).  tll_sampler keeps an ensemble of W walkers on the device and
 * advances it with the affine-invariant stretch move (Goodman & Weare 2010):
 * proposals, the lens's batched likelihood, accept / reject and the chain all
 * run in CUDA kernels, so tll_sampler_run enqueues any number of steps
 * without waiting.  One step updates walkers [0, W/2) against partners from
 * [W/2, W), then the reverse.  For walker k of half h, with r0..r3 the
 * Philox4x32-10 outputs (Salmon et al. 2011) for key (seed mod 2^32,
 * seed / 2^32) and counter (k, h, step mod 2^32, step / 2^32):
 *   partner  j = first walker of the other half + floor(r0 (W/2) / 2^32)
 *   stretch  z = ((a - 1) u + 1)^2 / a with u = (r1 + 1/2) / 2^32
 *   proposal Y = x_j + z (x_k - x_j) in FP64 (one rounding per operation),
 *            rounded to float32
 *   accept   if log((r2 + 1/2) / 2^32) < (ndim - 1) log z + lp(Y) - lp(x_k)
 * where lp = log L inside the box prior [lo, hi] and -inf outside (entries
 * with lo == hi are fixed: give every walker that value).  Steps are numbered
 * from 0 across runs, so a run continues the stream of random numbers.
 */
typedef struct tll_sampler tll_sampler;
/* nwalkers even, >= 4; lo, hi host float32 [tll_lens_nparam(L)]; a > 1 (2 is
 * the usual choice); ndim: dimension of the sampled space for the z^(ndim-1)
 * factor, <= 0 for the number of entries with lo < hi.  Allocates the
 * ensemble's buffers and the lens's one-lens image slots.  The sampler uses
 * the lens: no other call on the lens may overlap a run. */
int tll_sampler_create(tll_lens *L, int nwalkers, const float *lo, const float *hi,
                       double a, int ndim, unsigned long long seed, tll_sampler **out);
/* Copy the starting walkers (DEVICE float32 [W][nparam]) and evaluate their
 * log posterior, on stream. */
int tll_sampler_set_walkers(tll_sampler *S, const float *x0, void *stream);
/* Enqueue nsteps steps on stream.  Optional DEVICE outputs (NULL to skip):
 * chain float32 [nsteps][W][nparam] (the walkers after each step), lp_chain
 * float64 [nsteps][W] (their log posterior), lp_prop_chain float64
 * [nsteps][W] (each walker's proposal's log posterior at that step). */
int tll_sampler_run(tll_sampler *S, int nsteps, float *chain, double *lp_chain,
                    double *lp_prop_chain, void *stream);
/* Copy the current walkers (DEVICE float32 [W][nparam]) and log posteriors
 * (DEVICE float64 [W]) -- either may be NULL -- and report the steps taken
 * and the moves accepted and proposed so far; waits for stream. */
int tll_sampler_state(tll_sampler *S, float *x, double *lp, long long *step,
                      long long *accepted, long long *proposed, void *stream);
/* Wait for the device and release the sampler (NULL is a no-op). */
void tll_sampler_destroy(tll_sampler *S);

/* Image size and mode of a lens (any pointer may be NULL). */
int tll_lens_info(const tll_lens *L, int *nx, int *ny, int *sub, int *psf_size,
                  int *flags, int *separable);

/* Release a lens and its device memory (NULL is a no-op). */
void tll_destroy_lens(tll_lens *L);

/* Message for the last error on the calling thread ("" if none). */
const char *tll_last_error(void);

/* Library version, major*10000 + minor*100 + patch. */
int tll_version(void);

#ifdef __cplusplus
}
#endif
#endif /* TLL_H */
