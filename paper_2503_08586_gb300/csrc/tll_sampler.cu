// tll_sampler.cu -- a sampler loop that stays on the GPU.
//
// The paper's sampler runs on the CPU and calls the GPU likelihood for each
// batch of proposals; it names those host round trips as the bottleneck and
// proposes moving the sampler onto the GPU (Sec. 4.2).  This is such a loop:
// an ensemble of W walkers updated by the affine-invariant "stretch move" of
// Goodman & Weare (2010), every step on the device -- proposals, the batched
// likelihood of the lens (the library's own kernels), the accept / reject
// and the chain -- so a run of many steps is enqueued by the host without a
// single synchronisation.
//
// One step updates half 0 (walkers [0, W/2)) and then half 1 ([W/2, W)).
// For walker k of half h, with the Philox4x32-10 outputs r0..r3 (Salmon et
// al. 2011) at key (seed low, seed high) and counter (k, h, step low, step
// high):
//   partner  j = (first walker of the other half) + floor(r0 (W/2) / 2^32)
//   stretch  u = (r1 + 1/2) 2^-32, z = ((a - 1) u + 1)^2 / a  (density
//            ~ 1/sqrt(z) on [1/a, a])
//   proposal Y = x_j + z (x_k - x_j) in FP64, one rounding per operation,
//            then to float32
//   accept   when log((r2 + 1/2) 2^-32) < (ndim - 1) log z + lp(Y) - lp(x_k),
//            lp(Y) = log L(Y) inside the box prior [lo, hi] (coordinates with
//            lo == hi are fixed), -inf outside.
// (The per-walker steps are in tll_stretch.cuh.)  Launches per half step:
// when the half fits the likelihood kernel's grid (each CTA one vector,
// the kernel decoding its own vector), ONE -- the likelihood kernel makes
// its walker's proposal before the decode and takes the accept / reject
// after its log L; otherwise proposals, the likelihood's two, accept.  Plus
// two copies per step into the caller's chain buffers.
#include <cuda_runtime.h>

#include <math.h>
#include <stdint.h>

#include <algorithm>
#include <new>
#include <vector>

#include "tll.h"
#include "tll_internal.h"
#include "tll_stretch.cuh"

using namespace tll;

namespace {

// Proposals of half s.h: one thread per walker of the half.
__global__ void k_stretch_propose(const StretchStep s, float *__restrict__ Y)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < s.W / 2) stretch_propose_entries(s, t, 0, 1, Y + (size_t)t * s.P, nullptr);
}

// Accept / reject half s.h: one thread per walker of the half.  lpY holds
// the proposals' log L.
__global__ void k_stretch_accept(const StretchStep s, const float *__restrict__ Y,
                                 const double *__restrict__ lpY)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < s.W / 2) stretch_accept_one(s, t, Y + (size_t)t * s.P, lpY[t]);
}

// Initial walkers: log posterior = log L inside the box, -inf outside.
__global__ void k_apply_box(const float *__restrict__ x, int W, int P, const float *__restrict__ lo,
                            const float *__restrict__ hi, double *__restrict__ lp)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < W && !in_box(x + (size_t)k * P, lo, hi, P)) lp[k] = -INFINITY;
}

#define S_TRY(expr)                                                                    \
    do {                                                                               \
        cudaError_t e_ = (expr);                                                       \
        if (e_ != cudaSuccess)                                                         \
            return set_error(e_ == cudaErrorMemoryAllocation ? TLL_ENOMEM : TLL_ECUDA, \
                             "%s: %s", #expr, cudaGetErrorString(e_));                 \
    } while (0)

struct DevGuard {
    int prev = -1;
    explicit DevGuard(int dev)
    {
        if (cudaGetDevice(&prev) == cudaSuccess && prev != dev) cudaSetDevice(dev);
        else prev = -1;
    }
    ~DevGuard()
    {
        if (prev >= 0) cudaSetDevice(prev);
    }
};

}  // namespace

struct tll_sampler {
    tll_lens *L = nullptr;
    int dev = 0, W = 0, P = 0, ndim = 0;
    double a = 2.0;
    unsigned long long seed = 0;
    long long step = 0, proposed = 0;
    bool ready = false;
    float *d_x = nullptr, *d_Y = nullptr, *d_lo = nullptr, *d_hi = nullptr, *d_kc = nullptr;
    double *d_lp = nullptr, *d_lpY = nullptr;
    unsigned long long *d_nacc = nullptr;
};

namespace {
void sampler_free(tll_sampler *S)
{
    if (!S) return;
    void *ptrs[] = {S->d_x, S->d_Y, S->d_lo, S->d_hi, S->d_kc, S->d_lp, S->d_lpY, S->d_nacc};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    delete S;
}
}  // namespace

extern "C" {

int tll_sampler_create(tll_lens *L, int nwalkers, const float *lo, const float *hi, double a,
                       int ndim, unsigned long long seed, tll_sampler **out)
{
    if (!out) return set_error(TLL_EINVAL, "out is NULL");
    *out = nullptr;
    if (!L || !lo || !hi) return set_error(TLL_EINVAL, "NULL argument");
    if (nwalkers < 4 || nwalkers % 2 || nwalkers > (1 << 22))
        return set_error(TLL_EINVAL, "walker count %d must be even, 4 .. 2^22", nwalkers);
    if (!(a > 1.0) || !isfinite(a)) return set_error(TLL_EINVAL, "stretch scale a must be > 1");
    const int P = lens_nparam(L);
    int nfree = 0;
    for (int i = 0; i < P; ++i) {
        if (!isfinite(lo[i]) || !isfinite(hi[i]) || lo[i] > hi[i])
            return set_error(TLL_EINVAL, "prior box entry %d is not a finite lo <= hi", i);
        nfree += lo[i] < hi[i];
    }
    if (ndim <= 0) ndim = nfree;
    if (ndim < 1 || ndim > P) return set_error(TLL_EINVAL, "ndim %d out of range", ndim);
    tll_sampler *S = new (std::nothrow) tll_sampler;
    if (!S) return set_error(TLL_ENOMEM, "host allocation failed");
    S->L = L;
    S->dev = lens_device(L);
    S->W = nwalkers;
    S->P = P;
    S->ndim = ndim;
    S->a = a;
    S->seed = seed;
    DevGuard g(S->dev);
    const size_t W = nwalkers, half = W / 2;
    cudaError_t e = cudaSuccess;
    auto alloc = [&](void **p, size_t bytes) {
        if (e == cudaSuccess) e = cudaMalloc(p, bytes);
    };
    alloc((void **)&S->d_x, W * P * sizeof(float));
    alloc((void **)&S->d_Y, half * P * sizeof(float));
    alloc((void **)&S->d_lo, P * sizeof(float));
    alloc((void **)&S->d_hi, P * sizeof(float));
    alloc((void **)&S->d_kc, W * (size_t)const_block_floats() * sizeof(float));
    alloc((void **)&S->d_lp, W * sizeof(double));
    alloc((void **)&S->d_lpY, half * sizeof(double));
    alloc((void **)&S->d_nacc, sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaMemcpy(S->d_lo, lo, P * sizeof(float), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(S->d_hi, hi, P * sizeof(float), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(S->d_nacc, 0, sizeof(unsigned long long));
    if (e != cudaSuccess) {
        sampler_free(S);
        return set_error(e == cudaErrorMemoryAllocation ? TLL_ENOMEM : TLL_ECUDA,
                         "sampler buffers: %s", cudaGetErrorString(e));
    }
    if (int rc = lens_prepare(L)) {
        sampler_free(S);
        return rc;
    }
    *out = S;
    return TLL_OK;
}

int tll_sampler_set_walkers(tll_sampler *S, const float *x0, void *stream)
{
    if (!S || !x0) return set_error(TLL_EINVAL, "NULL argument");
    DevGuard g(S->dev);
    cudaStream_t st = (cudaStream_t)stream;
    S_TRY(cudaMemcpyAsync(S->d_x, x0, (size_t)S->W * S->P * sizeof(float),
                          cudaMemcpyDeviceToDevice, st));
    if (int rc = lens_eval(S->L, S->d_x, S->W, S->d_lp, st, S->d_kc)) return rc;
    k_apply_box<<<(S->W + 127) / 128, 128, 0, st>>>(S->d_x, S->W, S->P, S->d_lo, S->d_hi,
                                                      S->d_lp);
    S_TRY(cudaGetLastError());
    S->ready = true;
    return TLL_OK;
}

int tll_sampler_run(tll_sampler *S, int nsteps, float *chain, double *lp_chain,
                    double *lp_prop_chain, void *stream)
{
    if (!S) return set_error(TLL_EINVAL, "sampler is NULL");
    if (nsteps < 0) return set_error(TLL_EINVAL, "negative step count");
    if (!S->ready) return set_error(TLL_EINVAL, "set the walkers first");
    DevGuard g(S->dev);
    cudaStream_t st = (cudaStream_t)stream;
    const int half = S->W / 2, blocks = (half + 127) / 128;
    const bool fused = lens_eval_fuses(S->L, half);
    for (int s = 0; s < nsteps; ++s) {
        for (int h = 0; h < 2; ++h) {
            StretchStep ss;
            ss.x = S->d_x;
            ss.lp = S->d_lp;
            ss.lp_prop = lp_prop_chain ? lp_prop_chain + (size_t)s * S->W : nullptr;
            ss.nacc = S->d_nacc;
            ss.lo = S->d_lo;
            ss.hi = S->d_hi;
            ss.step = S->step;
            ss.seed = S->seed;
            ss.a = S->a;
            ss.W = S->W;
            ss.P = S->P;
            ss.h = h;
            ss.ndim = S->ndim;
            if (fused) {
                if (int rc = lens_eval_stretch(S->L, S->d_Y, half, S->d_lpY, st, S->d_kc, ss))
                    return rc;
                continue;
            }
            k_stretch_propose<<<blocks, 128, 0, st>>>(ss, S->d_Y);
            S_TRY(cudaGetLastError());
            if (int rc = lens_eval(S->L, S->d_Y, half, S->d_lpY, st, S->d_kc)) return rc;
            k_stretch_accept<<<blocks, 128, 0, st>>>(ss, S->d_Y, S->d_lpY);
            S_TRY(cudaGetLastError());
        }
        if (chain)
            S_TRY(cudaMemcpyAsync(chain + (size_t)s * S->W * S->P, S->d_x,
                                  (size_t)S->W * S->P * sizeof(float), cudaMemcpyDeviceToDevice,
                                  st));
        if (lp_chain)
            S_TRY(cudaMemcpyAsync(lp_chain + (size_t)s * S->W, S->d_lp, (size_t)S->W * sizeof(double),
                                  cudaMemcpyDeviceToDevice, st));
        ++S->step;
        S->proposed += S->W;
    }
    return TLL_OK;
}

int tll_sampler_state(tll_sampler *S, float *x, double *lp, long long *step,
                      long long *accepted, long long *proposed, void *stream)
{
    if (!S) return set_error(TLL_EINVAL, "sampler is NULL");
    DevGuard g(S->dev);
    cudaStream_t st = (cudaStream_t)stream;
    if (x)
        S_TRY(cudaMemcpyAsync(x, S->d_x, (size_t)S->W * S->P * sizeof(float),
                              cudaMemcpyDeviceToDevice, st));
    if (lp)
        S_TRY(cudaMemcpyAsync(lp, S->d_lp, (size_t)S->W * sizeof(double), cudaMemcpyDeviceToDevice,
                              st));
    unsigned long long n = 0;
    S_TRY(cudaMemcpyAsync(&n, S->d_nacc, sizeof n, cudaMemcpyDeviceToHost, st));
    S_TRY(cudaStreamSynchronize(st));
    if (step) *step = S->step;
    if (accepted) *accepted = (long long)n;
    if (proposed) *proposed = S->proposed;
    return TLL_OK;
}

void tll_sampler_destroy(tll_sampler *S)
{
    if (!S) return;
    DevGuard g(S->dev);
    cudaDeviceSynchronize();
    sampler_free(S);
}

}  // extern "C"
