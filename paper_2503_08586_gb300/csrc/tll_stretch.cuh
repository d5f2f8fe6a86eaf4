// tll_stretch.cuh -- the stretch move's per-walker steps (device), shared by
// the sampler's own kernels and by the likelihood kernel's fused sampler
// step (proposal before the decode, accept / reject after the log L).
//
// One step updates half 0 (walkers [0, W/2)) and then half 1 ([W/2, W)).
// For walker k of half h, with the Philox4x32-10 outputs r0..r3 (Salmon et
// al. 2011) at key (seed low, seed high) and counter (k, h, step low, step
// high):
//   partner  j = (first walker of the other half) + floor(r0 (W/2) / 2^32)
//   stretch  u = (r1 + 1/2) 2^-32, z = ((a - 1) u + 1)^2 / a  (density
//            ~ 1/sqrt(z) on [1/a, a])  (Goodman & Weare 2010)
//   proposal Y = x_j + z (x_k - x_j) in FP64, one rounding per operation,
//            then to float32
//   accept   when log((r2 + 1/2) 2^-32) < (ndim - 1) log z + lp(Y) - lp(x_k),
//            lp(Y) = log L(Y) inside the box prior [lo, hi] (coordinates with
//            lo == hi are fixed), -inf outside.
#pragma once

#include <stdint.h>

namespace tll {

// One half step of the sampler: the walkers x [W][P] and their log
// posteriors lp [W] (updated in place), the prior box, the optional
// proposals' log posteriors lp_prop [W] and the accept counter.
struct StretchStep {
    float *x;
    double *lp;
    double *lp_prop;               // or null
    unsigned long long *nacc;
    const float *lo, *hi;
    long long step;
    unsigned long long seed;
    double a;
    int W, P, h, ndim;
};

// Philox4x32-10: ten rounds; in each, the 32 x 32 -> 64-bit products of
// counter words 0 and 2 with the round multipliers are split into high and
// low halves and mixed with words 1, 3 and the key; the key advances by the
// Weyl constants between rounds.
__device__ __forceinline__ void philox10(uint32_t c[4], uint32_t k0, uint32_t k1)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        const uint32_t lo0 = 0xD2511F53u * c[0], hi0 = __umulhi(0xD2511F53u, c[0]);
        const uint32_t lo1 = 0xCD9E8D57u * c[2], hi1 = __umulhi(0xCD9E8D57u, c[2]);
        const uint32_t n0 = hi1 ^ c[1] ^ k0, n2 = hi0 ^ c[3] ^ k1;
        c[0] = n0;
        c[1] = lo1;
        c[2] = n2;
        c[3] = lo0;
    }
}

__device__ __forceinline__ void walker_draws(unsigned long long seed, long long step, int h,
                                             int k, uint32_t r[4])
{
    r[0] = (uint32_t)k;
    r[1] = (uint32_t)h;
    r[2] = (uint32_t)((unsigned long long)step & 0xffffffffull);
    r[3] = (uint32_t)((unsigned long long)step >> 32);
    philox10(r, (uint32_t)(seed & 0xffffffffull), (uint32_t)(seed >> 32));
}

__device__ __forceinline__ double unit_open(uint32_t v)
{
    return __dmul_rn(__dadd_rn((double)v, 0.5), 2.3283064365386963e-10);
}

// Walker k = h W/2 + t of the step: its draws, partner j and stretch z.
__device__ __forceinline__ void stretch_draw(const StretchStep &s, int t, uint32_t r[4], int &k,
                                             int &j, double &z)
{
    const int half = s.W / 2;
    k = s.h * half + t;
    walker_draws(s.seed, s.step, s.h, k, r);
    j = (1 - s.h) * half + (int)(((unsigned long long)r[0] * (unsigned long long)half) >> 32);
    const double w = __dadd_rn(__dmul_rn(__dsub_rn(s.a, 1.0), unit_open(r[1])), 1.0);
    z = __ddiv_rn(__dmul_rn(w, w), s.a);
}

// Proposal entries i = i0, i0 + di, ... of walker t (y: its row, P floats).
__device__ __forceinline__ void stretch_propose_entries(const StretchStep &s, int t, int i0,
                                                        int di, float *y, double *z_out)
{
    uint32_t r[4];
    int k, j;
    double z;
    stretch_draw(s, t, r, k, j, z);
    const float *xk = s.x + (size_t)k * s.P, *xj = s.x + (size_t)j * s.P;
    for (int i = i0; i < s.P; i += di) {
        const double dj = (double)xj[i];
        y[i] = __double2float_rn(__dadd_rn(dj, __dmul_rn(z, __dsub_rn((double)xk[i], dj))));
    }
    if (z_out) *z_out = z;
}

// Box prior: -inf outside [lo, hi] on a free coordinate (lo < hi).
__device__ __forceinline__ bool in_box(const float *v, const float *lo, const float *hi, int P)
{
    bool ok = true;
    for (int i = 0; i < P; ++i)
        if (lo[i] < hi[i] && !(v[i] >= lo[i] && v[i] <= hi[i])) ok = false;
    return ok;
}

// Accept / reject walker t given its proposal y and the proposal's log L.
__device__ __forceinline__ void stretch_accept_one(const StretchStep &s, int t, const float *y,
                                                   double lpY)
{
    uint32_t r[4];
    int k, j;
    double z;
    stretch_draw(s, t, r, k, j, z);
    const double lpy = in_box(y, s.lo, s.hi, s.P) ? lpY : -INFINITY;
    const double lu = log(unit_open(r[2]));
    const double rhs = __dsub_rn(__dadd_rn(__dmul_rn((double)(s.ndim - 1), log(z)), lpy), s.lp[k]);
    if (s.lp_prop) s.lp_prop[k] = lpy;
    if (lu < rhs) {
        for (int i = 0; i < s.P; ++i) s.x[(size_t)k * s.P + i] = y[i];
        s.lp[k] = lpy;
        atomicAdd(s.nacc, 1ull);
    }
}

}  // namespace tll
