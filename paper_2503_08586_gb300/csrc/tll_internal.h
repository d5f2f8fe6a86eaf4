// tll_internal.h -- entry points of tll.cu used by the library's other
// translation units (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>

#include "tll.h"

namespace tll {

// log L of B vectors (device params [B][nparam]) into out (device [B]) on
// stream st, through the lens's own batched path (two-column or
// multi-column), with the caller's constant-block scratch kc (device,
// NCONST floats per vector).  The lens's per-CTA image slots must exist
// (lens_prepare).
int lens_eval(tll_lens *L, const float *params, int B, double *out, cudaStream_t st, float *kc);
// Allocate what lens_eval needs besides kc (the one-lens image slots).
int lens_prepare(tll_lens *L);
struct StretchStep;   // tll_stretch.cuh
// Whether lens_eval_stretch applies to B vectors: a two-column lens on the
// fused convolution path whose batch fits the likelihood kernel's grid
// (each CTA one vector, decoded by the kernel itself).
bool lens_eval_fuses(const tll_lens *L, int B);
// lens_eval with a stretch-move half step fused into the likelihood launch:
// CTA b writes walker b's proposal into params row b (device [B][nparam]),
// its log L into out[b], then takes its accept / reject (ss).  TLL_EINVAL
// where lens_eval_fuses does not hold.
int lens_eval_stretch(tll_lens *L, float *params, int B, double *out, cudaStream_t st,
                      float *kc, const StretchStep &ss);
int lens_nparam(const tll_lens *L);
int lens_device(const tll_lens *L);
// Set the calling thread's tll_last_error message; returns code.
int set_error(int code, const char *fmt, ...);
// Floats per vector of the constant-block scratch.
int const_block_floats();

}  // namespace tll
