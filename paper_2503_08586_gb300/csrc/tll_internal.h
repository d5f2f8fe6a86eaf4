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
int lens_nparam(const tll_lens *L);
int lens_device(const tll_lens *L);
// Set the calling thread's tll_last_error message; returns code.
int set_error(int code, const char *fmt, ...);
// Floats per vector of the constant-block scratch.
int const_block_floats();

}  // namespace tll
