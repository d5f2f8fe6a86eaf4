// tll_split.cuh -- the split likelihood pipeline: the PSF convolution as its
// own kernel between a trace kernel and a sums kernel, with the binned and
// blurred images of a chunk of vectors in device memory.  It exists to run
// the convolution (Eq. 3) two ways on the same inputs:
//   direct   FP32 FMAs, one (vector, channel) image per CTA, the whole
//            zero-padded image in shared memory;
//   Toeplitz each PSF row's convolution as a GEMM with a banded Toeplitz
//            matrix on the tensor cores (tcgen05.mma kind::tf32, three TF32
//            products per term for FP32-level accuracy, accumulator in TMEM).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "tll_core.cuh"

namespace tll {

// Toeplitz tile geometry: an output tile is kTcM image rows x kTcN image
// columns; the input window is kTcKd columns (kTcN + K - 1 rounded up to the
// MMA's K step of 8) and kTcM + K - 1 rows.
constexpr int kTcM = 128, kTcN = 32, kTcKd = 64, kTcMaxK = kTcKd - kTcN + 1;
constexpr int kTcRows = kTcM + kTcMaxK - 1;       // staged input rows (allocated)

// Floats of the Toeplitz tiles for PSF side K: [K][2 parts][kTcKd/4][kTcN][4]
// (part 0: TF32-rounded values, part 1: the remainders), the exact
// shared-memory image of each tile.
inline size_t tc_tile_floats(int K) { return (size_t)K * 2 * kTcKd * kTcN; }

// Host: fill `out` (tc_tile_floats(K) floats) from the unit-sum PSF.
void build_tc_tiles(const float *psf, int K, float *out);

// Status codes the Toeplitz kernel writes (0: no error).
enum : int { TC_OK = 0, TC_TIMEOUT = 1 };

// Launchers (return the launch's cudaError_t).  Images are [nvec][2][npix]
// float32 (lens light, source), row-major, stride nx.
cudaError_t launch_trace_split(const LensDev &L, const float *kc, int nvec, float *unbl,
                               int grid, cudaStream_t st);
cudaError_t launch_conv_direct_split(const LensDev &L, const float *unbl, int nvec,
                                     float *blur, int grid, cudaStream_t st);
// The Toeplitz path first splits the images (unbl) into TF32 high and low
// parts, chunk-major, in hi / lo (tc_part_floats each), which the tensor
// maps mhi / mlo (make_tc_maps) describe; grid: one CTA per SM.
cudaError_t launch_conv_tc(const LensDev &L, const float *unbl, int nvec, float *hi,
                           float *lo, const CUtensorMap &mhi, const CUtensorMap &mlo,
                           float *blur, const float *tiles, int *status, int grid,
                           cudaStream_t st);
size_t tc_part_floats(int nimg, int ny, int nx);
// Host: the 4-D tensor maps (4 columns x rows x chunks x images) over the
// high and low parts; 0 on success.
int make_tc_maps(const float *hi, const float *lo, int nimg, int ny, int nx, int K,
                 CUtensorMap *mhi, CUtensorMap *mlo);
cudaError_t launch_sums_split(const LensDev &L, const float *kc, const float *blur,
                              int nvec, double *out, int grid, cudaStream_t st);

// The split-BF16 variant: the images as BF16 hi, mid and lo parts (three
// buffers of bf_part_bytes, chunk-major [image][8 columns][row][8]) under
// the tensor maps maps[0..2] (make_bf_maps); Toeplitz tiles of three BF16
// parts per PSF row (build_bf_tiles, bf_tile_elems 16-bit values).
void build_bf_tiles(const float *psf, int K, uint16_t *out);
size_t bf_tile_elems(int K);
size_t bf_part_bytes(int nimg, int ny, int nx);
int make_bf_maps(void *const *parts, int nimg, int ny, int nx, int K, CUtensorMap *maps);
cudaError_t launch_conv_bf(const LensDev &L, const float *unbl, int nvec, void *const *parts,
                           const CUtensorMap *maps, float *blur, const uint16_t *tiles,
                           int *status, int grid, cudaStream_t st);

// Shared memory the direct split kernel needs for one padded image (bytes),
// and the Toeplitz kernel's (constant per operand kind).
size_t conv_direct_split_smem(const LensDev &L);
size_t conv_tc_smem(bool bf);

}  // namespace tll
