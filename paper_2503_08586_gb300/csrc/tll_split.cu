// tll_split.cu -- kernels of the split likelihood pipeline (trace, the
// convolution two ways, sums), see tll_split.cuh.
#include <cuda.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>

#include "tll_kernels.cuh"
#include "tll_split.cuh"

namespace tll {
namespace {

// ---------------------------------------------------------------- trace
// Persistent CTAs, one vector at a time: the binned lens and source images
// of vector b go to unbl[b][0][.] and unbl[b][1][.] (invalid vectors are
// skipped; the sums kernel gives them -inf).
template <int SUB>
__global__ void __launch_bounds__(kThreads)
k_trace_split(const __grid_constant__ LensDev L, const float *__restrict__ kc, int nvec,
              float *__restrict__ unbl)
{
    __shared__ __align__(16) float sepl[kEplSmemFloats];
    const int tid = threadIdx.x, nthr = blockDim.x;
    for (int b = blockIdx.x; b < nvec; b += gridDim.x) {
        const float *k = kc + (size_t)b * NCONST;
        if (k[K_VALID] == 0.0f) continue;
        float *Il = unbl + (size_t)b * 2 * L.npix, *Is = Il + L.npix;
        trace_vector<SUB>(L, k, Il, Is, L.nx, 0, sepl, tid, nthr, false);
    }
}

// ------------------------------------------------- direct convolution
// One (vector, channel) image per CTA at a time, the whole image zero-padded
// in shared memory (image pixel (i, j) at (h + i) W + HL + j; rows h above
// and below and the columns outside [HL, HL + nx) stay zero).  K > 0:
// compiled for side K (a thread makes 4 adjacent outputs of a row from one
// float4 window per PSF row, taps from the parameter block); K == 0: any
// side, scalar loads.  m(i,j) = sum_{r,c} P[r][c] I(i+h-r, j+h-c) (Eq. 3).
template <int K>
__global__ void __launch_bounds__(kThreads)
k_conv_direct_split(const __grid_constant__ LensDev L, const float *__restrict__ unbl, int nvec,
                    float *__restrict__ blur)
{
    extern __shared__ __align__(16) float P[];
    const int tid = threadIdx.x, nthr = blockDim.x;
    const int Kr = K > 0 ? K : L.K, h = (Kr - 1) / 2;
    const int nx = L.nx, ny = L.ny, npix = L.npix, W = L.W, HL = L.HL;
    const int rows = ny + 2 * h;
    for (int t = tid; t < rows * W; t += nthr) P[t] = 0.0f;
    __syncthreads();
    for (int item = blockIdx.x; item < 2 * nvec; item += gridDim.x) {
        const float *src = unbl + (size_t)item * npix;
        float *dst = blur + (size_t)item * npix;
        for (int t = tid; t < npix; t += nthr) {
            const int i = t / nx, j = t - i * nx;
            P[(h + i) * W + HL + j] = src[t];
        }
        __syncthreads();
        if constexpr (K > 0) {
            using G = PadGeom<K>;
            const int ngroups = (nx + 3) >> 2;
            for (int it = tid; it < ny * ngroups; it += nthr) {
                const int i = it / ngroups, g = it - i * ngroups;
                float o0 = 0.0f, o1 = 0.0f, o2 = 0.0f, o3 = 0.0f;
#pragma unroll 1
                for (int r = 0; r < K; ++r) {
                    // PSF row r meets image row i + h - r = buffer row i + 2h - r
                    const float4 *w4 = reinterpret_cast<const float4 *>(P + (i + 2 * G::h - r) * W + 4 * g);
                    float win[4 * G::NW];
#pragma unroll
                    for (int q = 0; q < G::NW; ++q) {
                        const float4 v4 = w4[q];
                        win[4 * q] = v4.x; win[4 * q + 1] = v4.y;
                        win[4 * q + 2] = v4.z; win[4 * q + 3] = v4.w;
                    }
                    const float *tr = L.tk + r * tap_stride(K);
                    float a0 = 0.0f, a1 = 0.0f, a2 = 0.0f, a3 = 0.0f;
#pragma unroll
                    for (int c = 0; c < K; ++c) {
                        const float t = tr[c];
                        a0 = fmaf(t, win[G::D + K - 1 - c], a0);
                        a1 = fmaf(t, win[G::D + K - c], a1);
                        a2 = fmaf(t, win[G::D + K + 1 - c], a2);
                        a3 = fmaf(t, win[G::D + K + 2 - c], a3);
                    }
                    o0 += a0; o1 += a1; o2 += a2; o3 += a3;
                }
                const float o[4] = {o0, o1, o2, o3};
#pragma unroll
                for (int q = 0; q < 4; ++q)
                    if (4 * g + q < nx) dst[i * nx + 4 * g + q] = o[q];
            }
        } else {
            for (int t = tid; t < npix; t += nthr) {
                const int i = t / nx, j = t - i * nx;
                float m = 0.0f;
                for (int r = 0; r < Kr; ++r) {
                    const float *row = P + (i + 2 * h - r) * W + HL + j + h;
                    const float *tr = L.psf + r * Kr;
                    float a = 0.0f;
                    for (int c = 0; c < Kr; ++c) a = fmaf(tr[c], row[-c], a);
                    m += a;
                }
                dst[t] = m;
            }
        }
        __syncthreads();
    }
}

// ----------------------------------------------------------------- sums
// Persistent CTAs, one vector at a time: the five weighted sums over the
// blurred images, then the amplitudes and log L (as in the fused kernel).
__global__ void __launch_bounds__(kThreads)
k_sums_split(const __grid_constant__ LensDev L, const float *__restrict__ kc,
             const float *__restrict__ blur, int nvec, double *__restrict__ out)
{
    __shared__ float2 sred[32 * 5];
    const int tid = threadIdx.x, nthr = blockDim.x;
    const int lane = tid & 31, warp = tid >> 5, nwarp = nthr >> 5;
    for (int b = blockIdx.x; b < nvec; b += gridDim.x) {
        const float *k = kc + (size_t)b * NCONST;
        if (k[K_VALID] == 0.0f) {
            if (tid == 0) out[b] = -INFINITY;
            continue;
        }
        const float *bl = blur + (size_t)b * 2 * L.npix, *bs = bl + L.npix;
        float acc[10];
#pragma unroll
        for (int q = 0; q < 10; ++q) acc[q] = 0.0f;
        for (int t = tid; t < L.npix; t += nthr) accum_pixel(bl[t], bs[t], L.wpack[t], acc);
        warp_sums(acc, sred, lane, warp, false);
        __syncthreads();
        if (warp == 0) {
            double S[5];
            block_sums(sred, nwarp, lane, S);
            if (lane == 0) {
                double sl, ss, ll;
                finish_vector(L, S, k[K_IEL], k[K_IES], &sl, &ss, &ll);
                out[b] = ll;
            }
        }
        __syncthreads();
    }
}

// ------------------------------------------ Toeplitz convolution (tcgen05)
// For PSF row r, an output tile's rows i0 .. i0+127 and columns
// j0 .. j0+31 get
//   D[m][n] += sum_k A_r[m][k] T_r[k][n],
//   A_r[m][k] = I(i0 + m + h - r, j0 - o + k),  T_r[k][n] = P[r][n + h + o - k]
// (o = h rounded up to a multiple of 4, so the window starts on a 16-byte
// chunk; T_r is zero where the PSF index leaves [0, K)): K GEMMs of
// 128 x 32 x 64 per tile, each as 8 tcgen05.mma steps of K = 8.  Accuracy:
// three TF32 products per term, A_hi B_hi + A_hi B_lo + A_lo B_hi (x = x_hi +
// x_lo, x_hi rounded to TF32).  The tensor core's FP32 accumulation rounds
// toward zero (measured: -7.5e-6 relative, a bias, over one accumulator of 31
// rows), so each PSF row accumulates into a fresh TMEM accumulator -- two,
// used alternately -- and the rows' partial products are added in registers
// (round to nearest) while the next row's MMAs run.
//
// Data movement: the images are split into TF32 high and low parts and
// stored chunk-major -- [image][16-byte chunk of 4 columns][row][4] -- by
// k_tf32_split, so one 4-D TMA box (4 x rows x 16 chunks x 1) lands in shared
// memory in the canonical K-major no-swizzle layout; A_r for any r is then
// the same matrix with its start moved by 2h - r rows (16 bytes each).  Rows
// and chunks outside the image arrive as zeros (TMA fill).  The Toeplitz
// tiles of all PSF rows are in global memory (L2-resident) and stream
// through a 3-stage ring by bulk copies.
// Roles (192 threads): warps 0-3 drain the accumulators (TMEM lanes
// 32w .. 32w+31) and write the outputs, warp 4 issues the copies, warp 5
// issues the MMAs; mbarriers order them, every wait is bounded.
__device__ __forceinline__ uint32_t smem_u32(const void *p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

// Shared-memory matrix descriptor (tcgen05): start address, leading byte
// offset (between core matrices along K), stride byte offset (between 8-row
// groups), the fixed 0b001 at bits 46-48, no swizzle.
__device__ __forceinline__ uint64_t tc_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo)
{
    return (uint64_t)((saddr & 0x3FFFF) >> 4) | ((uint64_t)((lbo & 0x3FFFF) >> 4) << 16) |
           ((uint64_t)((sbo & 0x3FFFF) >> 4) << 32) | ((uint64_t)1 << 46);
}

// The two operand kinds of the Toeplitz GEMM.
//  TF32: x = hi + lo, hi the TF32 rounding of x (lo exact in FP32); the
//   products hi*hi + hi*lo + lo*hi; tcgen05.mma kind::tf32, K = 8 per step.
//  BF16: x = hi + mid + lo, each the BF16 rounding of what the earlier parts
//   leave (24 mantissa bits in all, so x exactly for FP32 x); the products
//   hi*hi + hi*mid + mid*hi + hi*lo + mid*mid + lo*hi -- every term down to
//   2^-24 relative, the dropped ones (mid*lo, lo*mid, lo*lo) below 2^-32;
//   tcgen05.mma kind::f16 with both operands BF16, K = 16 per step.
// Either way a 16-byte chunk holds kChunk consecutive columns of a row and
// an MMA step spans two chunks, so the shared-memory layouts and matrix
// descriptors are the same.  Instruction descriptor: D F32 (bit 4), A and B
// formats (bits 7, 10: TF32 2 under kind::tf32, BF16 1 under kind::f16),
// both K-major, N >> 3 at bit 17, M >> 4 at bit 24.
template <bool BF>
struct TcKind {
    static constexpr int kParts = BF ? 3 : 2, kElem = BF ? 2 : 4, kChunk = 16 / kElem;
    static constexpr int kProducts = BF ? 6 : 3;
    static constexpr int kChunks = kTcKd / kChunk;       // chunks of the window
    static constexpr int kSteps = kTcKd / (2 * kChunk);  // MMA steps per PSF row
    static constexpr int kPartTileBytes = kTcKd * kTcN * kElem;
    static constexpr int kTileBytes = kParts * kPartTileBytes;   // one PSF row
    static constexpr int kABytes = kChunks * kTcRows * 16;       // one part of one A buffer
    static constexpr uint32_t kIdesc = (1u << 4) | ((BF ? 1u : 2u) << 7) | ((BF ? 1u : 2u) << 10) |
                                       ((uint32_t)(kTcN >> 3) << 17) |
                                       ((uint32_t)(kTcM >> 4) << 24);
    // parts of A and B in product p
    __host__ __device__ static constexpr int apart(int p)
    {
        return BF ? (p == 2 || p == 4 ? 1 : p == 5 ? 2 : 0) : (p == 2 ? 1 : 0);
    }
    __host__ __device__ static constexpr int bpart(int p)
    {
        return BF ? (p == 1 || p == 4 ? 1 : p == 3 ? 2 : 0) : (p == 1 ? 1 : 0);
    }
};

constexpr int kTcStages = 3;                      // Toeplitz ring
constexpr int kTcNCol = 2 * kTcN;                 // TMEM columns: two accumulators
constexpr uint32_t kTcSpin = 1u << 22;            // wait limit (iterations)

// Wait for phase `parity` of an mbarrier; false (and the abort flag set)
// when the limit runs out or another role aborted.
__device__ __forceinline__ bool tc_wait(uint32_t mbar, uint32_t parity, volatile int *abort)
{
    for (uint32_t it = 0; it < kTcSpin; ++it) {
        uint32_t done;
        asm volatile("{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
                     "selp.u32 %0, 1, 0, p;\n}"
                     : "=r"(done) : "r"(mbar), "r"(parity) : "memory");
        if (done) return true;
        if ((it & 255u) == 255u && *abort) return false;
    }
    *abort = 1;
    return false;
}

__device__ __forceinline__ void mbar_init(uint64_t *m, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" :: "r"(smem_u32(m)), "r"(count));
}
__device__ __forceinline__ void mbar_arrive(uint64_t *m)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" :: "r"(smem_u32(m)) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t *m, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;"
                 :: "r"(smem_u32(m)), "r"(bytes) : "memory");
}
__device__ __forceinline__ void tc_commit(uint64_t *m)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                 :: "r"(smem_u32(m)) : "memory");
}

// out[c] += accumulator column c of this thread's TMEM lane (32 columns).
__device__ __forceinline__ void tmem_add32(uint32_t taddr, float *out)
{
    uint32_t v[32];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x32.b32 "
                 "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
                 "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
                 : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]),
                   "=r"(v[6]), "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]),
                   "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]), "=r"(v[16]),
                   "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]),
                   "=r"(v[22]), "=r"(v[23]), "=r"(v[24]), "=r"(v[25]), "=r"(v[26]),
                   "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
                 : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int c = 0; c < 32; ++c) out[c] += __uint_as_float(v[c]);
}

__device__ __forceinline__ float to_tf32(float x)
{
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return __uint_as_float(r);
}

// Images (row-major, nimg of ny x nx) -> TF32 high and low parts,
// chunk-major [image][chunk][row][4], columns past nx as zeros.
__global__ void k_tf32_split(const float *__restrict__ unbl, int nimg, int ny, int nx, int nch,
                             float4 *__restrict__ hi, float4 *__restrict__ lo)
{
    const long long n = (long long)nimg * nch * ny;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n;
         t += (long long)gridDim.x * blockDim.x) {
        const int row = (int)(t % ny);
        const long long q = t / ny;
        const int ch = (int)(q % nch);
        const long long img = q / nch;
        const float *src = unbl + (img * ny + row) * nx + 4 * ch;
        float v[4], h4[4], l4[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            v[k] = (4 * ch + k < nx) ? src[k] : 0.0f;
            h4[k] = to_tf32(v[k]);
            l4[k] = v[k] - h4[k];
        }
        hi[t] = make_float4(h4[0], h4[1], h4[2], h4[3]);
        lo[t] = make_float4(l4[0], l4[1], l4[2], l4[3]);
    }
}

// BF16 bits of x rounded to nearest, ties to even (finite x).
__host__ __device__ __forceinline__ uint32_t bf16_bits(float x)
{
#ifdef __CUDA_ARCH__
    const uint32_t u = __float_as_uint(x);
#else
    uint32_t u;
    memcpy(&u, &x, 4);
#endif
    return (u + 0x7fffu + ((u >> 16) & 1u)) >> 16;
}
__host__ __device__ __forceinline__ float bf16_value(uint32_t b)
{
#ifdef __CUDA_ARCH__
    return __uint_as_float(b << 16);
#else
    const uint32_t u = b << 16;
    float y;
    memcpy(&y, &u, 4);
    return y;
#endif
}
// x as hi + mid + lo BF16 parts (bits).
__host__ __device__ __forceinline__ void bf16_split3(float x, uint32_t *p)
{
    p[0] = bf16_bits(x);
    const float r1 = x - bf16_value(p[0]);
    p[1] = bf16_bits(r1);
    p[2] = bf16_bits(r1 - bf16_value(p[1]));
}

// Images (row-major, nimg of ny x nx) -> BF16 hi, mid and lo parts,
// chunk-major [image][chunk of 8 columns][row][8], columns past nx as zeros.
__global__ void k_bf16_split(const float *__restrict__ unbl, int nimg, int ny, int nx, int nch,
                             uint4 *__restrict__ p0, uint4 *__restrict__ p1,
                             uint4 *__restrict__ p2)
{
    const long long n = (long long)nimg * nch * ny;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n;
         t += (long long)gridDim.x * blockDim.x) {
        const int row = (int)(t % ny);
        const long long q = t / ny;
        const int ch = (int)(q % nch);
        const long long img = q / nch;
        const float *src = unbl + (img * ny + row) * nx + 8 * ch;
        uint32_t w[3][4] = {};
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            uint32_t b[3];
            bf16_split3((8 * ch + k < nx) ? src[k] : 0.0f, b);
#pragma unroll
            for (int part = 0; part < 3; ++part) w[part][k >> 1] |= b[part] << (16 * (k & 1));
        }
        p0[t] = make_uint4(w[0][0], w[0][1], w[0][2], w[0][3]);
        p1[t] = make_uint4(w[1][0], w[1][1], w[1][2], w[1][3]);
        p2[t] = make_uint4(w[2][0], w[2][1], w[2][2], w[2][3]);
    }
}

template <bool BF>
__global__ void __launch_bounds__(192, 1)
k_conv_tc(const __grid_constant__ LensDev L, const __grid_constant__ CUtensorMap tm0,
          const __grid_constant__ CUtensorMap tm1, const __grid_constant__ CUtensorMap tm2,
          int nimg, float *__restrict__ blur, const unsigned char *__restrict__ tiles,
          int *status)
{
    using KD = TcKind<BF>;
    extern __shared__ __align__(1024) unsigned char dsm[];
    // A: [2 buffers][kParts][kABytes], B: [kTcStages][kTileBytes]
    unsigned char *sA = dsm;
    unsigned char *sB = dsm + 2 * KD::kParts * KD::kABytes;
    __shared__ __align__(8) uint64_t a_full[2], a_empty[2], b_full[kTcStages],
        b_empty[kTcStages], acc_full[2], acc_empty[2], drained;
    __shared__ uint32_t tmem_base;
    __shared__ volatile int abort_flag;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int K = L.K, h = (K - 1) / 2, o = (h + KD::kChunk - 1) & ~(KD::kChunk - 1);
    const int nx = L.nx, ny = L.ny, npix = L.npix;
    const int nrb = (ny + kTcM - 1) / kTcM, ncb = (nx + kTcN - 1) / kTcN;
    const long long items = (long long)nimg * nrb * ncb;
    const int arows = kTcM + K - 1;                       // rows of the TMA box
    const uint32_t abox = (uint32_t)(KD::kChunks * arows * 16);
    if (tid == 0) {
        abort_flag = 0;
        for (int q = 0; q < 2; ++q) {
            mbar_init(&a_full[q], 1); mbar_init(&a_empty[q], 1);
            mbar_init(&acc_full[q], 1); mbar_init(&acc_empty[q], 4);
        }
        for (int q = 0; q < kTcStages; ++q) { mbar_init(&b_full[q], 1); mbar_init(&b_empty[q], 1); }
        mbar_init(&drained, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     :: "r"(smem_u32(&tmem_base)), "r"(kTcNCol));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_base;

    if (warp == 4) {
        // ---------------- copies: A window per tile, Toeplitz tiles per PSF row
        if (lane == 0) {
            uint32_t ae_par[2] = {1u, 1u}, be_par[kTcStages];
            int a_iss[2] = {0, 0}, b_iss[kTcStages];
            for (int q = 0; q < kTcStages; ++q) { be_par[q] = 1u; b_iss[q] = 0; }
            int ab = 0, st = 0;
            bool ok = true;
            for (long long item = blockIdx.x; item < items && ok; item += gridDim.x) {
                const int cb = (int)(item % ncb);
                const long long rest = item / ncb;
                const int rb = (int)(rest % nrb);
                const int img = (int)(rest / nrb);
                if (!(ok = tc_wait(smem_u32(&a_empty[ab]), ae_par[ab], &abort_flag))) break;
                ae_par[ab] ^= 1u;
                mbar_expect_tx(&a_full[ab], KD::kParts * abox);
                // innermost coordinate 0 (16-byte aligned); the chunk and row
                // coordinates may leave the image (zero fill)
                const int c0 = 0, c1 = rb * kTcM - h, c2 = (cb * kTcN - o) / KD::kChunk, c3 = img;
                for (int part = 0; part < KD::kParts; ++part) {
                    const uint32_t dst = smem_u32(sA + (KD::kParts * ab + part) * KD::kABytes);
                    const CUtensorMap *tm = part == 0 ? &tm0 : part == 1 ? &tm1 : &tm2;
                    asm volatile(
                        "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
                        " [%0], [%1, {%2, %3, %4, %5}], [%6];"
                        :: "r"(dst), "l"(tm), "r"(c0), "r"(c1), "r"(c2), "r"(c3),
                           "r"(smem_u32(&a_full[ab])) : "memory");
                }
                ++a_iss[ab];
                ab ^= 1;
                for (int r = 0; r < K; ++r) {
                    if (!(ok = tc_wait(smem_u32(&b_empty[st]), be_par[st], &abort_flag))) break;
                    be_par[st] ^= 1u;
                    mbar_expect_tx(&b_full[st], KD::kTileBytes);
                    asm volatile(
                        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes"
                        " [%0], [%1], %2, [%3];"
                        :: "r"(smem_u32(sB + st * KD::kTileBytes)),
                           "l"(tiles + (size_t)r * KD::kTileBytes), "r"(KD::kTileBytes),
                           "r"(smem_u32(&b_full[st])) : "memory");
                    ++b_iss[st];
                    st = (st + 1) % kTcStages;
                }
            }
            if (!ok) {
                // let issued copies land before the CTA's shared memory goes
                for (int q = 0; q < 2; ++q)
                    if (a_iss[q]) tc_wait(smem_u32(&a_full[q]), (uint32_t)(a_iss[q] - 1) & 1u, &abort_flag);
                for (int q = 0; q < kTcStages; ++q)
                    if (b_iss[q]) tc_wait(smem_u32(&b_full[q]), (uint32_t)(b_iss[q] - 1) & 1u, &abort_flag);
            }
        }
    } else if (warp == 5) {
        // ---------------- MMA issue
        if (lane == 0) {
            uint32_t af_par[2] = {0u, 0u}, bf_par[kTcStages], ce_par[2] = {1u, 1u};
            for (int q = 0; q < kTcStages; ++q) bf_par[q] = 0u;
            int ab = 0, st = 0;
            bool ok = true;
            const uint32_t lbo_a = (uint32_t)arows * 16u;
            for (long long item = blockIdx.x; item < items && ok; item += gridDim.x) {
                if (!(ok = tc_wait(smem_u32(&a_full[ab]), af_par[ab], &abort_flag))) break;
                af_par[ab] ^= 1u;
                uint32_t a_part[KD::kParts];
#pragma unroll
                for (int part = 0; part < KD::kParts; ++part)
                    a_part[part] = smem_u32(sA + (KD::kParts * ab + part) * KD::kABytes);
                for (int r = 0; r < K; ++r) {
                    const int acc = r & 1;
                    if (!(ok = tc_wait(smem_u32(&b_full[st]), bf_par[st], &abort_flag))) break;
                    bf_par[st] ^= 1u;
                    if (!(ok = tc_wait(smem_u32(&acc_empty[acc]), ce_par[acc], &abort_flag))) break;
                    ce_par[acc] ^= 1u;
                    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                    const uint32_t rowoff = 16u * (uint32_t)(2 * h - r);
                    const uint32_t b_base = smem_u32(sB + st * KD::kTileBytes);
                    const uint32_t d = tmem + (uint32_t)(acc * kTcN);
#pragma unroll 1
                    for (int ks = 0; ks < KD::kSteps; ++ks) {
                        const uint32_t ao = (uint32_t)(2 * ks) * lbo_a + rowoff;
                        const uint32_t bo = (uint32_t)(2 * ks * kTcN * 16);
#pragma unroll
                        for (int term = 0; term < KD::kProducts; ++term) {
                            const uint64_t ad = tc_desc(a_part[KD::apart(term)] + ao, lbo_a, 128);
                            const uint64_t bd =
                                tc_desc(b_base + (uint32_t)(KD::bpart(term) * KD::kPartTileBytes) + bo,
                                        kTcN * 16, 128);
                            const uint32_t accum = (ks > 0 || term > 0) ? 1u : 0u;
                            if constexpr (BF)
                                asm volatile("{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
                                             "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}"
                                             :: "r"(d), "l"(ad), "l"(bd), "r"(KD::kIdesc), "r"(accum)
                                             : "memory");
                            else
                                asm volatile("{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
                                             "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}"
                                             :: "r"(d), "l"(ad), "l"(bd), "r"(KD::kIdesc), "r"(accum)
                                             : "memory");
                        }
                    }
                    tc_commit(&b_empty[st]);
                    tc_commit(&acc_full[acc]);
                    st = (st + 1) % kTcStages;
                }
                if (!ok) break;
                tc_commit(&a_empty[ab]);
                ab ^= 1;
            }
            // every MMA this thread issued has finished once `drained` completes
            tc_commit(&drained);
            tc_wait(smem_u32(&drained), 0u, &abort_flag);
        }
    } else {
        // ---------------- accumulators -> registers -> outputs (warps 0-3)
        uint32_t cf_par[2] = {0u, 0u};
        const uint32_t lane_base = tmem + ((uint32_t)(warp * 32) << 16);
        bool ok = true;
        for (long long item = blockIdx.x; item < items && ok; item += gridDim.x) {
            const int cb = (int)(item % ncb);
            const long long rest = item / ncb;
            const int rb = (int)(rest % nrb);
            const long long img = rest / nrb;
            float acc[32];
#pragma unroll
            for (int c = 0; c < 32; ++c) acc[c] = 0.0f;
            for (int r = 0; r < K; ++r) {
                const int a = r & 1;
                if (!(ok = tc_wait(smem_u32(&acc_full[a]), cf_par[a], &abort_flag))) break;
                cf_par[a] ^= 1u;
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                tmem_add32(lane_base + (uint32_t)(a * kTcN), acc);
                asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
                __syncwarp();
                if (lane == 0) mbar_arrive(&acc_empty[a]);
            }
            if (!ok) break;
            const int row = rb * kTcM + warp * 32 + lane, j0 = cb * kTcN;
            if (row < ny) {
                float *dst = blur + img * npix + (size_t)row * nx;
#pragma unroll
                for (int c = 0; c < 32; ++c)
                    if (j0 + c < nx) dst[j0 + c] = acc[c];
            }
        }
    }
    __syncthreads();
    if (tid == 0 && abort_flag) atomicExch(status, TC_TIMEOUT);
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;"
                     :: "r"(tmem), "r"(kTcNCol));
}

// Round to TF32 (10 explicit mantissa bits), ties to even, on the host.
float host_tf32(float x)
{
    uint32_t u;
    memcpy(&u, &x, 4);
    if ((u & 0x7f800000u) == 0x7f800000u) return x;
    u += 0xfffu + ((u >> 13) & 1u);
    u &= ~0x1fffu;
    float y;
    memcpy(&y, &u, 4);
    return y;
}

}  // namespace

void build_tc_tiles(const float *psf, int K, float *out)
{
    const int h = (K - 1) / 2, o = (h + 3) & ~3;
    for (int r = 0; r < K; ++r)
        for (int part = 0; part < 2; ++part)
            for (int kc = 0; kc < kTcKd / 4; ++kc)
                for (int n = 0; n < kTcN; ++n)
                    for (int kk = 0; kk < 4; ++kk) {
                        const int k = 4 * kc + kk, c = n + h + o - k;
                        const float v = (c >= 0 && c < K) ? psf[r * K + c] : 0.0f;
                        const float hi = host_tf32(v);
                        out[((((size_t)r * 2 + part) * (kTcKd / 4) + kc) * kTcN + n) * 4 + kk] =
                            part ? v - hi : hi;
                    }
}

size_t conv_direct_split_smem(const LensDev &L)
{
    return (size_t)(L.ny + 2 * L.h) * L.W * sizeof(float);
}

void build_bf_tiles(const float *psf, int K, uint16_t *out)
{
    using KD = TcKind<true>;
    const int h = (K - 1) / 2, o = (h + KD::kChunk - 1) & ~(KD::kChunk - 1);
    for (int r = 0; r < K; ++r)
        for (int kc = 0; kc < KD::kChunks; ++kc)
            for (int n = 0; n < kTcN; ++n)
                for (int kk = 0; kk < KD::kChunk; ++kk) {
                    const int k = KD::kChunk * kc + kk, c = n + h + o - k;
                    uint32_t b[3];
                    bf16_split3((c >= 0 && c < K) ? psf[r * K + c] : 0.0f, b);
                    for (int part = 0; part < 3; ++part)
                        out[(((((size_t)r * 3 + part) * KD::kChunks + kc) * kTcN + n) *
                              KD::kChunk) + kk] = (uint16_t)b[part];
                }
}

size_t bf_tile_elems(int K) { return (size_t)K * TcKind<true>::kTileBytes / 2; }

size_t conv_tc_smem(bool bf)
{
    return bf ? (size_t)2 * TcKind<true>::kParts * TcKind<true>::kABytes +
                    (size_t)kTcStages * TcKind<true>::kTileBytes
              : (size_t)2 * TcKind<false>::kParts * TcKind<false>::kABytes +
                    (size_t)kTcStages * TcKind<false>::kTileBytes;
}

size_t bf_part_bytes(int nimg, int ny, int nx)
{
    return (size_t)nimg * ((nx + 7) / 8) * ny * 16;
}

size_t tc_part_floats(int nimg, int ny, int nx)
{
    return (size_t)nimg * ((nx + 3) / 4) * ny * 4;
}

namespace {
using EncodeFn = CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *,
                              const cuuint64_t *, const cuuint64_t *, const cuuint32_t *,
                              const cuuint32_t *, CUtensorMapInterleave, CUtensorMapSwizzle,
                              CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
EncodeFn tensor_map_encoder()
{
    static EncodeFn encode = nullptr;
    if (!encode) {
        void *fn = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000,
                                             cudaEnableDefault, &q) != cudaSuccess ||
            q != cudaDriverEntryPointSuccess || !fn)
            return nullptr;
        encode = reinterpret_cast<EncodeFn>(fn);
    }
    return encode;
}
}  // namespace

int make_bf_maps(void *const *parts, int nimg, int ny, int nx, int K, CUtensorMap *maps)
{
    const EncodeFn encode = tensor_map_encoder();
    if (!encode) return 1;
    using KD = TcKind<true>;
    const int nch = (nx + 7) / 8;
    const cuuint64_t dims[4] = {8, (cuuint64_t)ny, (cuuint64_t)nch, (cuuint64_t)nimg};
    const cuuint64_t strides[3] = {16, (cuuint64_t)ny * 16, (cuuint64_t)nch * ny * 16};
    const cuuint32_t box[4] = {8, (cuuint32_t)(kTcM + K - 1), KD::kChunks, 1};
    const cuuint32_t estr[4] = {1, 1, 1, 1};
    for (int part = 0; part < 3; ++part) {
        const CUresult r = encode(&maps[part], CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, parts[part],
                                  dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                                  CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (r != CUDA_SUCCESS) return 2;
    }
    return 0;
}

int make_tc_maps(const float *hi, const float *lo, int nimg, int ny, int nx, int K,
                 CUtensorMap *mhi, CUtensorMap *mlo)
{
    const EncodeFn encode = tensor_map_encoder();
    if (!encode) return 1;
    const int nch = (nx + 3) / 4;
    const cuuint64_t dims[4] = {4, (cuuint64_t)ny, (cuuint64_t)nch, (cuuint64_t)nimg};
    const cuuint64_t strides[3] = {16, (cuuint64_t)ny * 16, (cuuint64_t)nch * ny * 16};
    const cuuint32_t box[4] = {4, (cuuint32_t)(kTcM + K - 1), kTcKd / 4, 1};
    const cuuint32_t estr[4] = {1, 1, 1, 1};
    for (int part = 0; part < 2; ++part) {
        const CUresult r = encode(part ? mlo : mhi, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4,
                                  const_cast<float *>(part ? lo : hi), dims, strides, box, estr,
                                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                                  CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (r != CUDA_SUCCESS) return 2;
    }
    return 0;
}

cudaError_t launch_trace_split(const LensDev &L, const float *kc, int nvec, float *unbl,
                               int grid, cudaStream_t st)
{
    switch (sub_class(L.sub)) {
        case 4: k_trace_split<4><<<grid, kThreads, 0, st>>>(L, kc, nvec, unbl); break;
        case 5: k_trace_split<5><<<grid, kThreads, 0, st>>>(L, kc, nvec, unbl); break;
        default: k_trace_split<0><<<grid, kThreads, 0, st>>>(L, kc, nvec, unbl); break;
    }
    return cudaGetLastError();
}

cudaError_t launch_conv_direct_split(const LensDev &L, const float *unbl, int nvec,
                                     float *blur, int grid, cudaStream_t st)
{
    const size_t smem = conv_direct_split_smem(L);
    if (L.K == 31 && L.W == padded_stride(L.nx, 31)) {
        cudaError_t e = cudaFuncSetAttribute(k_conv_direct_split<31>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        k_conv_direct_split<31><<<grid, kThreads, smem, st>>>(L, unbl, nvec, blur);
    } else {
        cudaError_t e = cudaFuncSetAttribute(k_conv_direct_split<0>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        k_conv_direct_split<0><<<grid, kThreads, smem, st>>>(L, unbl, nvec, blur);
    }
    return cudaGetLastError();
}

cudaError_t launch_conv_tc(const LensDev &L, const float *unbl, int nvec, float *hi,
                           float *lo, const CUtensorMap &mhi, const CUtensorMap &mlo,
                           float *blur, const float *tiles, int *status, int grid,
                           cudaStream_t st)
{
    const int nimg = 2 * nvec, nch = (L.nx + 3) / 4;
    const long long n = (long long)nimg * nch * L.ny;
    const int sg = (int)std::min<long long>((n + 255) / 256, 65535);
    k_tf32_split<<<sg, 256, 0, st>>>(unbl, nimg, L.ny, L.nx, nch,
                                     reinterpret_cast<float4 *>(hi), reinterpret_cast<float4 *>(lo));
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const size_t smem = conv_tc_smem(false);
    e = cudaFuncSetAttribute(k_conv_tc<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem);
    if (e != cudaSuccess) return e;
    k_conv_tc<false><<<grid, 192, smem, st>>>(L, mhi, mlo, mlo, nimg, blur,
                                              reinterpret_cast<const unsigned char *>(tiles),
                                              status);
    return cudaGetLastError();
}

cudaError_t launch_conv_bf(const LensDev &L, const float *unbl, int nvec, void *const *parts,
                           const CUtensorMap *maps, float *blur, const uint16_t *tiles,
                           int *status, int grid, cudaStream_t st)
{
    const int nimg = 2 * nvec, nch = (L.nx + 7) / 8;
    const long long n = (long long)nimg * nch * L.ny;
    const int sg = (int)std::min<long long>((n + 255) / 256, 65535);
    k_bf16_split<<<sg, 256, 0, st>>>(unbl, nimg, L.ny, L.nx, nch,
                                     reinterpret_cast<uint4 *>(parts[0]),
                                     reinterpret_cast<uint4 *>(parts[1]),
                                     reinterpret_cast<uint4 *>(parts[2]));
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const size_t smem = conv_tc_smem(true);
    e = cudaFuncSetAttribute(k_conv_tc<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem);
    if (e != cudaSuccess) return e;
    k_conv_tc<true><<<grid, 192, smem, st>>>(L, maps[0], maps[1], maps[2], nimg, blur,
                                             reinterpret_cast<const unsigned char *>(tiles),
                                             status);
    return cudaGetLastError();
}

cudaError_t launch_sums_split(const LensDev &L, const float *kc, const float *blur,
                              int nvec, double *out, int grid, cudaStream_t st)
{
    k_sums_split<<<grid, kThreads, 0, st>>>(L, kc, blur, nvec, out);
    return cudaGetLastError();
}

}  // namespace tll
