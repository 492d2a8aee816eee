// Fitness of the current factors (Sec. "Evaluation Measures"):
//   fit = 1 - ||X - [[A, B, C]]||_F / ||X||_F.
// The residual is formed element by element (no cancellation between
// ||X||^2 and the model terms); each CTA sums its 32 x 256 tile in fp32 and the
// per-CTA sums are added in fp64.
#include "octen_internal.cuh"

namespace octen {

constexpr int kFitRows = 32;
constexpr int kFitCols = 256;

template <Elem EX>
__device__ __forceinline__ float ldx(const void *X, int64_t idx) {
  if constexpr (EX == Elem::F32) return static_cast<const float *>(X)[idx];
  else return __bfloat162float(static_cast<const __nv_bfloat16 *>(X)[idx]);
}

template <Elem EX>
__global__ void __launch_bounds__(kFitCols)
    fit_tile_kernel(const void *__restrict__ X, int64_t I, int64_t J, const float *__restrict__ A,
                    const float *__restrict__ B, const float *__restrict__ C, int R,
                    double *__restrict__ partial) {
  __shared__ float w[kFitRows][32];
  __shared__ float red0[kFitCols / 32], red1[kFitCols / 32];
  const int64_t k = blockIdx.z;
  const int64_t i0 = (int64_t)blockIdx.y * kFitRows;
  const int64_t j = (int64_t)blockIdx.x * kFitCols + threadIdx.x;
  for (int e = threadIdx.x; e < kFitRows * 32; e += blockDim.x) {
    const int ii = e / 32, r = e % 32;
    const int64_t i = i0 + ii;
    w[ii][r] = (i < I && r < R) ? A[i * R + r] * C[k * R + r] : 0.f;
  }
  __syncthreads();
  float s0 = 0.f, s1 = 0.f;
  if (j < J) {
    float b[32];
#pragma unroll
    for (int r = 0; r < 32; ++r) b[r] = r < R ? B[j * R + r] : 0.f;
    for (int ii = 0; ii < kFitRows; ++ii) {
      const int64_t i = i0 + ii;
      if (i >= I) break;
      float xh = 0.f;
#pragma unroll
      for (int r = 0; r < 32; ++r) xh = fmaf(w[ii][r], b[r], xh);
      const float x = ldx<EX>(X, (k * I + i) * J + j);
      const float e = x - xh;
      s0 = fmaf(x, x, s0);
      s1 = fmaf(e, e, s1);
    }
  }
  for (int o = 16; o > 0; o >>= 1) {
    s0 += __shfl_xor_sync(0xffffffffu, s0, o);
    s1 += __shfl_xor_sync(0xffffffffu, s1, o);
  }
  if ((threadIdx.x & 31) == 0) {
    red0[threadIdx.x >> 5] = s0;
    red1[threadIdx.x >> 5] = s1;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double t0 = 0.0, t1 = 0.0;
    for (int w8 = 0; w8 < kFitCols / 32; ++w8) { t0 += red0[w8]; t1 += red1[w8]; }
    const int64_t b = ((int64_t)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
    partial[2 * b] = t0;
    partial[2 * b + 1] = t1;
  }
}

__global__ void fit_reduce_kernel(const double *__restrict__ partial, int64_t n,
                                  double *__restrict__ out) {
  __shared__ double r0[1024], r1[1024];
  double t0 = 0.0, t1 = 0.0;
  for (int64_t b = threadIdx.x; b < n; b += blockDim.x) {
    t0 += partial[2 * b];
    t1 += partial[2 * b + 1];
  }
  r0[threadIdx.x] = t0;
  r1[threadIdx.x] = t1;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) {
      r0[threadIdx.x] += r0[threadIdx.x + s];
      r1[threadIdx.x] += r1[threadIdx.x + s];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    out[0] = r0[0];
    out[1] = r1[0];
  }
}

int64_t fit_rows_max() { return (int64_t)65535 * kFitRows; }

int64_t fit_partial_count(int64_t K, int64_t I, int64_t J) {
  return ((J + kFitCols - 1) / kFitCols) * ((I + kFitRows - 1) / kFitRows) * K;
}

void fit_sums(const void *X, Elem tx, int64_t K, int64_t I, int64_t J, const float *A,
              const float *B, const float *C, int R, double *partial, double *out,
              cudaStream_t st) {
  dim3 grid((unsigned)((J + kFitCols - 1) / kFitCols), (unsigned)((I + kFitRows - 1) / kFitRows),
            (unsigned)K);
  if (tx == Elem::F32)
    fit_tile_kernel<Elem::F32><<<grid, kFitCols, 0, st>>>(X, I, J, A, B, C, R, partial);
  else
    fit_tile_kernel<Elem::BF16><<<grid, kFitCols, 0, st>>>(X, I, J, A, B, C, R, partial);
  count_launch();
  fit_reduce_kernel<<<1, 1024, 0, st>>>(partial, fit_partial_count(K, I, J), out);
  count_launch();
}

}  // namespace octen
