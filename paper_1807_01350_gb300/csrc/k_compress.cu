// Compression helpers (Sec. "Parallel Compression and Decomposition"):
// layout/precision conversion of the projection matrices, per-slice e4m3
// quantisation of the slice batch, and the time-mode contraction fused with the
// summary update X_p = Y_p + Z_p (Eq. 2, Algorithm 1's second step).
#include <cstdlib>

#include "octen_internal.cuh"

namespace octen {

__device__ __forceinline__ float round_as(float v, Elem te) {
  if (te == Elem::BF16) return __bfloat162float(__float2bfloat16_rn(v));
  if (te == Elem::E4M3) return float(__nv_fp8_e4m3(v));  // RNE, saturating to +-448
  return v;
}

__device__ __forceinline__ void store_as(void *out, int64_t idx, float v, Elem te) {
  if (te == Elem::F32) static_cast<float *>(out)[idx] = v;
  else if (te == Elem::BF16) static_cast<__nv_bfloat16 *>(out)[idx] = __float2bfloat16_rn(v);
  else static_cast<__nv_fp8_e4m3 *>(out)[idx] = __nv_fp8_e4m3(v);
}

// out[(p * Q + q) * rows + r] = M_all[r * Qd + col_p(q)] in type te, where
// col_p(q) = q for anchors (q < S) and S + p (Q - S) + (q - S) otherwise.
__global__ void replica_transpose_kernel(const float *__restrict__ M, int64_t rows, int P, int Q,
                                         int S, int Qd, void *out, Elem te) {
  __shared__ float tile[32][33];
  const int p = blockIdx.z;
  const int64_t r0 = (int64_t)blockIdx.x * 32;
  const int q0 = blockIdx.y * 32;
  const int tx = threadIdx.x, ty = threadIdx.y;  // 32 x 8
  for (int yy = ty; yy < 32; yy += 8) {
    const int64_t r = r0 + yy;
    const int q = q0 + tx;
    float v = 0.f;
    if (r < rows && q < Q) {
      const int c = q < S ? q : S + p * (Q - S) + (q - S);
      v = M[r * Qd + c];
    }
    tile[yy][tx] = v;
  }
  __syncthreads();
  for (int yy = ty; yy < 32; yy += 8) {
    const int q = q0 + yy;
    const int64_t r = r0 + tx;
    if (q < Q && r < rows) store_as(out, ((int64_t)p * Q + q) * rows + r, tile[tx][yy], te);
  }
}

void make_replica_transpose(const float *M_all, int64_t rows, int P, int Q, int S, int Qd,
                            void *out, Elem te, cudaStream_t st) {
  dim3 grid((unsigned)((rows + 31) / 32), (Q + 31) / 32, P);
  replica_transpose_kernel<<<grid, dim3(32, 8), 0, st>>>(M_all, rows, P, Q, S, Qd, out, te);
  count_launch();
}

void make_transpose(const float *M_all, int64_t rows, int Qd, void *out, Elem te,
                    cudaStream_t st) {
  make_replica_transpose(M_all, rows, 1, Qd, 0, Qd, out, te, st);
}

__global__ void round_copy_kernel(const float *__restrict__ in, float *__restrict__ out,
                                  int64_t n, Elem te) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    out[i] = round_as(in[i], te);
}

void round_copy(const float *in, float *out, int64_t n, Elem te, cudaStream_t st) {
  if (n <= 0) return;
  const int blocks = (int)((n + 255) / 256 < 4096 ? (n + 255) / 256 : 4096);
  round_copy_kernel<<<blocks, 256, 0, st>>>(in, out, n, te);
  count_launch();
}

// ---------------------------------------------------------------------------
// Per-slice absmax scaling to e4m3: s_k = max|X_k| / 448, X8 = rne(X / s_k).
// ---------------------------------------------------------------------------
// With VEC every thread reads 8 bf16 at a time (16-byte loads; IJ a multiple
// of 8 and X 16-byte aligned), else one.
template <bool VEC>
__global__ void slice_absmax_kernel(const __nv_bfloat16 *__restrict__ X, int64_t IJ,
                                    unsigned int *__restrict__ amax_bits) {
  const int k = blockIdx.y;
  const __nv_bfloat16 *x = X + (int64_t)k * IJ;
  float m = 0.f;
  if (VEC) {
    const uint4 *x8 = reinterpret_cast<const uint4 *>(x);
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < IJ / 8;
         i += (int64_t)gridDim.x * blockDim.x) {
      const uint4 raw = __ldg(x8 + i);
      const __nv_bfloat162 *h = reinterpret_cast<const __nv_bfloat162 *>(&raw);
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const float2 v = __bfloat1622float2(h[e]);
        m = fmaxf(m, fmaxf(fabsf(v.x), fabsf(v.y)));
      }
    }
  } else {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < IJ;
         i += (int64_t)gridDim.x * blockDim.x)
      m = fmaxf(m, fabsf(__bfloat162float(x[i])));
  }
  for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) atomicMax(amax_bits + k, __float_as_uint(m));
}

__global__ void slice_scale_kernel(const unsigned int *__restrict__ amax_bits, int64_t t,
                                   float *__restrict__ scale) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k < t) {
    const float a = __uint_as_float(amax_bits[k]);
    scale[k] = a > 0.f ? a / 448.f : 1.f;
  }
}

// X8 = rne_e4m3(X / s_k) (IEEE division, then the satfinite RNE conversion),
// 8 elements per thread and step with VEC (16-byte loads, 8-byte stores).
template <bool VEC>
__global__ void quantize_kernel(const __nv_bfloat16 *__restrict__ X, int64_t IJ,
                                const float *__restrict__ scale,
                                __nv_fp8_e4m3 *__restrict__ X8) {
  const int k = blockIdx.y;
  const float s = scale[k];
  const __nv_bfloat16 *x = X + (int64_t)k * IJ;
  __nv_fp8_e4m3 *y = X8 + (int64_t)k * IJ;
  if (VEC) {
    const uint4 *x8 = reinterpret_cast<const uint4 *>(x);
    uint2 *y8 = reinterpret_cast<uint2 *>(y);
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < IJ / 8;
         i += (int64_t)gridDim.x * blockDim.x) {
      const uint4 raw = __ldg(x8 + i);
      const __nv_bfloat16 *h = reinterpret_cast<const __nv_bfloat16 *>(&raw);
      __align__(8) __nv_fp8_e4m3 q[8];
#pragma unroll
      for (int e = 0; e < 8; ++e) q[e] = __nv_fp8_e4m3(__fdiv_rn(__bfloat162float(h[e]), s));
      y8[i] = *reinterpret_cast<const uint2 *>(q);
    }
  } else {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < IJ;
         i += (int64_t)gridDim.x * blockDim.x)
      y[i] = __nv_fp8_e4m3(__fdiv_rn(__bfloat162float(x[i]), s));
  }
}

void quantize_e4m3(const __nv_bfloat16 *X, int64_t t, int64_t IJ, __nv_fp8_e4m3 *X8,
                   float *scale, cudaStream_t st) {
  // the scale buffer doubles as the absmax bit store before it holds scales
  unsigned int *bits = reinterpret_cast<unsigned int *>(scale);
  cudaMemsetAsync(bits, 0, t * sizeof(unsigned int), st);
  // 16-byte loads need IJ a multiple of 8 and 16-byte aligned slices
  const bool vec = IJ % 8 == 0 && (reinterpret_cast<uintptr_t>(X) & 15) == 0 &&
                   (reinterpret_cast<uintptr_t>(X8) & 7) == 0;
  // about four CTAs of 256 threads per SM over the whole batch
  const int64_t per = vec ? IJ / 8 : IJ;
  int64_t bx = (4 * 152 + t - 1) / t;
  if (bx > (per + 255) / 256) bx = (per + 255) / 256;
  if (bx < 1) bx = 1;
  const dim3 grid((unsigned)bx, (unsigned)t);
  if (vec) slice_absmax_kernel<true><<<grid, 256, 0, st>>>(X, IJ, bits);
  else slice_absmax_kernel<false><<<grid, 256, 0, st>>>(X, IJ, bits);
  count_launch();
  slice_scale_kernel<<<(unsigned)((t + 127) / 128), 128, 0, st>>>(bits, t, scale);
  count_launch();
  if (vec) quantize_kernel<true><<<grid, 256, 0, st>>>(X, IJ, scale, X8);
  else quantize_kernel<false><<<grid, 256, 0, st>>>(X, IJ, scale, X8);
  count_launch();
}

// ---------------------------------------------------------------------------
// Time-mode contraction + summary update:
//   Y[p][a][b][c] += sum_k T2[p][k][a][b] * W[k][col_p(c)]
// One CTA owns kRows consecutive (a, b) rows of one replica and every c.
// ---------------------------------------------------------------------------
constexpr int kRows = 32;

__global__ void __launch_bounds__(256)
    mode3_kernel(const float *__restrict__ T2, const float *__restrict__ W, float *__restrict__ Y,
                 int t, int Q, int S, int Qd) {
  extern __shared__ float sm[];
  float *Ws = sm;                       // [t][Q]
  float *Ts = sm + (size_t)t * Q;       // [t][kRows]
  const int p = blockIdx.y;
  const int64_t QQ = (int64_t)Q * Q;
  const int64_t row0 = (int64_t)blockIdx.x * kRows;
  const int nrows = (int)(QQ - row0 < kRows ? QQ - row0 : kRows);
  for (int e = threadIdx.x; e < t * Q; e += blockDim.x) {
    const int k = e / Q, c = e % Q;
    const int col = c < S ? c : S + p * (Q - S) + (c - S);
    Ws[e] = W[(int64_t)k * Qd + col];
  }
  for (int e = threadIdx.x; e < t * kRows; e += blockDim.x) {
    const int k = e / kRows, r = e % kRows;
    Ts[e] = r < nrows ? T2[((int64_t)p * t + k) * QQ + row0 + r] : 0.f;
  }
  __syncthreads();
  float *Yp = Y + (int64_t)p * QQ * Q + row0 * Q;
  for (int e = threadIdx.x; e < nrows * Q; e += blockDim.x) {
    const int r = e / Q, c = e % Q;
    float acc = 0.f;
    for (int k = 0; k < t; ++k) acc = fmaf(Ts[k * kRows + r], Ws[k * Q + c], acc);
    Yp[e] += acc;
  }
}

// Streaming form for Q % 4 == 0.  A CTA keeps W_p (rows padded to a multiple
// of 4 with zeros) in shared memory and walks blocks of rows (a, b) of one
// replica; per block it stages T2 transposed to [row][k] and every thread owns
// 4 consecutive c (one float4) of kRG rows: the kRG loads of Y are issued
// together, the t-term sums taken from shared memory, then the rows stored.
// With Xa / Xc given it also writes the bf16 copies of the updated X_p that
// the tensor-core CP-ALS reads, Xa[p][(a,b)][c] and Xc[p][c][(a,b)] (the
// latter through a [c][row] block in shared memory, 16-byte stores).
template <int kRG>
__global__ void __launch_bounds__(256, 2)
    mode3_stream_kernel(const float *__restrict__ T2, const float *__restrict__ W,
                        float *__restrict__ Y, int t, int Q, int S, int Qd,
                        __nv_bfloat16 *__restrict__ Xa, __nv_bfloat16 *__restrict__ Xc) {
  extern __shared__ __align__(16) float sm3[];
  const int tp = (t + 3) & ~3;                 // padded k extent
  const int ncg = Q / 4;                       // float4 column groups
  const int lanes = blockDim.x / ncg;          // rows in flight per pass
  const int rows_blk = lanes * kRG;
  const int xp = rows_blk + 1;                 // pitch of the [c][row] bf16 block
  float *Ws = sm3;                             // [tp][Q]
  float *Ts = sm3 + (size_t)tp * Q;            // [rows_blk][tp]
  __nv_bfloat16 *Xs = reinterpret_cast<__nv_bfloat16 *>(Ts + (size_t)rows_blk * tp);   // [Q][xp]
  const int p = blockIdx.y;
  const int64_t QQ = (int64_t)Q * Q;
  for (int e = threadIdx.x; e < tp * Q; e += blockDim.x) {
    const int k = e / Q, c = e - (e / Q) * Q;
    const int col = c < S ? c : S + p * (Q - S) + (c - S);
    Ws[e] = k < t ? W[(int64_t)k * Qd + col] : 0.f;
  }
  const int cg = threadIdx.x % ncg, rl = threadIdx.x / ncg;
  const bool active = rl < lanes;
  const int64_t nblk = (QQ + rows_blk - 1) / rows_blk;
  float *Yp = Y + (int64_t)p * QQ * Q;
  for (int64_t blk = blockIdx.x; blk < nblk; blk += gridDim.x) {
    const int64_t row0 = blk * rows_blk;
    {
      // this CTA's next block of Y rows (and of T2) into the L2 while this
      // block computes; every address lies inside the next block's rows
      const int64_t nrow0 = row0 + (int64_t)gridDim.x * rows_blk;
      if (nrow0 < QQ) {
        const int64_t nr = QQ - nrow0 < rows_blk ? QQ - nrow0 : rows_blk;
        const char *ny = reinterpret_cast<const char *>(Yp + nrow0 * Q);
        const int64_t lines = nr * Q * (int64_t)sizeof(float) / 128;
        for (int64_t e = threadIdx.x; e < lines; e += blockDim.x) prefetch_l2(ny + e * 128);
        for (int k = threadIdx.x; k < t; k += blockDim.x)
          prefetch_l2(T2 + ((int64_t)p * t + k) * QQ + nrow0);
      }
    }
    __syncthreads();   // Ws ready / previous block's Ts consumed
    for (int e = threadIdx.x; e < rows_blk * tp; e += blockDim.x) {
      const int k = e / rows_blk, r = e - (e / rows_blk) * rows_blk;
      Ts[r * tp + k] =
          (k < t && row0 + r < QQ) ? T2[((int64_t)p * t + k) * QQ + row0 + r] : 0.f;
    }
    __syncthreads();
    if (active) {
      float4 y[kRG], acc[kRG];
#pragma unroll
      for (int i = 0; i < kRG; ++i) {
        const int64_t row = row0 + rl + (int64_t)lanes * i;
        y[i] = row < QQ ? reinterpret_cast<const float4 *>(Yp + row * Q)[cg]
                        : make_float4(0.f, 0.f, 0.f, 0.f);
        acc[i] = make_float4(0.f, 0.f, 0.f, 0.f);
      }
      for (int k = 0; k < tp; k += 4) {
        const float4 w0 = reinterpret_cast<const float4 *>(Ws + (k + 0) * Q)[cg];
        const float4 w1 = reinterpret_cast<const float4 *>(Ws + (k + 1) * Q)[cg];
        const float4 w2 = reinterpret_cast<const float4 *>(Ws + (k + 2) * Q)[cg];
        const float4 w3 = reinterpret_cast<const float4 *>(Ws + (k + 3) * Q)[cg];
#pragma unroll
        for (int i = 0; i < kRG; ++i) {
          const float4 x = *reinterpret_cast<const float4 *>(Ts + (rl + lanes * i) * tp + k);
          acc[i].x = fmaf(x.x, w0.x, fmaf(x.y, w1.x, fmaf(x.z, w2.x, fmaf(x.w, w3.x, acc[i].x))));
          acc[i].y = fmaf(x.x, w0.y, fmaf(x.y, w1.y, fmaf(x.z, w2.y, fmaf(x.w, w3.y, acc[i].y))));
          acc[i].z = fmaf(x.x, w0.z, fmaf(x.y, w1.z, fmaf(x.z, w2.z, fmaf(x.w, w3.z, acc[i].z))));
          acc[i].w = fmaf(x.x, w0.w, fmaf(x.y, w1.w, fmaf(x.z, w2.w, fmaf(x.w, w3.w, acc[i].w))));
        }
      }
#pragma unroll
      for (int i = 0; i < kRG; ++i) {
        const int64_t row = row0 + rl + (int64_t)lanes * i;
        const float4 v = make_float4(y[i].x + acc[i].x, y[i].y + acc[i].y, y[i].z + acc[i].z,
                                     y[i].w + acc[i].w);
        if (row < QQ) reinterpret_cast<float4 *>(Yp + row * Q)[cg] = v;
        if (Xa) {
          __align__(8) const __nv_bfloat16 h[4] = {
              __float2bfloat16_rn(v.x), __float2bfloat16_rn(v.y), __float2bfloat16_rn(v.z),
              __float2bfloat16_rn(v.w)};
          if (row < QQ)
            *reinterpret_cast<uint2 *>(Xa + ((int64_t)p * QQ + row) * Q + 4 * cg) =
                *reinterpret_cast<const uint2 *>(h);
          const int rr = rl + lanes * i;
#pragma unroll
          for (int j = 0; j < 4; ++j) Xs[(4 * cg + j) * xp + rr] = h[j];
        }
      }
    }
    if (Xc) {
      // the block's rows of every c: 8 rows (16 bytes) per store
      __syncthreads();
      const int nseg = rows_blk / 8;
      for (int e = threadIdx.x; e < Q * nseg; e += blockDim.x) {
        const int c = e / nseg, sg = e - (e / nseg) * nseg;
        const int64_t r0 = row0 + 8 * sg;
        __nv_bfloat16 *dst = Xc + ((int64_t)p * Q + c) * QQ + r0;
        const __nv_bfloat16 *src = Xs + c * xp + 8 * sg;
        if (r0 + 8 <= QQ) {
          __align__(16) __nv_bfloat16 h[8];
#pragma unroll
          for (int j = 0; j < 8; ++j) h[j] = src[j];
          *reinterpret_cast<uint4 *>(dst) = *reinterpret_cast<const uint4 *>(h);
        } else {
          for (int j = 0; j < 8 && r0 + j < QQ; ++j) dst[j] = src[j];
        }
      }
    }
  }
}

// Rows of Y per thread of the streaming mode-3 kernel (4, tried: 80
// registers and three CTAs per SM, but 0.98 ms against 0.70 ms at 4000^2).
// Also tried and dropped: the next block of Y rows prefetched into shared
// memory by a bulk asynchronous copy while the current block is computed
// (0.83 ms against 0.69 ms at 4000^2); prefetched into the L2 instead (the
// prefetch_l2 lines of the kernel), 0.681 against 0.691 - 0.697 ms.
constexpr int kMode3Rows = 8;

template <int RG>
static bool mode3_stream(const float *T2, const float *W, float *Y, int64_t t, int P, int Q,
                         int S, int Qd, cudaStream_t st, __nv_bfloat16 *Xa,
                         __nv_bfloat16 *Xc) {
  const int64_t QQ = (int64_t)Q * Q;
  const int tp = (int)((t + 3) & ~int64_t(3));
  const int ncg = Q / 4;
  const int lanes = 256 / ncg;
  const int rows_blk = lanes * RG;
  const bool layouts = Xa != nullptr && Xc != nullptr;
  const size_t smem = ((size_t)tp * Q + (size_t)rows_blk * tp) * sizeof(float) +
                      (layouts ? (size_t)Q * (rows_blk + 1) * sizeof(__nv_bfloat16) : 0);
  if (smem > 200 * 1024) return false;
  cudaFuncSetAttribute(mode3_stream_kernel<RG>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       200 * 1024);
  int dev = 0, sms = 0, per_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, mode3_stream_kernel<RG>, 256, smem);
  if (per_sm < 1) per_sm = 1;
  const int64_t nblk = (QQ + rows_blk - 1) / rows_blk;
  int64_t gx = ((int64_t)sms * per_sm + P - 1) / P;   // one wave over all replicas
  if (gx > nblk) gx = nblk;
  if (gx < 1) gx = 1;
  mode3_stream_kernel<RG><<<dim3((unsigned)gx, P), 256, smem, st>>>(
      T2, W, Y, (int)t, Q, S, Qd, layouts ? Xa : nullptr, layouts ? Xc : nullptr);
  count_launch();
  return true;
}

bool mode3_accumulate(const float *T2, const float *W, float *Y, int64_t t, int P, int Q,
                      int S, int Qd, cudaStream_t st, __nv_bfloat16 *Xa, __nv_bfloat16 *Xc) {
  const int64_t QQ = (int64_t)Q * Q;
  if (Q % 4 == 0 && Q <= 1024) {
    const bool layouts = Xa != nullptr && Xc != nullptr;
    const bool ran = mode3_stream<kMode3Rows>(T2, W, Y, t, P, Q, S, Qd, st, Xa, Xc);
    if (ran) return layouts;
  }
  const size_t smem = ((size_t)t * Q + (size_t)t * kRows) * sizeof(float);
  cudaFuncSetAttribute(mode3_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  dim3 grid((unsigned)((QQ + kRows - 1) / kRows), P);
  mode3_kernel<<<grid, 256, smem, st>>>(T2, W, Y, (int)t, Q, S, Qd);
  count_launch();
  return false;
}

}  // namespace octen
