// SIMT fp32-accumulate GEMMs: the generic strided GEMM used by the small
// contractions (warm start, lift, Grams, fit) and the fp32 path of the two
// large compression contractions (mode 2 and mode 1 of the compression step,
// Sec. "Parallel Compression and Decomposition").  Every product is an fp32
// FFMA (no TF32).
#include "octen_internal.cuh"

namespace octen {

template <Elem E>
__device__ __forceinline__ float ld_elem(const void *p, int64_t idx) {
  if constexpr (E == Elem::F32) {
    return __ldg(static_cast<const float *>(p) + idx);
  } else if constexpr (E == Elem::BF16) {
    return __bfloat162float(static_cast<const __nv_bfloat16 *>(p)[idx]);
  } else {
    return float(static_cast<const __nv_fp8_e4m3 *>(p)[idx]);
  }
}

template <Elem E>
__device__ __forceinline__ void st_elem(void *p, int64_t idx, float v) {
  if constexpr (E == Elem::F32) {
    static_cast<float *>(p)[idx] = v;
  } else {
    static_cast<__nv_bfloat16 *>(p)[idx] = __float2bfloat16_rn(v);
  }
}

// Operand addressing: element (z, row, k) of an operand lives at
// (z / zdiv) * s_hi + (z % zdiv) * s_lo + row * s_row + k * s_k.
struct Operand {
  const void *p;
  int64_t s_hi, s_lo, s_row, s_k;
};

struct StridedEpi {
  float *D;
  int64_t s_hi, s_lo, s_m, s_n;
  float alpha, beta;
  __device__ __forceinline__ void operator()(int z, int zdiv, int m, int n, float v) const {
    float *d = D + (int64_t)(z / zdiv) * s_hi + (int64_t)(z % zdiv) * s_lo + (int64_t)m * s_m +
               (int64_t)n * s_n;
    *d = beta == 0.f ? alpha * v : fmaf(beta, *d, alpha * v);
  }
};

// Mode-2 epilogue: row m = k * I + i, column c of V_all; the value goes to every
// replica that owns column c (all of them for an anchor column).
template <Elem ET>
struct Mode2Epi {
  void *T;
  const float *scale;
  int64_t I;
  int P, Q, S;
  __device__ __forceinline__ void operator()(int, int, int m, int c, float v) const {
    const int64_t k = m / I, i = m - k * I;
    if (scale) v *= scale[k];
    if (c < S) {
      for (int p = 0; p < P; ++p) st_elem<ET>(T, ((k * P + p) * Q + c) * I + i, v);
    } else {
      const int p = (c - S) / (Q - S);
      const int b = S + (c - S) - p * (Q - S);
      st_elem<ET>(T, ((k * P + p) * Q + b) * I + i, v);
    }
  }
};

constexpr int kThreads = 256;
constexpr int kBK = 16;

// 256 threads as 16 x 16; each thread owns TM consecutive rows and TN columns
// strided by 16 (conflict-free shared reads of the B tile).
// kc > 0 splits K: batch index z covers k in [z * kc, min(z * kc + kc, K)) and the
// operands take no batch offset (the epilogue writes partial z).
template <Elem EA, Elem EB, int BM, int BN, class Epi>
__global__ void __launch_bounds__(kThreads)
    gemm_kernel(Operand A, Operand B, int M, int N, int K, int zdiv, int kc, Epi epi) {
  constexpr int TM = BM / 16, TN = BN / 16;
  __shared__ __align__(16) float As[kBK][BM + 4];
  __shared__ __align__(16) float Bs[kBK][BN + 1];
  const int z = blockIdx.z;
  const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int64_t offA = kc ? 0 : (int64_t)(z / zdiv) * A.s_hi + (int64_t)(z % zdiv) * A.s_lo;
  const int64_t offB = kc ? 0 : (int64_t)(z / zdiv) * B.s_hi + (int64_t)(z % zdiv) * B.s_lo;
  const bool a_kfast = A.s_k == 1, b_kfast = B.s_k == 1;
  const int kbeg = kc ? z * kc : 0;
  const int kend = kc ? min(K, kbeg + kc) : K;

  float acc[TM][TN];
#pragma unroll
  for (int i = 0; i < TM; ++i)
#pragma unroll
    for (int j = 0; j < TN; ++j) acc[i][j] = 0.f;

  for (int k0 = kbeg; k0 < kend; k0 += kBK) {
    for (int e = tid; e < BM * kBK; e += kThreads) {
      int mm, kk;
      if (a_kfast) { mm = e / kBK; kk = e % kBK; } else { mm = e % BM; kk = e / BM; }
      const int m = m0 + mm, k = k0 + kk;
      float v = 0.f;
      if (m < M && k < kend) v = ld_elem<EA>(A.p, offA + (int64_t)m * A.s_row + (int64_t)k * A.s_k);
      As[kk][mm] = v;
    }
    for (int e = tid; e < BN * kBK; e += kThreads) {
      int nn, kk;
      if (b_kfast) { nn = e / kBK; kk = e % kBK; } else { nn = e % BN; kk = e / BN; }
      const int n = n0 + nn, k = k0 + kk;
      float v = 0.f;
      if (n < N && k < kend) v = ld_elem<EB>(B.p, offB + (int64_t)n * B.s_row + (int64_t)k * B.s_k);
      Bs[kk][nn] = v;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < kBK; ++kk) {
      float a[TM], b[TN];
#pragma unroll
      for (int i = 0; i < TM; i += 4) {
        const float4 v = *reinterpret_cast<const float4 *>(&As[kk][ty * TM + i]);
        a[i] = v.x; a[i + 1] = v.y; a[i + 2] = v.z; a[i + 3] = v.w;
      }
#pragma unroll
      for (int j = 0; j < TN; ++j) b[j] = Bs[kk][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < TM; ++i) {
    const int m = m0 + ty * TM + i;
    if (m >= M) continue;
#pragma unroll
    for (int j = 0; j < TN; ++j) {
      const int n = n0 + tx + 16 * j;
      if (n < N) epi(z, zdiv, m, n, acc[i][j]);
    }
  }
}

// fp32 GEMM with both operands K-contiguous and 16-byte aligned rows, 128 x 128
// tiles: float4 global loads prefetched into registers during the previous
// tile's arithmetic, double-buffered shared tiles (stored [k][m] / [k][n]),
// and an 8 x 8 block per thread read as four 16-byte shared loads per k
// (rows ty*4 .. +3 and 64 + ty*4 .., columns tx*4 .. +3 and 64 + tx*4 ..).
// Every output is the same sequence of FMAs over k as in gemm_kernel.
constexpr int kTnBK = 16, kTnLD = 128 + 4;

__device__ __forceinline__ void tn_load(const float *p, int64_t s_row, int rows, int r0, int k0,
                                        int K, int t, float4 (&v)[2]) {
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const int idx = t + 256 * h, row = idx >> 2, k = k0 + 4 * (idx & 3);
    const int r = r0 + row;
    float4 x = make_float4(0.f, 0.f, 0.f, 0.f);
    if (r < rows) {
      const float *q = p + (int64_t)r * s_row + k;
      if (k + 3 < K) {
        x = __ldg(reinterpret_cast<const float4 *>(q));
      } else {
        if (k < K) x.x = __ldg(q);
        if (k + 1 < K) x.y = __ldg(q + 1);
        if (k + 2 < K) x.z = __ldg(q + 2);
      }
    }
    v[h] = x;
  }
}

__device__ __forceinline__ void tn_store(float (*S)[kTnLD], int t, const float4 (&v)[2]) {
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const int idx = t + 256 * h, row = idx >> 2, k = 4 * (idx & 3);
    S[k][row] = v[h].x;
    S[k + 1][row] = v[h].y;
    S[k + 2][row] = v[h].z;
    S[k + 3][row] = v[h].w;
  }
}

template <class Epi>
__global__ void __launch_bounds__(kThreads, 2)
    sgemm_tn_kernel(Operand A, Operand B, int M, int N, int K, int zdiv, Epi epi) {
  __shared__ __align__(16) float As[2][kTnBK][kTnLD];
  __shared__ __align__(16) float Bs[2][kTnBK][kTnLD];
  const int z = blockIdx.z;
  const int m0 = blockIdx.y * 128, n0 = blockIdx.x * 128;
  const int t = threadIdx.x, tx = t & 15, ty = t >> 4;
  const float *pa = static_cast<const float *>(A.p) + (int64_t)(z / zdiv) * A.s_hi +
                    (int64_t)(z % zdiv) * A.s_lo;
  const float *pb = static_cast<const float *>(B.p) + (int64_t)(z / zdiv) * B.s_hi +
                    (int64_t)(z % zdiv) * B.s_lo;
  float acc[8][8];
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int j = 0; j < 8; ++j) acc[i][j] = 0.f;
  float4 ra[2], rb[2];
  tn_load(pa, A.s_row, M, m0, 0, K, t, ra);
  tn_load(pb, B.s_row, N, n0, 0, K, t, rb);
  tn_store(As[0], t, ra);
  tn_store(Bs[0], t, rb);
  __syncthreads();
  int buf = 0;
  for (int k0 = 0; k0 < K; k0 += kTnBK) {
    const bool more = k0 + kTnBK < K;
    if (more) {   // the next tile's loads are in flight during this tile's arithmetic
      tn_load(pa, A.s_row, M, m0, k0 + kTnBK, K, t, ra);
      tn_load(pb, B.s_row, N, n0, k0 + kTnBK, K, t, rb);
    }
#pragma unroll
    for (int kk = 0; kk < kTnBK; ++kk) {
      const float4 a0 = *reinterpret_cast<const float4 *>(&As[buf][kk][ty * 4]);
      const float4 a1 = *reinterpret_cast<const float4 *>(&As[buf][kk][64 + ty * 4]);
      const float4 b0 = *reinterpret_cast<const float4 *>(&Bs[buf][kk][tx * 4]);
      const float4 b1 = *reinterpret_cast<const float4 *>(&Bs[buf][kk][64 + tx * 4]);
      const float a[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
      const float b[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
      for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
    }
    if (more) {
      tn_store(As[buf ^ 1], t, ra);
      tn_store(Bs[buf ^ 1], t, rb);
    }
    __syncthreads();
    buf ^= 1;
  }
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const int m = m0 + (i < 4 ? ty * 4 + i : 64 + ty * 4 + i - 4);
    if (m >= M) continue;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const int n = n0 + (j < 4 ? tx * 4 + j : 64 + tx * 4 + j - 4);
      if (n < N) epi(z, zdiv, m, n, acc[i][j]);
    }
  }
}

// The K-contiguous fp32 kernel applies when both operands have unit K stride
// and every row (and batch offset) starts 16-byte aligned.
static bool tn_ok(const Operand &A, const Operand &B) {
  auto al = [](const Operand &o) {
    return o.s_k == 1 && o.s_row % 4 == 0 && o.s_hi % 4 == 0 && o.s_lo % 4 == 0 &&
           (reinterpret_cast<uintptr_t>(o.p) & 15) == 0;
  };
  return al(A) && al(B);
}

template <Elem EA, Elem EB, int BM, int BN, class Epi>
static void launch_gemm(const Operand &A, const Operand &B, int M, int N, int K, int batch,
                        int zdiv, const Epi &epi, cudaStream_t st, int kc = 0) {
  if (M <= 0 || N <= 0 || batch <= 0) return;
  dim3 grid((N + BN - 1) / BN, (M + BM - 1) / BM, batch);
  if constexpr (EA == Elem::F32 && EB == Elem::F32 && BM == 128 && BN == 128) {
    if (kc == 0 && K > 0 && tn_ok(A, B)) {
      sgemm_tn_kernel<Epi><<<grid, kThreads, 0, st>>>(A, B, M, N, K, zdiv, epi);
      count_launch();
      return;
    }
  }
  gemm_kernel<EA, EB, BM, BN, Epi><<<grid, kThreads, 0, st>>>(A, B, M, N, K, zdiv, kc, epi);
  count_launch();
}

// D(m, n) = alpha * sum_z part[z](m, n) + beta * D(m, n)
__global__ void splitk_reduce_kernel(const float *__restrict__ part, int splits, int M, int N,
                                     float *D, int64_t s_m, int64_t s_n, float alpha, float beta) {
  const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t MN = (int64_t)M * N;
  if (idx >= MN) return;
  float acc = 0.f;
  for (int z = 0; z < splits; ++z) acc += part[z * MN + idx];
  const int m = (int)(idx / N), n = (int)(idx % N);
  float *d = D + m * s_m + n * s_n;
  *d = beta == 0.f ? alpha * acc : fmaf(beta, *d, alpha * acc);
}

template <Elem EA, Elem EB>
static void gemm_dispatch_tile(const Operand &A, const Operand &B, const GemmArgs &g,
                               const StridedEpi &epi, cudaStream_t st) {
  // Small problems get 64 x 64 tiles so that more CTAs are in flight.
  const int64_t tiles128 = (int64_t)((g.M + 127) / 128) * ((g.N + 127) / 128) * g.batch;
  if (tiles128 >= 152)
    launch_gemm<EA, EB, 128, 128>(A, B, g.M, g.N, g.K, g.batch, 1, epi, st);
  else
    launch_gemm<EA, EB, 64, 64>(A, B, g.M, g.N, g.K, g.batch, 1, epi, st);
}

// Skinny fp32 GEMM (N <= 32): D = alpha A B + beta D, or (one batch item only)
// the split-K partials part[split][m][n] of A B; batch items along grid z.  A CTA covers 128 rows over one K
// range in steps of 32: the A step is staged as As[k][m] (loads coalesced along
// m or along k, whichever is contiguous), the B step as Bs[k][n] (zero beyond
// N); thread t owns rows t % 32 + 32 j (j < 4) and columns 8 (t / 32) .. + 7.
constexpr int kSkBM = 128, kSkBK = 32;

__global__ void __launch_bounds__(128)
    gemm_skinny_kernel(const float *__restrict__ A, int64_t sAm, int64_t sAk,
                       const float *__restrict__ B, int64_t sBn, int64_t sBk, int M, int N, int K,
                       int kc, float *D, int64_t sDm, int64_t sDn, float alpha, float beta,
                       float *__restrict__ part, int64_t sAz, int64_t sBz, int64_t sDz) {
  __shared__ float As[kSkBK][kSkBM + 1];
  // batch item blockIdx.z (never split: part is null then)
  A += blockIdx.z * sAz;
  B += blockIdx.z * sBz;
  D += blockIdx.z * sDz;
  __shared__ __align__(16) float Bs[kSkBK][32];
  const int tid = threadIdx.x, rg = tid & 31, cg = tid >> 5;
  const int m0 = blockIdx.x * kSkBM;
  const int k_begin = blockIdx.y * kc;
  const int k_end = min(K, k_begin + kc);
  float acc[4][8];
#pragma unroll
  for (int j = 0; j < 4; ++j)
#pragma unroll
    for (int c = 0; c < 8; ++c) acc[j][c] = 0.f;
  for (int k0 = k_begin; k0 < k_end; k0 += kSkBK) {
    __syncthreads();   // the previous step's tiles are consumed
    if (sAm == 1) {
      const int m = m0 + tid;
#pragma unroll 8
      for (int kk = 0; kk < kSkBK; ++kk) {
        const int k = k0 + kk;
        As[kk][tid] = (m < M && k < k_end) ? __ldg(A + m + (int64_t)k * sAk) : 0.f;
      }
    } else {
      const int kk = tid & 31, k = k0 + kk;
#pragma unroll 8
      for (int j = 0; j < kSkBM / 4; ++j) {
        const int mm = (tid >> 5) + 4 * j, m = m0 + mm;
        As[kk][mm] = (m < M && k < k_end) ? __ldg(A + (int64_t)m * sAm + (int64_t)k * sAk) : 0.f;
      }
    }
    {
      const int n = tid & 31;
#pragma unroll
      for (int j = 0; j < kSkBK / 4; ++j) {
        const int kk = (tid >> 5) + 4 * j, k = k0 + kk;
        Bs[kk][n] = (n < N && k < k_end) ? __ldg(B + (int64_t)k * sBk + (int64_t)n * sBn) : 0.f;
      }
    }
    __syncthreads();
#pragma unroll 4
    for (int kk = 0; kk < kSkBK; ++kk) {
      const float4 b0 = *reinterpret_cast<const float4 *>(&Bs[kk][8 * cg]);
      const float4 b1 = *reinterpret_cast<const float4 *>(&Bs[kk][8 * cg + 4]);
      const float bv[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const float a = As[kk][rg + 32 * j];
#pragma unroll
        for (int c = 0; c < 8; ++c) acc[j][c] = fmaf(a, bv[c], acc[j][c]);
      }
    }
  }
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const int m = m0 + rg + 32 * j;
    if (m >= M) continue;
#pragma unroll
    for (int c = 0; c < 8; ++c) {
      const int n = 8 * cg + c;
      if (n >= N) continue;
      if (part) {
        part[((int64_t)blockIdx.y * M + m) * N + n] = acc[j][c];
      } else {
        float *d = D + (int64_t)m * sDm + (int64_t)n * sDn;
        *d = beta == 0.f ? alpha * acc[j][c] : fmaf(beta, *d, alpha * acc[j][c]);
      }
    }
  }
}

// The same product for A stored with m contiguous (sAm == 1, sAk a multiple of
// 4, A 16-byte aligned): the projected factors U_all^T F and the lift L e.  A
// CTA of 256 threads covers 128 rows; each K step of 32 stages A as As[k][m]
// from 16-byte loads (a warp reads 512 contiguous bytes of one k row) and B as
// Bs[k][n]; thread t owns rows 4 (t % 32) .. + 3 and columns 4 (t / 32) .. + 3,
// read as one 16-byte shared load each per k.  The next step's loads are
// issued into registers before the current step is multiplied.  Every output
// is the sequential fp32 sum over its K range in k order, as in
// gemm_skinny_kernel (same splits, same partials), so the two agree bit for bit.
constexpr int kMcThreads = 256;

__global__ void __launch_bounds__(kMcThreads)
    gemm_skinny_mc_kernel(const float *__restrict__ A, int64_t sAk, const float *__restrict__ B,
                          int64_t sBn, int64_t sBk, int M, int N, int K, int kc, float *D,
                          int64_t sDm, int64_t sDn, float alpha, float beta,
                          float *__restrict__ part) {
  __shared__ __align__(16) float As[kSkBK][kSkBM];
  __shared__ __align__(16) float Bs[kSkBK][32];
  const int tid = threadIdx.x, rq = tid & 31, cq = tid >> 5;
  const int m0 = blockIdx.x * kSkBM;
  const int k_begin = blockIdx.y * kc;
  const int k_end = min(K, k_begin + kc);
  // loader roles: A float4 (row kk = tid / 32 + 8 j, rows 4 (tid % 32) ..), B (kk, n = tid % 32)
  const int lm = m0 + 4 * rq;
  float4 ra[4];
  float rb[4];
  auto load = [&](int k0) {
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int k = k0 + cq + 8 * j;
      float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
      if (k < k_end) {
        const float *src = A + (int64_t)k * sAk + lm;
        if (lm + 3 < M) {
          v = __ldg(reinterpret_cast<const float4 *>(src));
        } else {
          if (lm < M) v.x = __ldg(src);
          if (lm + 1 < M) v.y = __ldg(src + 1);
          if (lm + 2 < M) v.z = __ldg(src + 2);
        }
      }
      ra[j] = v;
      rb[j] = (k < k_end && rq < N) ? __ldg(B + (int64_t)k * sBk + (int64_t)rq * sBn) : 0.f;
    }
  };
  float acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int c = 0; c < 4; ++c) acc[i][c] = 0.f;
  if (k_begin < k_end) load(k_begin);
  for (int k0 = k_begin; k0 < k_end; k0 += kSkBK) {
    __syncthreads();   // the previous step's tiles are consumed
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      *reinterpret_cast<float4 *>(&As[cq + 8 * j][4 * rq]) = ra[j];
      Bs[cq + 8 * j][rq] = rb[j];
    }
    __syncthreads();
    if (k0 + kSkBK < k_end) load(k0 + kSkBK);
#pragma unroll 8
    for (int kk = 0; kk < kSkBK; ++kk) {
      const float4 a = *reinterpret_cast<const float4 *>(&As[kk][4 * rq]);
      const float4 b = *reinterpret_cast<const float4 *>(&Bs[kk][4 * cq]);
      const float av[4] = {a.x, a.y, a.z, a.w}, bv[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int c = 0; c < 4; ++c) acc[i][c] = fmaf(av[i], bv[c], acc[i][c]);
    }
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int m = lm + i;
    if (m >= M) continue;
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const int n = 4 * cq + c;
      if (n >= N) continue;
      if (part) {
        part[((int64_t)blockIdx.y * M + m) * N + n] = acc[i][c];
      } else {
        float *d = D + (int64_t)m * sDm + (int64_t)n * sDn;
        *d = beta == 0.f ? alpha * acc[i][c] : fmaf(beta, *d, alpha * acc[i][c]);
      }
    }
  }
}

static void gemm_skinny(const GemmArgs &g, cudaStream_t st) {
  if (g.M <= 0 || g.N <= 0) return;
  const int tiles_m = (g.M + kSkBM - 1) / kSkBM;
  int splits = 1;
  if (g.split_scratch && g.batch == 1) {
    splits = 608 / tiles_m;   // about four CTAs per SM in flight
    if (splits > g.K / 128) splits = g.K / 128;
    const int64_t MN = (int64_t)g.M * g.N;
    if ((int64_t)splits * MN > (int64_t)g.split_scratch_floats)
      splits = (int)(g.split_scratch_floats / MN);
    if (splits < 1) splits = 1;
  }
  int kc = ((g.K + splits - 1) / splits + kSkBK - 1) / kSkBK * kSkBK;
  if (kc < kSkBK) kc = kSkBK;
  splits = (g.K + kc - 1) / kc;
  if (splits < 1) splits = 1;
  const float *A = static_cast<const float *>(g.A);
  const float *B = static_cast<const float *>(g.B);
  const dim3 grid((unsigned)tiles_m, (unsigned)splits, (unsigned)g.batch);
  const bool mc = g.batch == 1 && g.sAm == 1 && g.sAk % 4 == 0 &&
                  (reinterpret_cast<uintptr_t>(A) & 15) == 0;
  if (mc) {
    float *part = splits >= 2 ? g.split_scratch : nullptr;
    gemm_skinny_mc_kernel<<<grid, kMcThreads, 0, st>>>(A, g.sAk, B, g.sBn, g.sBk, g.M, g.N, g.K,
                                                       splits >= 2 ? kc : (g.K < 1 ? 1 : g.K),
                                                       g.D, g.sDm, g.sDn, g.alpha, g.beta, part);
    count_launch();
    if (splits >= 2) {
      const int64_t MN = (int64_t)g.M * g.N;
      splitk_reduce_kernel<<<(unsigned)((MN + 255) / 256), 256, 0, st>>>(
          g.split_scratch, splits, g.M, g.N, g.D, g.sDm, g.sDn, g.alpha, g.beta);
      count_launch();
    }
    return;
  }
  if (splits >= 2) {
    gemm_skinny_kernel<<<grid, 128, 0, st>>>(A, g.sAm, g.sAk, B, g.sBn, g.sBk, g.M, g.N, g.K, kc,
                                             nullptr, 0, 0, 1.f, 0.f, g.split_scratch, 0, 0, 0);
    count_launch();
    const int64_t MN = (int64_t)g.M * g.N;
    splitk_reduce_kernel<<<(unsigned)((MN + 255) / 256), 256, 0, st>>>(
        g.split_scratch, splits, g.M, g.N, g.D, g.sDm, g.sDn, g.alpha, g.beta);
    count_launch();
  } else {
    gemm_skinny_kernel<<<grid, 128, 0, st>>>(A, g.sAm, g.sAk, B, g.sBn, g.sBk, g.M, g.N, g.K,
                                             g.K < 1 ? 1 : g.K, g.D, g.sDm, g.sDn, g.alpha,
                                             g.beta, nullptr, g.sAz, g.sBz, g.sDz);
    count_launch();
  }
}

void gemm_strided(const GemmArgs &g, cudaStream_t st) {
  // zdiv = 1: the whole batch index goes through the s_hi strides
  Operand A{g.A, g.sAz, 0, g.sAm, g.sAk};
  Operand B{g.B, g.sBz, 0, g.sBn, g.sBk};
  if ((g.batch == 1 || g.skinny_batch) && g.N <= 32 && g.ta == Elem::F32 && g.tb == Elem::F32) {
    gemm_skinny(g, st);
    return;
  }
  // few output tiles and a long K: split K over CTAs into the caller's scratch
  const int64_t tiles64 = (int64_t)((g.M + 63) / 64) * ((g.N + 63) / 64);
  if (g.batch == 1 && g.split_scratch && tiles64 < 76 && g.K >= 1024 &&
      g.ta == Elem::F32 && g.tb == Elem::F32) {
    int splits = (int)(304 / tiles64);
    if (splits > g.K / 256) splits = g.K / 256;
    const int64_t MN = (int64_t)g.M * g.N;
    if ((int64_t)splits * MN > (int64_t)g.split_scratch_floats)
      splits = (int)(g.split_scratch_floats / MN);
    if (splits >= 2) {
      const int kc = ((g.K + splits - 1) / splits + kBK - 1) / kBK * kBK;
      splits = (g.K + kc - 1) / kc;
      StridedEpi pe{g.split_scratch, MN, 0, g.N, 1, 1.f, 0.f};
      launch_gemm<Elem::F32, Elem::F32, 64, 64>(A, B, g.M, g.N, g.K, splits, 1, pe, st, kc);
      splitk_reduce_kernel<<<(unsigned)((MN + 255) / 256), 256, 0, st>>>(
          g.split_scratch, splits, g.M, g.N, g.D, g.sDm, g.sDn, g.alpha, g.beta);
      count_launch();
      return;
    }
  }
  StridedEpi epi{g.D, g.sDz, 0, g.sDm, g.sDn, g.alpha, g.beta};
  if (g.ta == Elem::F32 && g.tb == Elem::F32)
    gemm_dispatch_tile<Elem::F32, Elem::F32>(A, B, g, epi, st);
  else if (g.ta == Elem::BF16 && g.tb == Elem::F32)
    gemm_dispatch_tile<Elem::BF16, Elem::F32>(A, B, g, epi, st);
  else if (g.ta == Elem::BF16 && g.tb == Elem::BF16)
    gemm_dispatch_tile<Elem::BF16, Elem::BF16>(A, B, g, epi, st);
  else
    fprintf(stderr, "octen: gemm_strided: unsupported operand types\n");
}

void mode2_simt(const Mode2Args &a, cudaStream_t st) {
  const int64_t M = a.t * a.I;
  Operand A{a.X, 0, 0, a.J, 1};
  Operand B{a.Vt, 0, 0, a.J, 1};
  if (a.tt == Elem::F32) {
    Mode2Epi<Elem::F32> epi{a.T, a.slice_scale, a.I, a.P, a.Q, a.S};
    if (a.tx == Elem::F32)
      launch_gemm<Elem::F32, Elem::F32, 128, 128>(A, B, (int)M, a.Qd, (int)a.J, 1, 1, epi, st);
    else
      fprintf(stderr, "octen: mode2_simt: fp32 output needs fp32 slices\n");
  } else {
    Mode2Epi<Elem::BF16> epi{a.T, a.slice_scale, a.I, a.P, a.Q, a.S};
    if (a.tx == Elem::BF16)
      launch_gemm<Elem::BF16, Elem::BF16, 128, 128>(A, B, (int)M, a.Qd, (int)a.J, 1, 1, epi, st);
    else if (a.tx == Elem::E4M3)
      launch_gemm<Elem::E4M3, Elem::E4M3, 128, 128>(A, B, (int)M, a.Qd, (int)a.J, 1, 1, epi, st);
    else
      fprintf(stderr, "octen: mode2_simt: unsupported slice type\n");
  }
}

void mode1_simt(const Mode1Args &a, cudaStream_t st) {
  // batch z = k * P + p
  Operand A{a.Ut, 0, (int64_t)a.Q * a.I, a.I, 1};
  Operand B{a.T, (int64_t)a.P * a.Q * a.I, (int64_t)a.Q * a.I, a.I, 1};
  StridedEpi epi{a.T2, (int64_t)a.Q * a.Q, a.t * a.Q * a.Q, a.Q, 1, 1.f, 0.f};
  const int batch = (int)(a.t * a.P);
  const bool big = a.Q > 64;
  if (a.te == Elem::F32) {
    if (big) launch_gemm<Elem::F32, Elem::F32, 128, 128>(A, B, a.Q, a.Q, (int)a.I, batch, a.P, epi, st);
    else launch_gemm<Elem::F32, Elem::F32, 64, 64>(A, B, a.Q, a.Q, (int)a.I, batch, a.P, epi, st);
  } else {
    if (big) launch_gemm<Elem::BF16, Elem::BF16, 128, 128>(A, B, a.Q, a.Q, (int)a.I, batch, a.P, epi, st);
    else launch_gemm<Elem::BF16, Elem::BF16, 64, 64>(A, B, a.Q, a.Q, (int)a.I, batch, a.P, epi, st);
  }
}

}  // namespace octen
