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

template <Elem EA, Elem EB, int BM, int BN, class Epi>
static void launch_gemm(const Operand &A, const Operand &B, int M, int N, int K, int batch,
                        int zdiv, const Epi &epi, cudaStream_t st, int kc = 0) {
  if (M <= 0 || N <= 0 || batch <= 0) return;
  dim3 grid((N + BN - 1) / BN, (M + BM - 1) / BM, batch);
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

void gemm_strided(const GemmArgs &g, cudaStream_t st) {
  // zdiv = 1: the whole batch index goes through the s_hi strides
  Operand A{g.A, g.sAz, 0, g.sAm, g.sAk};
  Operand B{g.B, g.sBz, 0, g.sBn, g.sBk};
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
