// Replica CP-ALS (Algorithm 1's CP(X_p, R) step, Sec. "Parallel Compression and
// Decomposition") for all P replicas at once.
//
// Each sweep updates C, then A, then B by the normal equations
//   C = M3 (A^T A * B^T B)^-1,  A = M1 (B^T B * C^T C)^-1,  B = M2 (A^T A * C^T C)^-1
// with A and B normalised to unit-l2 columns, and a final C update after the
// last sweep.  The three MTTKRPs share work: one pass over X_p forms
//   H[a][c][r] = sum_b X[a][b][c] B[b][r]
// from which M3[c][r] = sum_a A[a][r] H[a][c][r] and (after C is updated)
// M1[a][r] = sum_c C[c][r] H[a][c][r]; a second pass over X_p forms M2.
// The R x R Gram Hadamard products are factored by Cholesky in fp64 (one warp),
// the Grams and the triangular substitutions run in fp32.
#include "octen_internal.cuh"

namespace octen {

// Block-wide sum of v[0..RT) held per thread; the result lands in out[RT]
// (shared) for every thread after the call.  blockDim.x must be a multiple of 32.
template <int RT>
__device__ __forceinline__ void block_sum_rows(float (&v)[RT], float *red /*[32][RT]*/,
                                               float *out /*[RT]*/) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int r = 0; r < RT; ++r) {
    float x = v[r];
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    v[r] = x;
  }
  if (lane == 0) {
#pragma unroll
    for (int r = 0; r < RT; ++r) red[warp * RT + r] = v[r];
  }
  __syncthreads();
  if (threadIdx.x < RT) {
    float s = 0.f;
    for (int w = 0; w < nw; ++w) s += red[w * RT + threadIdx.x];
    out[threadIdx.x] = s;
  }
  __syncthreads();
}

// H[p][a][c][:] = sum_b X_p[a][b][c] B_p[b][:]      grid (Q, P), thread c
template <int RT>
__global__ void __launch_bounds__(256)
    als_h_kernel(const float *__restrict__ Y, const float *__restrict__ Bf, float *__restrict__ H,
                 int Q) {
  extern __shared__ __align__(16) float Bs[];  // [Q][RT]
  const int a = blockIdx.x, p = blockIdx.y, c = threadIdx.x;
  const int64_t QQ = (int64_t)Q * Q;
  for (int e = threadIdx.x; e < Q * RT; e += blockDim.x) Bs[e] = Bf[(int64_t)p * Q * RT + e];
  __syncthreads();
  if (c >= Q) return;
  float acc[RT];
#pragma unroll
  for (int r = 0; r < RT; ++r) acc[r] = 0.f;
  const float *x = Y + (int64_t)p * QQ * Q + (int64_t)a * QQ + c;
  for (int b = 0; b < Q; ++b) {
    const float xv = __ldg(x + (int64_t)b * Q);
    const float4 *br = reinterpret_cast<const float4 *>(Bs + b * RT);
#pragma unroll
    for (int r4 = 0; r4 < RT / 4; ++r4) {
      const float4 w = br[r4];
      acc[4 * r4 + 0] = fmaf(xv, w.x, acc[4 * r4 + 0]);
      acc[4 * r4 + 1] = fmaf(xv, w.y, acc[4 * r4 + 1]);
      acc[4 * r4 + 2] = fmaf(xv, w.z, acc[4 * r4 + 2]);
      acc[4 * r4 + 3] = fmaf(xv, w.w, acc[4 * r4 + 3]);
    }
  }
  float4 *h = reinterpret_cast<float4 *>(H + (((int64_t)p * Q + a) * Q + c) * RT);
#pragma unroll
  for (int r4 = 0; r4 < RT / 4; ++r4)
    h[r4] = make_float4(acc[4 * r4], acc[4 * r4 + 1], acc[4 * r4 + 2], acc[4 * r4 + 3]);
}

// M3[p][c][r] = sum_a A_p[a][r] H[p][a][c][r]      grid (ceil(Q*RT/256), P)
template <int RT>
__global__ void als_m3_kernel(const float *__restrict__ H, const float *__restrict__ Af,
                              float *__restrict__ M, int Q) {
  const int p = blockIdx.y;
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= Q * RT) return;
  const int r = e % RT;
  const float *h = H + (int64_t)p * Q * Q * RT + e;
  const float *af = Af + (int64_t)p * Q * RT + r;
  float acc = 0.f;
  for (int a = 0; a < Q; ++a) acc = fmaf(__ldg(af + a * RT), __ldg(h + (int64_t)a * Q * RT), acc);
  M[(int64_t)p * Q * RT + e] = acc;
}

// M1[p][a][r] = sum_c C_p[c][r] H[p][a][c][r]      grid (Q, P), 256 threads
template <int RT>
__global__ void __launch_bounds__(256)
    als_m1_kernel(const float *__restrict__ H, const float *__restrict__ Cf,
                  float *__restrict__ M, int Q) {
  __shared__ float red[256];
  const int a = blockIdx.x, p = blockIdx.y;
  constexpr int G = 256 / RT;
  const int r = threadIdx.x % RT, g = threadIdx.x / RT;
  const float *h = H + (((int64_t)p * Q + a) * Q) * RT;
  const float *cf = Cf + (int64_t)p * Q * RT;
  float acc = 0.f;
  for (int c = g; c < Q; c += G) acc = fmaf(__ldg(cf + c * RT + r), __ldg(h + c * RT + r), acc);
  red[threadIdx.x] = acc;
  __syncthreads();
  if (threadIdx.x < RT) {
    float s = 0.f;
    for (int gg = 0; gg < G; ++gg) s += red[gg * RT + threadIdx.x];
    M[((int64_t)p * Q + a) * RT + threadIdx.x] = s;
  }
}

// M2[p][b][r] = sum_{a,c} X_p[a][b][c] A_p[a][r] C_p[c][r]      grid (Q, P), thread c
template <int RT>
__global__ void __launch_bounds__(256)
    als_m2_kernel(const float *__restrict__ Y, const float *__restrict__ Af,
                  const float *__restrict__ Cf, float *__restrict__ M, int Q) {
  extern __shared__ __align__(16) float sm[];
  float *As = sm;               // [Q][RT]
  float *red = sm + Q * RT;     // [8][RT]
  float *out = red + 8 * RT;    // [RT]
  const int b = blockIdx.x, p = blockIdx.y, c = threadIdx.x;
  const int64_t QQ = (int64_t)Q * Q;
  for (int e = threadIdx.x; e < Q * RT; e += blockDim.x) As[e] = Af[(int64_t)p * Q * RT + e];
  __syncthreads();
  float acc[RT];
#pragma unroll
  for (int r = 0; r < RT; ++r) acc[r] = 0.f;
  if (c < Q) {
    const float *x = Y + (int64_t)p * QQ * Q + (int64_t)b * Q + c;
    for (int a = 0; a < Q; ++a) {
      const float xv = __ldg(x + (int64_t)a * QQ);
      const float4 *ar = reinterpret_cast<const float4 *>(As + a * RT);
#pragma unroll
      for (int r4 = 0; r4 < RT / 4; ++r4) {
        const float4 w = ar[r4];
        acc[4 * r4 + 0] = fmaf(xv, w.x, acc[4 * r4 + 0]);
        acc[4 * r4 + 1] = fmaf(xv, w.y, acc[4 * r4 + 1]);
        acc[4 * r4 + 2] = fmaf(xv, w.z, acc[4 * r4 + 2]);
        acc[4 * r4 + 3] = fmaf(xv, w.w, acc[4 * r4 + 3]);
      }
    }
    const float *cf = Cf + ((int64_t)p * Q + c) * RT;
#pragma unroll
    for (int r = 0; r < RT; ++r) acc[r] *= __ldg(cf + r);
  }
  block_sum_rows<RT>(acc, red, out);
  if (threadIdx.x < RT) M[((int64_t)p * Q + b) * RT + threadIdx.x] = out[threadIdx.x];
}

// Cholesky of the R x R leading block of G (fp64, row-major [RT][RT]) by one
// warp: lane i owns row i.  Returns false if a pivot is not positive.
template <int RT>
__device__ bool warp_cholesky(double *G, double *L, int R) {
  const int lane = threadIdx.x & 31;
  bool ok = true;
  for (int j = 0; j < R; ++j) {
    if (lane == j) {
      double d = G[j * RT + j];
      for (int k = 0; k < j; ++k) d -= L[j * RT + k] * L[j * RT + k];
      L[j * RT + j] = d > 0.0 ? sqrt(d) : 0.0;
    }
    __syncwarp();
    const double piv = L[j * RT + j];
    if (!(piv > 0.0)) ok = false;
    if (ok && lane > j && lane < R) {
      double s = G[lane * RT + j];
      for (int k = 0; k < j; ++k) s -= L[lane * RT + k] * L[j * RT + k];
      L[lane * RT + j] = s / piv;
    }
    __syncwarp();
    if (!ok) break;
  }
  return ok;
}

// F_p = M_p (F1_p^T F1_p * F2_p^T F2_p)^-1, optionally with unit-l2 columns.
// grid P, 256 threads (Q <= 256: thread q owns row q).
template <int RT>
__global__ void __launch_bounds__(256)
    als_solve_kernel(const float *__restrict__ M, const float *__restrict__ F1,
                     const float *__restrict__ F2, float *__restrict__ F, int Q, int R,
                     int normalize, int *status) {
  __shared__ float g1[RT * RT], g2[RT * RT];
  __shared__ double Gd[RT * RT], Ld[RT * RT];
  __shared__ float Lf[RT * RT];
  __shared__ float red[8 * RT], out[RT];
  __shared__ int ok_s;
  const int p = blockIdx.x;
  const float *f1 = F1 + (int64_t)p * Q * RT, *f2 = F2 + (int64_t)p * Q * RT;
  for (int e = threadIdx.x; e < RT * RT; e += blockDim.x) {
    const int r = e / RT, s = e % RT;
    float a1 = 0.f, a2 = 0.f;
    if (r < R && s < R) {
      for (int q = 0; q < Q; ++q) {
        a1 = fmaf(f1[q * RT + r], f1[q * RT + s], a1);
        a2 = fmaf(f2[q * RT + r], f2[q * RT + s], a2);
      }
    }
    g1[e] = a1;
    g2[e] = a2;
  }
  __syncthreads();
  for (int e = threadIdx.x; e < RT * RT; e += blockDim.x) {
    Gd[e] = (double)g1[e] * (double)g2[e];
    Ld[e] = 0.0;
  }
  __syncthreads();
  if (threadIdx.x < 32) {
    bool ok = warp_cholesky<RT>(Gd, Ld, R);
    if (!ok) {
      // load the diagonal by 1e-12 * trace / R and retry once
      double tr = 0.0;
      for (int r = 0; r < R; ++r) tr += Gd[r * RT + r];
      const double add = 1e-12 * tr / R;
      if (threadIdx.x < R) Gd[threadIdx.x * RT + threadIdx.x] += add;
      for (int e = threadIdx.x; e < RT * RT; e += 32) Ld[e] = 0.0;
      __syncwarp();
      ok = warp_cholesky<RT>(Gd, Ld, R);
    }
    if (threadIdx.x == 0) ok_s = ok ? 1 : 0;
  }
  __syncthreads();
  if (!ok_s) {
    if (threadIdx.x == 0) atomicOr(status, kDevCholesky);
    for (int e = threadIdx.x; e < RT * RT; e += blockDim.x) Lf[e] = (e / RT == e % RT) ? 1.f : 0.f;
  } else {
    for (int e = threadIdx.x; e < RT * RT; e += blockDim.x) Lf[e] = (float)Ld[e];
  }
  __syncthreads();

  const int q = threadIdx.x;
  float f[RT];
#pragma unroll
  for (int r = 0; r < RT; ++r) f[r] = 0.f;
  if (q < Q) {
    const float *m = M + ((int64_t)p * Q + q) * RT;
    float y[RT];
#pragma unroll
    for (int i = 0; i < RT; ++i) {
      if (i < R) {
        float s = m[i];
#pragma unroll
        for (int k = 0; k < i; ++k) s = fmaf(-Lf[i * RT + k], y[k], s);
        y[i] = s / Lf[i * RT + i];
      } else {
        y[i] = 0.f;
      }
    }
#pragma unroll
    for (int i = RT - 1; i >= 0; --i) {
      if (i < R) {
        float s = y[i];
#pragma unroll
        for (int k = i + 1; k < RT; ++k)
          if (k < R) s = fmaf(-Lf[k * RT + i], f[k], s);
        f[i] = s / Lf[i * RT + i];
      }
    }
  }
  if (normalize) {
    float sq[RT];
#pragma unroll
    for (int r = 0; r < RT; ++r) sq[r] = f[r] * f[r];
    block_sum_rows<RT>(sq, red, out);
#pragma unroll
    for (int r = 0; r < RT; ++r) {
      const float n = sqrtf(out[r]);
      if (n > 0.f) f[r] = f[r] / n;
    }
  }
  if (q < Q) {
    float4 *o = reinterpret_cast<float4 *>(F + ((int64_t)p * Q + q) * RT);
#pragma unroll
    for (int r4 = 0; r4 < RT / 4; ++r4)
      o[r4] = make_float4(f[4 * r4], f[4 * r4 + 1], f[4 * r4 + 2], f[4 * r4 + 3]);
  }
}

// F_p = unit-l2 columns of the replica-p rows of PF (Qd x R), padded to RT.
template <int RT>
__global__ void __launch_bounds__(256)
    warm_start_kernel(const float *__restrict__ PF, int Q, int S, int R, float *__restrict__ F) {
  __shared__ float red[8 * RT], out[RT];
  const int p = blockIdx.x, q = threadIdx.x;
  float f[RT];
#pragma unroll
  for (int r = 0; r < RT; ++r) f[r] = 0.f;
  if (q < Q) {
    const int row = q < S ? q : S + p * (Q - S) + (q - S);
#pragma unroll
    for (int r = 0; r < RT; ++r)
      if (r < R) f[r] = PF[(int64_t)row * R + r];
  }
  float sq[RT];
#pragma unroll
  for (int r = 0; r < RT; ++r) sq[r] = f[r] * f[r];
  block_sum_rows<RT>(sq, red, out);
  if (q < Q) {
    float4 *o = reinterpret_cast<float4 *>(F + ((int64_t)p * Q + q) * RT);
#pragma unroll
    for (int r4 = 0; r4 < RT / 4; ++r4) {
      float v[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int r = 4 * r4 + u;
        const float n = sqrtf(out[r]);
        v[u] = n > 0.f ? f[r] / n : f[r];
      }
      o[r4] = make_float4(v[0], v[1], v[2], v[3]);
    }
  }
}

static int block_for(int Q) { return ((Q + 31) / 32) * 32; }

template <int RT>
static void als_run_t(const float *Y, int P, int Q, int R, int iters, AlsBuffers &b,
                      cudaStream_t st, const Marker &mk) {
  const int bq = block_for(Q);
  const size_t smem_h = (size_t)Q * RT * sizeof(float);
  const size_t smem_m2 = ((size_t)Q * RT + 9 * RT) * sizeof(float);
  cudaFuncSetAttribute(als_h_kernel<RT>, cudaFuncAttributeMaxDynamicSharedMemorySize, 64 * 1024);
  cudaFuncSetAttribute(als_m2_kernel<RT>, cudaFuncAttributeMaxDynamicSharedMemorySize, 64 * 1024);
  const dim3 gQP(Q, P);
  const dim3 gM3((Q * RT + 255) / 256, P);
  auto pass_h_m3_c = [&]() {
    mk(kStAlsPass, 1);
    als_h_kernel<RT><<<gQP, bq, smem_h, st>>>(Y, b.Bf, b.H, Q);
    mk(kStAlsPass, 0);
    mk(kStAlsSmall, 1);
    als_m3_kernel<RT><<<gM3, 256, 0, st>>>(b.H, b.Af, b.M, Q);
    als_solve_kernel<RT><<<P, 256, 0, st>>>(b.M, b.Af, b.Bf, b.Cf, Q, R, 0, b.status);
    mk(kStAlsSmall, 0);
    count_launch(); count_launch(); count_launch();
  };
  for (int it = 0; it < iters; ++it) {
    pass_h_m3_c();
    mk(kStAlsSmall, 1);
    als_m1_kernel<RT><<<gQP, 256, 0, st>>>(b.H, b.Cf, b.M, Q);
    als_solve_kernel<RT><<<P, 256, 0, st>>>(b.M, b.Bf, b.Cf, b.Af, Q, R, 1, b.status);
    mk(kStAlsSmall, 0);
    mk(kStAlsPass, 1);
    als_m2_kernel<RT><<<gQP, bq, smem_m2, st>>>(Y, b.Af, b.Cf, b.M, Q);
    mk(kStAlsPass, 0);
    mk(kStAlsSmall, 1);
    als_solve_kernel<RT><<<P, 256, 0, st>>>(b.M, b.Af, b.Cf, b.Bf, Q, R, 1, b.status);
    mk(kStAlsSmall, 0);
    count_launch(); count_launch(); count_launch(); count_launch();
  }
  pass_h_m3_c();
}

void als_run(const float *Y, int P, int Q, int R, int RT, int iters, AlsBuffers &b,
             cudaStream_t st, const Marker &mk) {
  if (RT == 8) als_run_t<8>(Y, P, Q, R, iters, b, st, mk);
  else if (RT == 16) als_run_t<16>(Y, P, Q, R, iters, b, st, mk);
  else als_run_t<32>(Y, P, Q, R, iters, b, st, mk);
}

void warm_start(const float *PF, int P, int Q, int S, int R, int RT, float *F,
                cudaStream_t st) {
  if (RT == 8) warm_start_kernel<8><<<P, 256, 0, st>>>(PF, Q, S, R, F);
  else if (RT == 16) warm_start_kernel<16><<<P, 256, 0, st>>>(PF, Q, S, R, F);
  else warm_start_kernel<32><<<P, 256, 0, st>>>(PF, Q, S, R, F);
  count_launch();
}

}  // namespace octen
