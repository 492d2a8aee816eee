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
// The R x R Gram Hadamard products are factored (L D L^T) in fp64 over four
// warps, the Grams and the triangular substitutions run in fp32 (k_solve.cuh).
#include <cstdlib>

#include "k_solve.cuh"

namespace octen {

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

// F_p = unit-l2 columns of the replica-p rows of PF (Qd x R), padded to RT,
// and its Gram.  grid P, 256 threads; dynamic smem Q * RT floats.
template <int RT>
__global__ void __launch_bounds__(256)
    warm_start_kernel(const float *__restrict__ PF, int Q, int S, int R, float *__restrict__ F,
                      float *__restrict__ Gout) {
  extern __shared__ __align__(16) float Fs[];
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
#pragma unroll
  for (int r = 0; r < RT; ++r) {
    const float n = sqrtf(out[r]);
    if (n > 0.f) f[r] = f[r] / n;
  }
  if (q < Q) {
    float4 *o = reinterpret_cast<float4 *>(F + ((int64_t)p * Q + q) * RT);
    float4 *os = reinterpret_cast<float4 *>(Fs + q * RT);
#pragma unroll
    for (int r4 = 0; r4 < RT / 4; ++r4) {
      const float4 v = make_float4(f[4 * r4], f[4 * r4 + 1], f[4 * r4 + 2], f[4 * r4 + 3]);
      o[r4] = v;
      os[r4] = v;
    }
  }
  __syncthreads();
  smem_gram<RT>(Fs, Q, Gout + (int64_t)p * RT * RT);
}

// ---------------------------------------------------------------------------
// Tensor-core path (bf16 / e4m3 modes): both passes of a sweep are GEMMs with
// K-major bf16 operands.
//   Xa[p][a][b][c] = bf16(X_p)          (rows (a, b), K = c)
//   Xc[p][c][a][b] = bf16(X_p)          (rows (c, a), K = b)
//   M3[c][r] = sum_a A[a][r] sum_b Xc[(c,a)][b] B[b][r]      (32 | Q: the a sum in
//              the GEMM's epilogue, per 32 rows; otherwise M3 = Xc . KR^T over
//              K = (a, b) with KR[r][(a,b)] = A[a][r] B[b][r])
//   Tc[(a,b)][r] = sum_c Xa[(a,b)][c] C[c][r]
//   M1[a][r] = sum_b Tc[(a,b)][r] B[b][r],  M2[b][r] = sum_a Tc[(a,b)][r] A[a][r]
// ---------------------------------------------------------------------------
// With Qp > Q the copies are those of X_p zero-padded to Qp x Qp x Qp (every
// index in [0, Qp), zero where one is >= Q): Xa[p][(a,b)][c] with (a,b) = a Qp
// + b, Xc[p][c][(a,b)].  grid (ceil(Qp / 32), ceil(Qp^2 / 32), P), 32 x 8 threads.
__global__ void bf16_layouts_kernel(const float *__restrict__ Y, int Q, int Qp,
                                    __nv_bfloat16 *__restrict__ Xa,
                                    __nv_bfloat16 *__restrict__ Xc) {
  __shared__ float tile[32][33];
  const int p = blockIdx.z;
  const int64_t QQ = (int64_t)Q * Q, QQp = (int64_t)Qp * Qp;
  const int64_t ab0 = (int64_t)blockIdx.y * 32;
  const int c0 = blockIdx.x * 32;
  const float *y = Y + (int64_t)p * QQ * Q;
  for (int yy = threadIdx.y; yy < 32; yy += 8) {
    const int64_t ab = ab0 + yy;
    const int c = c0 + threadIdx.x;
    const int a = (int)(ab / Qp), b = (int)(ab - (int64_t)a * Qp);
    float v = 0.f;
    if (ab < QQp && c < Qp) {
      if (a < Q && b < Q && c < Q) v = y[((int64_t)a * Q + b) * Q + c];
      Xa[(int64_t)p * QQp * Qp + ab * Qp + c] = __float2bfloat16_rn(v);
    }
    tile[yy][threadIdx.x] = v;
  }
  __syncthreads();
  for (int yy = threadIdx.y; yy < 32; yy += 8) {
    const int c = c0 + yy;
    const int64_t ab = ab0 + threadIdx.x;
    if (ab < QQp && c < Qp)
      Xc[(int64_t)p * QQp * Qp + (int64_t)c * QQp + ab] =
          __float2bfloat16_rn(tile[threadIdx.x][yy]);
  }
}

// KR[p][r][(a,b)] = bf16(A[a][r] B[b][r]) for r < NP (zero beyond the rank).
// One CTA per (r, replica) with columns r of A and B staged in shared memory;
// each thread writes 8 consecutive b of one a as a 16-byte store (Q % 8 == 0,
// Q <= 256), so a CTA streams its Q^2 outputs contiguously.
template <int RT>
__global__ void __launch_bounds__(256)
    kr_kernel(const float *__restrict__ Af, const float *__restrict__ Bf, int Q,
              __nv_bfloat16 *__restrict__ KR) {
  __shared__ __align__(16) float ac[256], bc[256];
  const int r = blockIdx.x, p = blockIdx.y, NP = gridDim.x;
  const int64_t QQ = (int64_t)Q * Q;
  for (int q = threadIdx.x; q < Q; q += blockDim.x) {
    ac[q] = r < RT ? Af[((int64_t)p * Q + q) * RT + r] : 0.f;
    bc[q] = r < RT ? Bf[((int64_t)p * Q + q) * RT + r] : 0.f;
  }
  __syncthreads();
  uint4 *out = reinterpret_cast<uint4 *>(KR + ((int64_t)p * NP + r) * QQ);
  const int nch = static_cast<int>(QQ / 8);
  for (int ch = threadIdx.x; ch < nch; ch += blockDim.x) {
    const int e = ch * 8, a = e / Q, b = e - a * Q;
    const float x = ac[a];
    const float4 b0 = *reinterpret_cast<const float4 *>(bc + b);
    const float4 b1 = *reinterpret_cast<const float4 *>(bc + b + 4);
    __align__(16) __nv_bfloat162 h[4] = {__floats2bfloat162_rn(x * b0.x, x * b0.y),
                           __floats2bfloat162_rn(x * b0.z, x * b0.w),
                           __floats2bfloat162_rn(x * b1.x, x * b1.y),
                           __floats2bfloat162_rn(x * b1.z, x * b1.w)};
    out[ch] = *reinterpret_cast<const uint4 *>(h);
  }
}

// M1[p][a][r] = sum_b Tc[p][(a,b)][r] B[p][b][r] and M2[p][b][r] = sum_a
// Tc[p][(a,b)][r] A[p][a][r], Tc in bf16.  A CTA of 256 threads owns 32
// column octets (256 / RT output rows of RT / 8 octets); thread (octet j < 32,
// slice s < 8) sums every 8th term of the reduction starting at s with 16-byte
// loads of Tc, and the 8 slice sums are added in shared memory in a fixed order.
//   kind 1 (M1): output row a, reduction over b: term b at Tc[(a, b)]
//   kind 2 (M2): output row b, reduction over a: term a at Tc[(a, b)]
template <int RT, int KIND>
__global__ void __launch_bounds__(256)
    tc_mred_kernel(const __nv_bfloat16 *__restrict__ Tc, const float *__restrict__ Fac, int Q,
                   float *__restrict__ M) {
  constexpr int OCT = RT / 8;            // column octets per output row
  constexpr int ROWS = 32 / OCT;         // output rows per CTA
  __shared__ float4 part[8][32][2];
  pdl_trigger();
  pdl_wait();   // the factor is the previous kernel's
  const int p = blockIdx.y;
  const int j = threadIdx.x & 31, sl = threadIdx.x >> 5;
  const int row = blockIdx.x * ROWS + j / OCT, r = 8 * (j % OCT);
  float acc[8];
#pragma unroll
  for (int e = 0; e < 8; ++e) acc[e] = 0.f;
  if (row < Q) {
    const __nv_bfloat16 *t = Tc + (int64_t)p * Q * Q * RT + r;
    const float *f = Fac + (int64_t)p * Q * RT + r;
#pragma unroll 8
    for (int k = sl; k < Q; k += 8) {
      const int64_t ab = KIND == 1 ? (int64_t)row * Q + k : (int64_t)k * Q + row;
      const uint4 raw = *reinterpret_cast<const uint4 *>(t + ab * RT);
      const __nv_bfloat162 *h = reinterpret_cast<const __nv_bfloat162 *>(&raw);
      const float4 w0 = *reinterpret_cast<const float4 *>(f + k * RT);
      const float4 w1 = *reinterpret_cast<const float4 *>(f + k * RT + 4);
      const float2 v0 = __bfloat1622float2(h[0]), v1 = __bfloat1622float2(h[1]);
      const float2 v2 = __bfloat1622float2(h[2]), v3 = __bfloat1622float2(h[3]);
      acc[0] = fmaf(v0.x, w0.x, acc[0]); acc[1] = fmaf(v0.y, w0.y, acc[1]);
      acc[2] = fmaf(v1.x, w0.z, acc[2]); acc[3] = fmaf(v1.y, w0.w, acc[3]);
      acc[4] = fmaf(v2.x, w1.x, acc[4]); acc[5] = fmaf(v2.y, w1.y, acc[5]);
      acc[6] = fmaf(v3.x, w1.z, acc[6]); acc[7] = fmaf(v3.y, w1.w, acc[7]);
    }
  }
  part[sl][j][0] = make_float4(acc[0], acc[1], acc[2], acc[3]);
  part[sl][j][1] = make_float4(acc[4], acc[5], acc[6], acc[7]);
  __syncthreads();
  if (sl == 0 && row < Q) {
    float4 s0 = part[0][j][0], s1 = part[0][j][1];
#pragma unroll
    for (int q = 1; q < 8; ++q) {
      const float4 u0 = part[q][j][0], u1 = part[q][j][1];
      s0.x += u0.x; s0.y += u0.y; s0.z += u0.z; s0.w += u0.w;
      s1.x += u1.x; s1.y += u1.y; s1.z += u1.z; s1.w += u1.w;
    }
    float4 *o = reinterpret_cast<float4 *>(M + ((int64_t)p * Q + row) * RT + r);
    o[0] = s0;
    o[1] = s1;
  }
}

// Ft[p][r][q] = bf16(F[p][q][r]) for r < NP (zero beyond RT): the transposed
// bf16 operand of a factor.  grid (ceil(Q / 256), P), 256 threads.
template <int RT>
__global__ void __launch_bounds__(256)
    factor_bf16_t_kernel(const float *__restrict__ F, int Q, int NP,
                         __nv_bfloat16 *__restrict__ Ft) {
  const int p = blockIdx.y, q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= Q) return;
  const float *f = F + ((int64_t)p * Q + q) * RT;
  for (int r = 0; r < NP; ++r)
    Ft[((int64_t)p * NP + r) * Q + q] = __float2bfloat16_rn(r < RT ? f[r] : 0.f);
}

static int block_for(int Q) { return ((Q + 31) / 32) * 32; }

// K atoms per stage the ALS GEMMs start from (the autotuner also tries the
// others): kAlsKAtoms, or OCTEN_ALS_KATOMS (1, 2 or 4), a debug setting that
// pins the configuration a profiler capture sees when the autotuner is off.
static int als_katoms() {
  const char *v = getenv("OCTEN_ALS_KATOMS");
  if (v && (v[0] == '1' || v[0] == '2' || v[0] == '4') && v[1] == 0) return v[0] - '0';
  return kAlsKAtoms;
}

// The M1 / M2 reduction, as a programmatic dependent of the previous kernel
// when `pdl` is set.
template <int RT, int KIND>
static void mred(dim3 grid, const __nv_bfloat16 *Tc, const float *Fac, int Q, float *M, bool pdl,
                 cudaStream_t st) {
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute attr[1];
  cfg.gridDim = grid;
  cfg.blockDim = dim3(256);
  cfg.stream = st;
  if (pdl) {
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
  }
  if (cudaLaunchKernelEx(&cfg, tc_mred_kernel<RT, KIND>, Tc, Fac, Q, M) != cudaSuccess) {
    cudaGetLastError();
    tc_mred_kernel<RT, KIND><<<grid, 256, 0, st>>>(Tc, Fac, Q, M);
  }
}

int als_factor_floats(int RT) {
  return RT == 8 ? factor_floats<8>() : (RT == 16 ? factor_floats<16>() : factor_floats<32>());
}

// Shared memory the tensor-core GEMMs leave free on every SM for the factor
// kernel (als_ldl_kernel, at most 26 KB with the per-block reservation).
constexpr int kLdlReserve = 28 * 1024;

// Forks the factor of an update onto b.side: L D L^T of Gnew * Gother into
// b.L (Gnew the Gram of the factor updated last, formed by its solve).
template <int RT>
static void factor_async(const float *Gnew, const float *Gother, int P, int R, AlsBuffers &b,
                         cudaStream_t st) {
  // runs beside the update's GEMM (or M2 reduction): the same on-chip split
  static const bool shared_split = (prefer_max_shared(als_ldl_kernel<RT>), true);
  (void)shared_split;
  cudaEventRecord(b.ev_fork, st);
  cudaStreamWaitEvent(b.side, b.ev_fork, 0);
  als_ldl_kernel<RT><<<P, 128, 0, b.side>>>(Gnew, Gother, R, b.L, b.status);
  count_launch();
  cudaEventRecord(b.ev_join, b.side);
}

// Joins the factor and solves: F = M (L D L^T)^-1 with M row q of replica p
// the sum over s < nsplit of M[s * split_stride + (p * Q + q) * row_stride].
// Clusters of up to 8 CTAs share a replica (at most 32 rows each, a multiple
// of 8); one CTA per replica if the cluster launch is refused.
template <int RT>
static void apply(const float *M, int nsplit, int64_t split_stride, int64_t row_stride, float *F,
                  __nv_bfloat16 *Ft, int NP, int P, int Q, int normalize, float *Gout,
                  AlsBuffers &b, cudaStream_t st, int segQ = 0) {
  cudaStreamWaitEvent(st, b.ev_join, 0);
  int cl = (Q + 31) / 32;
  if (cl > 8) cl = 8;
  const int rows = ((Q + cl - 1) / cl + 7) / 8 * 8;
  cl = (Q + rows - 1) / rows;
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute attr[2];
  cfg.gridDim = dim3(P * cl);
  cfg.blockDim = dim3(256);
  cfg.dynamicSmemBytes = (size_t)rows * RT * sizeof(float);
  cfg.stream = st;
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = cl;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  attr[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[1].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = b.pdl ? 2 : 1;
  if (cudaLaunchKernelEx(&cfg, als_apply_kernel<RT>, M, nsplit, split_stride, row_stride,
                         (const float *)b.L, F, Ft, NP, Q, rows, normalize, Gout,
                         segQ) != cudaSuccess) {
    cudaGetLastError();
    als_apply_kernel<RT><<<P, 256, (size_t)Q * RT * sizeof(float), st>>>(
        M, nsplit, split_stride, row_stride, b.L, F, Ft, NP, Q, Q, normalize, Gout, segQ);
  }
  count_launch();
}

// fp32 path: SIMT passes over X_p.
template <int RT>
static void als_run_simt(const float *Y, int P, int Q, int R, int iters, AlsBuffers &b,
                         cudaStream_t st, const Marker &mk) {
  const int bq = block_for(Q);
  const size_t smem_h = (size_t)Q * RT * sizeof(float);
  const size_t smem_m2 = ((size_t)Q * RT + 9 * RT) * sizeof(float);
  const dim3 gQP(Q, P);
  const dim3 gM3((Q * RT + 255) / 256, P);
  auto c_update = [&]() {
    factor_async<RT>(b.GB, b.GA, P, R, b, st);
    mk(kStAlsGemm, 1);
    als_h_kernel<RT><<<gQP, bq, smem_h, st>>>(Y, b.Bf, b.H, Q);
    count_launch();
    mk(kStAlsGemm, 0);
    mk(kStAlsAux, 1);
    als_m3_kernel<RT><<<gM3, 256, 0, st>>>(b.H, b.Af, b.M, Q);
    count_launch();
    mk(kStAlsAux, 0);
    mk(kStAlsSolve, 1);
    apply<RT>(b.M, 1, 0, RT, b.Cf, nullptr, 0, P, Q, 0, b.GC, b, st);
    mk(kStAlsSolve, 0);
  };
  for (int it = 0; it < iters; ++it) {
    c_update();
    factor_async<RT>(b.GC, b.GB, P, R, b, st);
    mk(kStAlsAux, 1);
    als_m1_kernel<RT><<<gQP, 256, 0, st>>>(b.H, b.Cf, b.M, Q);
    count_launch();
    mk(kStAlsAux, 0);
    mk(kStAlsSolve, 1);
    apply<RT>(b.M, 1, 0, RT, b.Af, nullptr, 0, P, Q, 1, b.GA, b, st);
    mk(kStAlsSolve, 0);
    factor_async<RT>(b.GA, b.GC, P, R, b, st);
    mk(kStAlsGemm, 1);
    als_m2_kernel<RT><<<gQP, bq, smem_m2, st>>>(Y, b.Af, b.Cf, b.M, Q);
    count_launch();
    mk(kStAlsGemm, 0);
    mk(kStAlsSolve, 1);
    apply<RT>(b.M, 1, 0, RT, b.Bf, nullptr, 0, P, Q, 1, b.GB, b, st);
    mk(kStAlsSolve, 0);
  }
  c_update();
}

// bf16 / e4m3 modes: both passes on tcgen05 (bf16 copies of X_p in two layouts).
template <int RT>
static bool als_run_tc(const float *Y, int P, int Q, int R, int iters, AlsBuffers &b,
                       cudaStream_t st, const Marker &mk) {
  const int NP = kAlsNP;
  const int64_t QQ = (int64_t)Q * Q;
  if (b.wait_first) cudaStreamWaitEvent(st, b.wait_first, 0);
  if (!b.layouts_ready) {
    mk(kStAlsAux, 1);
    bf16_layouts_kernel<<<dim3((Q + 31) / 32, (unsigned)((QQ + 31) / 32), P), dim3(32, 8), 0,
                          st>>>(Y, Q, Q, b.Xa, b.Xc);
    count_launch();
    mk(kStAlsAux, 0);
  }
  // M3 = Xc . KR^T (split over K = (a, b)), Tc = Xa . C
  TcStoreArgs m3{};
  m3.A = b.Xc; m3.a_inner = QQ; m3.a_rows = (int64_t)P * Q; m3.a_rows_per_z = Q;
  m3.B = b.KR; m3.b_inner = QQ; m3.b_rows = (int64_t)P * NP; m3.b_rows_per_z = NP;
  m3.M = Q; m3.N = RT; m3.K = (int)QQ; m3.BN = NP; m3.batch = P; m3.ksplit = b.ksplit;
  m3.D = b.Mparts; m3.s_split = (int64_t)P * Q * RT; m3.s_z = (int64_t)Q * RT; m3.s_m = RT;
  TcStoreArgs tc{};
  tc.A = b.Xa; tc.a_inner = Q; tc.a_rows = (int64_t)P * QQ; tc.a_rows_per_z = (int)QQ;
  tc.B = b.Ct; tc.b_inner = Q; tc.b_rows = (int64_t)P * NP; tc.b_rows_per_z = NP;
  tc.M = (int)QQ; tc.N = RT; tc.K = Q; tc.BN = NP; tc.batch = P; tc.ksplit = 1;
  // Tc is kept in bf16 (half the bytes; it fits the L2 for the M2 pass)
  __nv_bfloat16 *Th = reinterpret_cast<__nv_bfloat16 *>(b.H);
  tc.D = nullptr; tc.Dh = Th; tc.s_split = 0; tc.s_z = QQ * RT; tc.s_m = RT;
  tc.d_keep = true;   // Tc is read again by the M2 reduction
  // M1 fused into the Tc GEMM: per-warp partials over 32 consecutive b (in
  // two segments where a warp's rows cross from one a to the next, 32 not
  // dividing Q)
  const bool seg = Q % 32 != 0 && Q >= 32;
  const bool fuse_m1 = Q % 32 == 0 || seg;
  const int segQ = seg ? Q : 0;
  if (fuse_m1) {
    tc.m1_B = b.Bf; tc.m1_part = b.Mparts; tc.Q = Q; tc.RT = RT; tc.m1_seg = seg;
  }
  // the factor kernel of each update (about 25 KB of shared memory) runs
  // beside these GEMMs: leave it room
  m3.smem_reserve = tc.smem_reserve = kLdlReserve;
  // the bf16 copies of X_p stream through once per pass (evict-first), so Tc
  // stays in the L2 for the M2 pass
  m3.a_stream = tc.a_stream = true;
  m3.katoms = kAlsKAtoms;   // split-K: the split count below follows these atoms
  tc.katoms = als_katoms();
  m3.max_ctas = tc.max_ctas = b.max_ctas;
  m3.pdl = tc.pdl = b.pdl;
  const int ks = tc_gemm_splits(m3.K, b.ksplit, kAlsKAtoms);
  const dim3 gKR(NP, P);
  const dim3 gM((Q + 256 / RT - 1) / (256 / RT), P);   // 32 output octets per CTA
  // With Q >= 32 the M3 pass needs no Khatri-Rao operand: the GEMM contracts b,
  //   Tb[(c, a)][r] = sum_b Xc[(c, a)][b] B[b][r]   (B^T in bf16 as the B operand),
  // and its epilogue reduces every 32 consecutive a with weights A[a][r] in
  // fp32 (the fused reduction of the Tc pass, segmented where 32 does not
  // divide Q), so M3[c][r] = a sum of partials; Tb itself is never stored.
  const bool m3_fused = fuse_m1 && b.Bt != nullptr;
  TcStoreArgs m3f{};
  if (m3_fused) {
    m3f.A = b.Xc; m3f.a_inner = Q; m3f.a_rows = (int64_t)P * QQ; m3f.a_rows_per_z = (int)QQ;
    m3f.B = b.Bt; m3f.b_inner = Q; m3f.b_rows = (int64_t)P * NP; m3f.b_rows_per_z = NP;
    m3f.M = (int)QQ; m3f.N = RT; m3f.K = Q; m3f.BN = NP; m3f.batch = P; m3f.ksplit = 1;
    m3f.D = nullptr; m3f.Dh = nullptr; m3f.s_split = 0; m3f.s_z = 0; m3f.s_m = 0;
    m3f.m1_B = b.Af; m3f.m1_part = b.Mparts; m3f.Q = Q; m3f.RT = RT; m3f.m1_seg = seg;
    m3f.smem_reserve = kLdlReserve;
    m3f.a_stream = true;
    m3f.katoms = als_katoms();
    m3f.max_ctas = b.max_ctas;
    m3f.pdl = b.pdl;
    // B^T of the warm start; every later B update writes it from its solve
    mk(kStAlsAux, 1);
    factor_bf16_t_kernel<RT><<<dim3((Q + 255) / 256, P), 256, 0, st>>>(b.Bf, Q, NP, b.Bt);
    count_launch();
    mk(kStAlsAux, 0);
  }
  bool ok = true;
  bool first = true;
  auto c_update = [&]() {
    factor_async<RT>(b.GB, b.GA, P, R, b, st);
    if (m3_fused) {
      mk(kStAlsGemm, 1);
      ok = ok && tc_gemm_store(m3f, b.status, st);
      mk(kStAlsGemm, 0);
      if (first && b.ev_first) cudaEventRecord(b.ev_first, st);
      first = false;
      mk(kStAlsSolve, 1);
      apply<RT>(b.Mparts, Q / 32, RT, (int64_t)(Q / 32) * RT, b.Cf, b.Ct, NP, P, Q, 0, b.GC, b, st,
                segQ);
      mk(kStAlsSolve, 0);
      return;
    }
    mk(kStAlsAux, 1);
    kr_kernel<RT><<<gKR, 256, 0, st>>>(b.Af, b.Bf, Q, b.KR);
    count_launch();
    mk(kStAlsAux, 0);
    mk(kStAlsGemm, 1);
    ok = ok && tc_gemm_store(m3, b.status, st);
    mk(kStAlsGemm, 0);
    mk(kStAlsSolve, 1);
    apply<RT>(b.Mparts, ks, (int64_t)P * Q * RT, RT, b.Cf, b.Ct, NP, P, Q, 0, b.GC, b, st);
    mk(kStAlsSolve, 0);
  };
  for (int it = 0; it < iters && ok; ++it) {
    c_update();
    factor_async<RT>(b.GC, b.GB, P, R, b, st);
    mk(kStAlsGemm, 1);
    ok = ok && tc_gemm_store(tc, b.status, st);
    mk(kStAlsGemm, 0);
    if (fuse_m1) {
      mk(kStAlsSolve, 1);
      apply<RT>(b.Mparts, Q / 32, RT, (int64_t)(Q / 32) * RT, b.Af, nullptr, 0, P, Q, 1, b.GA, b, st,
                segQ);
      mk(kStAlsSolve, 0);
    } else {
      mk(kStAlsAux, 1);
      mred<RT, 1>(gM, Th, b.Bf, Q, b.M, b.pdl, st);
      count_launch();
      mk(kStAlsAux, 0);
      mk(kStAlsSolve, 1);
      apply<RT>(b.M, 1, 0, RT, b.Af, nullptr, 0, P, Q, 1, b.GA, b, st);
      mk(kStAlsSolve, 0);
    }
    factor_async<RT>(b.GA, b.GC, P, R, b, st);
    mk(kStAlsAux, 1);
    mred<RT, 2>(gM, Th, b.Af, Q, b.M, b.pdl, st);
    count_launch();
    mk(kStAlsAux, 0);
    mk(kStAlsSolve, 1);
    apply<RT>(b.M, 1, 0, RT, b.Bf, m3_fused ? b.Bt : nullptr, NP, P, Q, 1, b.GB, b, st);
    mk(kStAlsSolve, 0);
  }
  if (ok) c_update();
  return ok;
}

// The replicas in b.groups contiguous groups, each group's sweeps an
// independent chain of launches: group 0 on `st`, group g on b.gst[g] (forked
// from `st` and joined back at the end), each with its own factor stream and
// events, group g starting after group g - 1's first GEMM.  Every buffer is indexed by
// replica first with a stride that does not depend on P, so a group is the
// same buffers offset to its first replica; per replica the launches and their
// arithmetic are those of one group.
template <int RT>
static bool als_run_tc_groups(const float *Y, int P, int Q, int R, int iters, AlsBuffers &b,
                              cudaStream_t st) {
  const int G = b.groups;
  const char *sv = getenv("OCTEN_ALS_GROUP_SPLIT");
  const bool split_sms = sv && sv[0] == '1';
  int nsm = 0, dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  const int64_t QQ = (int64_t)Q * Q, Q3 = QQ * Q;
  // per-replica stride of the fused partials: Q^2 / 32 blocks of RT, or two
  // segment sums per block when 32 does not divide Q
  const int64_t mparts = (Q % 32 == 0 ? QQ / 32 : 2 * ((QQ + 31) / 32)) * RT;
  cudaEventRecord(b.gsplit, st);
  bool ok = true;
  for (int g = 0; g < G; ++g) {
    const int p0 = (int)((int64_t)g * P / G), p1 = (int)((int64_t)(g + 1) * P / G);
    AlsBuffers bg = b;
    bg.groups = 1;
    bg.Af = b.Af + (int64_t)p0 * Q * RT;
    bg.Bf = b.Bf + (int64_t)p0 * Q * RT;
    bg.Cf = b.Cf + (int64_t)p0 * Q * RT;
    bg.GA = b.GA + (int64_t)p0 * RT * RT;
    bg.GB = b.GB + (int64_t)p0 * RT * RT;
    bg.GC = b.GC + (int64_t)p0 * RT * RT;
    bg.M = b.M + (int64_t)p0 * Q * RT;
    // the bf16 Tc occupies the first half of H, [p][(a, b)][r]
    bg.H = reinterpret_cast<float *>(reinterpret_cast<__nv_bfloat16 *>(b.H) + p0 * QQ * RT);
    bg.Xa = b.Xa + p0 * Q3;
    bg.Xc = b.Xc + p0 * Q3;
    bg.KR = b.KR ? b.KR + (int64_t)p0 * kAlsNP * QQ : nullptr;
    bg.Ct = b.Ct + (int64_t)p0 * kAlsNP * Q;
    bg.Bt = b.Bt ? b.Bt + (int64_t)p0 * kAlsNP * Q : nullptr;
    bg.Mparts = b.Mparts + p0 * mparts;
    bg.L = b.L + (int64_t)p0 * als_factor_floats(RT);
    bg.side = g == 0 ? b.side : b.gside[g];
    bg.ev_fork = g == 0 ? b.ev_fork : b.gev_fork[g];
    bg.ev_join = g == 0 ? b.ev_join : b.gev_join[g];
    // every group's GEMMs on all SMs (a group's solves co-reside with the
    // next group's GEMM CTAs), or OCTEN_ALS_GROUP_SPLIT=1: SMs / groups each
    bg.max_ctas = split_sms ? (nsm / G > 0 ? nsm / G : 1) : 0;
    bg.wait_first = g > 0 ? b.gfirst[g - 1] : nullptr;
    bg.ev_first = g + 1 < G ? b.gfirst[g] : nullptr;
    cudaStream_t sg = g == 0 ? st : b.gst[g];
    if (g > 0) cudaStreamWaitEvent(sg, b.gsplit, 0);
    ok = als_run_tc<RT>(Y + p0 * Q3, p1 - p0, Q, R, iters, bg, sg, Marker{}) && ok;
    if (g > 0) cudaEventRecord(b.gdone[g], sg);
  }
  for (int g = 1; g < G; ++g) cudaStreamWaitEvent(st, b.gdone[g], 0);
  return ok;
}

// Q % 8 == 0, or Q >= 32 run zero-padded to the next multiple of 8 (below 32
// the replicas are small enough for the single-launch or split-K paths)
bool als_tc_eligible(int Q) { return (Q % 8 == 0 || Q >= 32) && tc_supported(); }

int als_tc_splits(int P, int Q, int desired) {
  (void)P;
  return tc_gemm_splits(Q * Q, desired, kAlsKAtoms);
}

// OCTEN_ALS_FUSED=0 keeps small replicas on the multi-launch path (used to
// cross-check the single-launch kernel).
static bool fused_wanted() {
  const char *v = getenv("OCTEN_ALS_FUSED");
  return !(v && v[0] == '0');
}

bool als_run(const float *Y, int P, int Q, int R, int RT, int iters, AlsBuffers &b,
             cudaStream_t st, const Marker &mk) {
  if (fused_wanted() && als_fused_fits(Q, RT)) {
    mk(kStAlsFused, 1);
    const bool ran = als_run_fused(Y, P, Q, R, RT, iters, b, st);
    mk(kStAlsFused, 0);
    if (ran) return true;
  }
  const int smem = (int)((size_t)Q * RT * sizeof(float));
  const int smem_ap = smem;   // the solve's rows (all Q without clusters)
  if (RT == 8) {
    cudaFuncSetAttribute(als_apply_kernel<8>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_ap);
  } else if (RT == 16) {
    cudaFuncSetAttribute(als_apply_kernel<16>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_ap);
  } else {
    cudaFuncSetAttribute(als_apply_kernel<32>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_ap);
  }
  if (b.use_tc && b.Qp > Q) {
    // zero-padded replicas: warm starts into the padded factors, the passes at
    // Qp, the factors back to Q rows (the padding rows stay zero)
    const int Qp = b.Qp;
    const size_t rowb = (size_t)Q * RT * sizeof(float), rowp = (size_t)Qp * RT * sizeof(float);
    mk(kStAlsAux, 1);
    cudaMemsetAsync(b.Af_pad, 0, rowp * P, st);
    cudaMemsetAsync(b.Bf_pad, 0, rowp * P, st);
    cudaMemsetAsync(b.Cf_pad, 0, rowp * P, st);
    cudaMemcpy2DAsync(b.Af_pad, rowp, b.Af, rowb, rowb, P, cudaMemcpyDeviceToDevice, st);
    cudaMemcpy2DAsync(b.Bf_pad, rowp, b.Bf, rowb, rowb, P, cudaMemcpyDeviceToDevice, st);
    const int64_t QQp = (int64_t)Qp * Qp;
    bf16_layouts_kernel<<<dim3((Qp + 31) / 32, (unsigned)((QQp + 31) / 32), P), dim3(32, 8), 0,
                          st>>>(Y, Q, Qp, b.Xa, b.Xc);
    count_launch();
    mk(kStAlsAux, 0);
    AlsBuffers bp = b;
    bp.Af = b.Af_pad; bp.Bf = b.Bf_pad; bp.Cf = b.Cf_pad;
    bp.Qp = 0;
    bp.layouts_ready = true;
    const bool ok = als_run(Y, P, Qp, R, RT, iters, bp, st, mk);
    mk(kStAlsAux, 1);
    cudaMemcpy2DAsync(b.Af, rowb, b.Af_pad, rowp, rowb, P, cudaMemcpyDeviceToDevice, st);
    cudaMemcpy2DAsync(b.Bf, rowb, b.Bf_pad, rowp, rowb, P, cudaMemcpyDeviceToDevice, st);
    cudaMemcpy2DAsync(b.Cf, rowb, b.Cf_pad, rowp, rowb, P, cudaMemcpyDeviceToDevice, st);
    mk(kStAlsAux, 0);
    return ok;
  }
  if (b.use_tc) {
    if (b.groups > 1 && !mk.fn && Q >= 32 && P >= b.groups) {
      if (RT == 8) return als_run_tc_groups<8>(Y, P, Q, R, iters, b, st);
      if (RT == 16) return als_run_tc_groups<16>(Y, P, Q, R, iters, b, st);
      return als_run_tc_groups<32>(Y, P, Q, R, iters, b, st);
    }
    if (RT == 8) return als_run_tc<8>(Y, P, Q, R, iters, b, st, mk);
    if (RT == 16) return als_run_tc<16>(Y, P, Q, R, iters, b, st, mk);
    return als_run_tc<32>(Y, P, Q, R, iters, b, st, mk);
  }
  cudaFuncSetAttribute(als_h_kernel<8>, cudaFuncAttributeMaxDynamicSharedMemorySize, 64 * 1024);
  cudaFuncSetAttribute(als_h_kernel<16>, cudaFuncAttributeMaxDynamicSharedMemorySize, 64 * 1024);
  cudaFuncSetAttribute(als_h_kernel<32>, cudaFuncAttributeMaxDynamicSharedMemorySize, 64 * 1024);
  cudaFuncSetAttribute(als_m2_kernel<8>, cudaFuncAttributeMaxDynamicSharedMemorySize, 64 * 1024);
  cudaFuncSetAttribute(als_m2_kernel<16>, cudaFuncAttributeMaxDynamicSharedMemorySize, 64 * 1024);
  cudaFuncSetAttribute(als_m2_kernel<32>, cudaFuncAttributeMaxDynamicSharedMemorySize, 64 * 1024);
  if (RT == 8) als_run_simt<8>(Y, P, Q, R, iters, b, st, mk);
  else if (RT == 16) als_run_simt<16>(Y, P, Q, R, iters, b, st, mk);
  else als_run_simt<32>(Y, P, Q, R, iters, b, st, mk);
  return true;
}

void warm_start(const float *PF, int P, int Q, int S, int R, int RT, float *F, float *G,
                cudaStream_t st) {
  const size_t smem = (size_t)Q * RT * sizeof(float);
  if (RT == 8) warm_start_kernel<8><<<P, 256, smem, st>>>(PF, Q, S, R, F, G);
  else if (RT == 16) warm_start_kernel<16><<<P, 256, smem, st>>>(PF, Q, S, R, F, G);
  else {
    cudaFuncSetAttribute(warm_start_kernel<32>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)smem);
    warm_start_kernel<32><<<P, 256, smem, st>>>(PF, Q, S, R, F, G);
  }
  count_launch();
}

}  // namespace octen
