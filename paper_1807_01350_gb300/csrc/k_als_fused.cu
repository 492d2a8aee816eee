// Replica CP-ALS for small replicas in a single launch (Algorithm 1's
// CP(X_p, R) step, the same sweeps as k_als.cu): one CTA per replica keeps X_p
// (Q³ fp32), the pass-1 product H = X_p ×2 B, the factors, their Grams and the
// factor of the current normal equations in shared memory and runs every sweep
// without leaving the kernel.  For small Q the separate-launch form is bound by
// launch latency (about ten launches per sweep); here the fp64 L D L^T of each
// update (warps 0..3, the same device code as als_ldl_kernel) runs while
// warps 4..7 form the update's MTTKRP, and the whole CP costs one launch.
#include "k_solve.cuh"

namespace octen {

namespace {

constexpr int kFusedThreads = 256;

// Shared floats: X Q³ (rounded up to a multiple of 4, so that every later
// array starts 16-byte aligned for the vector loads) | H Q²·RT | A, B, C, M
// Q·RT each | GA, GB, GC, Lc, Lr RT² each | rf RT | red 8·RT | scale RT.
// RT is a multiple of 8, so only X needs the rounding.
__host__ __device__ inline size_t fused_x_floats(int Q) {
  return ((size_t)Q * Q * Q + 3) & ~size_t(3);
}
size_t fused_floats(int Q, int RT) {
  const size_t q = (size_t)Q;
  return fused_x_floats(Q) + q * q * RT + 4 * q * RT + 5 * (size_t)RT * RT + 10 * (size_t)RT;
}

__device__ __forceinline__ void mttkrp_barrier() {
  asm volatile("bar.sync 2, 128;" ::: "memory");
}

// grid P, 256 threads (Q <= 256); dynamic smem fused_floats(Q, RT) floats.
// In: X_p (Y), the warm-started A, B (unit columns, rank padded to RT with
// zeros) and their Grams.  Out: the replica factors A, B, C.
template <int RT>
__global__ void __launch_bounds__(kFusedThreads, 1)
    als_fused_kernel(const float *__restrict__ Y, int Q, int R, int iters, float *At, float *Bt,
                     float *Ct, const float *__restrict__ GAin, const float *__restrict__ GBin,
                     int *status) {
  extern __shared__ __align__(16) float sm[];
  __shared__ double Craw[RT * (RT + 1)], Rs[RT];
  __shared__ int fail_s;
  const int p = blockIdx.x, tid = threadIdx.x;
  const int QQ = Q * Q;
  float *X = sm;                        // [a][b][c]
  float *H = X + fused_x_floats(Q);     // [a][c][r]
  float *A = H + (size_t)QQ * RT;       // [q][r]
  float *B = A + Q * RT;
  float *C = B + Q * RT;
  float *M = C + Q * RT;
  float *GA = M + Q * RT, *GB = GA + RT * RT, *GC = GB + RT * RT;
  float *Lc = GC + RT * RT, *Lr = Lc + RT * RT, *rf = Lr + RT * RT;
  float *red = rf + RT, *scl = red + 8 * RT;

  const float *yp = Y + (size_t)p * QQ * Q;
  for (int e = tid; e < QQ * Q; e += blockDim.x) X[e] = yp[e];
  for (int e = tid; e < Q * RT; e += blockDim.x) {
    A[e] = At[(size_t)p * Q * RT + e];
    B[e] = Bt[(size_t)p * Q * RT + e];
  }
  for (int e = tid; e < RT * RT; e += blockDim.x) {
    GA[e] = GAin[(size_t)p * RT * RT + e];
    GB[e] = GBin[(size_t)p * RT * RT + e];
  }
  __syncthreads();
  const int u = tid - 128;   // MTTKRP thread index (warps 4..7)

  // C = M3 (GA * GB)^-1,  M3[c][r] = sum_a A[a][r] H[a][c][r],  H = X ×2 B
  auto c_update = [&]() {
    if (tid < 128) {
      ldl_factor<RT>(GA, GB, R, Craw, Rs, Lc, Lr, rf, &fail_s);
    } else {
      for (int e = u; e < QQ * RT; e += 128) {
        const int a = e / (Q * RT), rem = e - a * (Q * RT), c = rem / RT, r = rem - c * RT;
        const float *x = X + (size_t)a * QQ + c;
        float acc = 0.f;
        for (int b = 0; b < Q; ++b) acc = fmaf(x[b * Q], B[b * RT + r], acc);
        H[e] = acc;
      }
      mttkrp_barrier();
      for (int e = u; e < Q * RT; e += 128) {
        const int c = e / RT, r = e - c * RT;
        float acc = 0.f;
        for (int a = 0; a < Q; ++a) acc = fmaf(A[a * RT + r], H[((size_t)a * Q + c) * RT + r], acc);
        M[e] = acc;
      }
    }
    __syncthreads();
    if (fail_s && tid == 0) atomicOr(status, kDevCholesky);
    solve_rows_smem<RT>(M, C, Q, false, Lc, Lr, rf, red, scl);
    __syncthreads();
    smem_gram<RT>(C, Q, GC);
    __syncthreads();
  };

  for (int it = 0; it < iters; ++it) {
    c_update();
    // A = M1 (GB * GC)^-1 normalised,  M1[a][r] = sum_c C[c][r] H[a][c][r]
    if (tid < 128) {
      ldl_factor<RT>(GB, GC, R, Craw, Rs, Lc, Lr, rf, &fail_s);
    } else {
      for (int e = u; e < Q * RT; e += 128) {
        const int a = e / RT, r = e - a * RT;
        const float *h = H + (size_t)a * Q * RT + r;
        float acc = 0.f;
        for (int c = 0; c < Q; ++c) acc = fmaf(C[c * RT + r], h[c * RT], acc);
        M[e] = acc;
      }
    }
    __syncthreads();
    if (fail_s && tid == 0) atomicOr(status, kDevCholesky);
    solve_rows_smem<RT>(M, A, Q, true, Lc, Lr, rf, red, scl);
    __syncthreads();
    smem_gram<RT>(A, Q, GA);
    __syncthreads();
    // B = M2 (GA * GC)^-1 normalised,  M2[b][r] = sum_a A[a][r] sum_c X[a][b][c] C[c][r]
    if (tid < 128) {
      ldl_factor<RT>(GA, GC, R, Craw, Rs, Lc, Lr, rf, &fail_s);
    } else {
      for (int e = u; e < Q * RT; e += 128) {
        const int b = e / RT, r = e - b * RT;
        float acc = 0.f;
        for (int a = 0; a < Q; ++a) {
          const float *x = X + ((size_t)a * Q + b) * Q;
          float t = 0.f;
          for (int c = 0; c < Q; ++c) t = fmaf(x[c], C[c * RT + r], t);
          acc = fmaf(A[a * RT + r], t, acc);
        }
        M[e] = acc;
      }
    }
    __syncthreads();
    if (fail_s && tid == 0) atomicOr(status, kDevCholesky);
    solve_rows_smem<RT>(M, B, Q, true, Lc, Lr, rf, red, scl);
    __syncthreads();
    smem_gram<RT>(B, Q, GB);
    __syncthreads();
  }
  c_update();
  for (int e = tid; e < Q * RT; e += blockDim.x) {
    At[(size_t)p * Q * RT + e] = A[e];
    Bt[(size_t)p * Q * RT + e] = B[e];
    Ct[(size_t)p * Q * RT + e] = C[e];
  }
}

constexpr size_t kFusedSmemLimit = 200 * 1024;

}  // namespace

bool als_fused_fits(int Q, int RT) {
  return Q <= kFusedThreads && fused_floats(Q, RT) * sizeof(float) <= kFusedSmemLimit;
}

bool als_run_fused(const float *Y, int P, int Q, int R, int RT, int iters, AlsBuffers &b,
                   cudaStream_t st) {
  if (!als_fused_fits(Q, RT)) return false;
  const size_t smem = fused_floats(Q, RT) * sizeof(float);
  cudaError_t e;
  if (RT == 8) {
    cudaFuncSetAttribute(als_fused_kernel<8>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)smem);
    als_fused_kernel<8><<<P, kFusedThreads, smem, st>>>(Y, Q, R, iters, b.Af, b.Bf, b.Cf, b.GA,
                                                        b.GB, b.status);
  } else if (RT == 16) {
    cudaFuncSetAttribute(als_fused_kernel<16>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)smem);
    als_fused_kernel<16><<<P, kFusedThreads, smem, st>>>(Y, Q, R, iters, b.Af, b.Bf, b.Cf, b.GA,
                                                         b.GB, b.status);
  } else {
    cudaFuncSetAttribute(als_fused_kernel<32>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)smem);
    als_fused_kernel<32><<<P, kFusedThreads, smem, st>>>(Y, Q, R, iters, b.Af, b.Bf, b.Cf, b.GA,
                                                         b.GB, b.status);
  }
  e = cudaGetLastError();
  if (e != cudaSuccess) return false;
  count_launch();
  return true;
}

}  // namespace octen
