// Dense CP-ALS of the existing tensor, for an init without a supplied
// decomposition (the paper assumes one exists, Sec. "Problem Formulation";
// this computes it).  X_old is [k][i][j] (t_old x I x J) and the model is
// X_old[k][i][j] = sum_r A[i][r] B[j][r] C[k][r]; the sweeps are those of the
// replica CP-ALS: C, then A, then B by the normal equations with the Hadamard
// product of Grams, A and B normalised to unit l2, a final C update.
//
// MTTKRPs (dimension tree, two passes over X_old per sweep):
//   T[k][i][r] = sum_j X[k][i][j] B[j][r]     M_C[k] = sum_i A[i] T[k][i]   M_A[i] = sum_k C[k] T[k][i]
//   U[k][j][r] = sum_i X[k][i][j] A[i][r]     M_B[j] = sum_k C[k] U[k][j]
// T and U are fp32-accumulate GEMMs on the SIMT kernels (any element type of
// X_old); the R x R solves use the fp64 L D L^T device code of the replica ALS
// with the rows of a factor spread over many CTAs.
#include "k_solve.cuh"

namespace octen {

namespace {

// out[row][r] = sum_{t < nterms} T[row * s_row + t * s_t + r] * F[t][r]   (F is [t][RT])
template <int RT>
__global__ void __launch_bounds__(256)
    dense_reduce_kernel(const float *__restrict__ T, int64_t s_row, int64_t s_t, int nrows,
                        int nterms, const float *__restrict__ F, float *__restrict__ out) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= (int64_t)nrows * RT) return;
  const int64_t row = e / RT;
  const int r = (int)(e - row * RT);
  const float *t = T + row * s_row + r;
  float acc = 0.f;
  for (int k = 0; k < nterms; ++k) acc = fmaf(t[k * s_t], F[k * RT + r], acc);
  out[e] = acc;
}

// One CTA: L D L^T of G1 * G2 into Lout (packed as for the replica solve).
template <int RT>
__global__ void __launch_bounds__(128)
    dense_factor_kernel(const float *__restrict__ G1, const float *__restrict__ G2, int R,
                        float *__restrict__ Lout, int *status) {
  __shared__ double Craw[RT * (RT + 1)], Rs[RT];
  __shared__ __align__(16) float Lc[RT * RT], Lr[RT * RT], rf[RT];
  __shared__ int fail_s;
  ldl_factor<RT>(G1, G2, R, Craw, Rs, Lc, Lr, rf, &fail_s);
  __syncthreads();
  if (fail_s && threadIdx.x == 0) atomicOr(status, kDevCholesky);
  for (int e = threadIdx.x; e < RT * RT; e += blockDim.x) {
    Lout[e] = Lc[e];
    Lout[RT * RT + e] = Lr[e];
  }
  if (threadIdx.x < RT) Lout[2 * RT * RT + threadIdx.x] = rf[threadIdx.x];
}

// Rows of F (256 per CTA): F[q] = M[q] (L D L^T)^-1, or, with M == nullptr,
// F[q] = F0[q] (R columns, padded to RT with zeros).  With `part`, the CTA's
// column sums of squares go to part[blockIdx.x][RT].
template <int RT>
__global__ void __launch_bounds__(256)
    dense_rows_kernel(const float *__restrict__ M, const float *__restrict__ F0, int R, int nrows,
                      const float *__restrict__ Lin, float *__restrict__ F, float *part) {
  __shared__ __align__(16) float Lc[RT * RT], Lr[RT * RT], rf[RT];
  __shared__ float red[8 * RT], out[RT];
  const int tid = threadIdx.x;
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + tid;
  const bool own = q < nrows;
  float y[RT];
#pragma unroll
  for (int r = 0; r < RT; ++r) y[r] = 0.f;
  if (M) {
    for (int e = tid; e < RT * RT; e += blockDim.x) {
      Lc[e] = Lin[e];
      Lr[e] = Lin[RT * RT + e];
    }
    if (tid < RT) rf[tid] = Lin[2 * RT * RT + tid];
    __syncthreads();
    if (own) {
#pragma unroll
      for (int r = 0; r < RT; ++r) y[r] = M[q * RT + r];
      ldl_substitute<RT>(y, Lc, Lr, rf);
    }
  } else if (own) {
#pragma unroll
    for (int r = 0; r < RT; ++r) y[r] = r < R ? F0[q * R + r] : 0.f;
  }
  if (own) {
#pragma unroll
    for (int r = 0; r < RT; ++r) F[q * RT + r] = y[r];
  }
  if (part) {
    float sq[RT];
#pragma unroll
    for (int r = 0; r < RT; ++r) sq[r] = y[r] * y[r];
    block_sum_rows<RT>(sq, red, out);
    if (tid < RT) part[(int64_t)blockIdx.x * RT + tid] = out[tid];
  }
}

// F[q][r] /= ||F[:, r]|| with the norms summed from nparts partial sums in a
// fixed order (every CTA the same order); a zero column is left as it is.
template <int RT>
__global__ void __launch_bounds__(256)
    dense_scale_kernel(float *__restrict__ F, int nrows, const float *__restrict__ part,
                       int nparts) {
  __shared__ float inv[RT];
  if (threadIdx.x < RT) {
    float s = 0.f;
    for (int c = 0; c < nparts; ++c) s += part[c * RT + threadIdx.x];
    const float n = sqrtf(s);
    inv[threadIdx.x] = n > 0.f ? 1.f / n : 1.f;
  }
  __syncthreads();
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e < (int64_t)nrows * RT) F[e] *= inv[e % RT];
}

// F (rows x R, compact) <- Fp (rows x RT, padded)
__global__ void unpad_kernel(const float *__restrict__ Fp, int64_t rows, int R, int RT,
                             float *__restrict__ F) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= rows * R) return;
  const int64_t q = e / R;
  F[e] = Fp[q * RT + (e - q * R)];
}

unsigned blocks(int64_t n, int per = 256) { return (unsigned)((n + per - 1) / per); }

// ---------------------------------------------------------------------------
// N-way form (the higher-order extension, Sec. "Extending to Higher-Order
// Tensors"): X_old is [k][i_1]...[i_nm], mode 0 the time mode k, mode m >= 1
// the non-temporal mode i_m.  The mode-n MTTKRP
//   M[i][r] = sum over every element with index i in mode n of
//             x * prod_{m != n} F_m[index in mode m][r]
// is one pass over X_old: CTA (i, split) walks the split's share of the
// elements of row i (the other modes' indices decoded from one counter, the
// innermost varying fastest, so a warp reads consecutive elements unless n
// is the innermost mode), each thread accumulating RT sums; the CTA sums its
// threads in a fixed order and a second kernel sums the splits in order.
struct NDenseShape {
  const float *F[kMaxNModes];   // factors, [rows][RT]
  int64_t dim[kMaxNModes];      // extent of every mode (mode 0: time)
  int64_t stride[kMaxNModes];   // element stride of every mode in X_old
  int NN;
};

template <int RT, Elem XT>
__global__ void __launch_bounds__(256)
    nmttkrp_kernel(const void *__restrict__ X, const NDenseShape sh, int mode, int64_t per,
                   float *__restrict__ part) {
  __shared__ float red[8 * RT], out[RT];
  const int64_t row = blockIdx.x;
  const int split = blockIdx.y, nsplit = gridDim.y;
  const int64_t others = [&] {
    int64_t n = 1;
    for (int m = 0; m < sh.NN; ++m)
      if (m != mode) n *= sh.dim[m];
    return n;
  }();
  const int64_t o0 = (int64_t)split * per;
  const int64_t o1 = o0 + per < others ? o0 + per : others;
  float acc[RT];
#pragma unroll
  for (int r = 0; r < RT; ++r) acc[r] = 0.f;
  for (int64_t o = o0 + threadIdx.x; o < o1; o += blockDim.x) {
    int64_t rem = o, off = row * sh.stride[mode];
    float w[RT];
#pragma unroll
    for (int r = 0; r < RT; ++r) w[r] = 1.f;
    for (int m = sh.NN - 1; m >= 0; --m) {
      if (m == mode) continue;
      const int64_t idx = rem % sh.dim[m];
      rem /= sh.dim[m];
      off += idx * sh.stride[m];
      const float4 *f = reinterpret_cast<const float4 *>(sh.F[m] + idx * RT);
#pragma unroll
      for (int r4 = 0; r4 < RT / 4; ++r4) {
        const float4 v = __ldg(f + r4);
        w[4 * r4] *= v.x; w[4 * r4 + 1] *= v.y; w[4 * r4 + 2] *= v.z; w[4 * r4 + 3] *= v.w;
      }
    }
    const float x = XT == Elem::BF16
                        ? __bfloat162float(static_cast<const __nv_bfloat16 *>(X)[off])
                        : __ldg(static_cast<const float *>(X) + off);
#pragma unroll
    for (int r = 0; r < RT; ++r) acc[r] = fmaf(x, w[r], acc[r]);
  }
  block_sum_rows<RT>(acc, red, out);
  if (threadIdx.x < RT) part[(row * nsplit + split) * RT + threadIdx.x] = out[threadIdx.x];
}

// M[row][r] = sum over the splits, in order
template <int RT>
__global__ void nsplit_sum_kernel(const float *__restrict__ part, int64_t rows, int nsplit,
                                  float *__restrict__ M) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= rows * RT) return;
  const int64_t row = e / RT;
  const int r = (int)(e - row * RT);
  float s = 0.f;
  for (int k = 0; k < nsplit; ++k) s += part[(row * nsplit + k) * RT + r];
  M[e] = s;
}

// out = elementwise product of the Grams of every mode but `skip1` and `skip2`
// (RT x RT each; all ones if there is none)
struct NGrams {
  const float *G[kMaxNModes];
};

template <int RT>
__global__ void gram_product_kernel(const NGrams g, int NN, int skip1, int skip2,
                                    float *__restrict__ out) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= RT * RT) return;
  float v = 1.f;
  for (int m = 0; m < NN; ++m)
    if (m != skip1 && m != skip2) v *= g.G[m][e];
  out[e] = v;
}

template <int RT>
struct DenseCp {
  const void *X;
  Elem xt;
  int64_t K, I, J;
  int R;
  float *A, *B, *C, *T, *U, *M, *GA, *GB, *GC, *L, *part;
  float *splitk;
  size_t splitk_floats;
  int *status;
  cudaStream_t st;

  void gram(const float *F, int64_t rows, float *G) const {
    GemmArgs g{};
    g.A = F; g.ta = Elem::F32; g.sAm = 1; g.sAk = RT;
    g.B = F; g.tb = Elem::F32; g.sBn = 1; g.sBk = RT;
    g.D = G; g.sDm = RT; g.sDn = 1;
    g.M = RT; g.N = RT; g.K = (int)rows; g.batch = 1; g.alpha = 1.f; g.beta = 0.f;
    g.split_scratch = splitk; g.split_scratch_floats = splitk_floats;
    gemm_strided(g, st);
  }
  // F (rows) = M (G1 * G2)^-1, normalised if asked; then its Gram into Gout
  void solve(float *F, int64_t rows, const float *G1, const float *G2, bool normalize,
             float *Gout) const {
    dense_factor_kernel<RT><<<1, 128, 0, st>>>(G1, G2, R, L, status);
    count_launch();
    const unsigned nb = blocks(rows);
    dense_rows_kernel<RT><<<nb, 256, 0, st>>>(M, nullptr, R, (int)rows, L, F,
                                              normalize ? part : nullptr);
    count_launch();
    if (normalize) {
      dense_scale_kernel<RT><<<blocks(rows * RT), 256, 0, st>>>(F, (int)rows, part, (int)nb);
      count_launch();
    }
    gram(F, rows, Gout);
  }
  void unit_columns(const float *F0, int64_t rows, float *F, float *G) const {
    const unsigned nb = blocks(rows);
    dense_rows_kernel<RT><<<nb, 256, 0, st>>>(nullptr, F0, R, (int)rows, nullptr, F, part);
    count_launch();
    dense_scale_kernel<RT><<<blocks(rows * RT), 256, 0, st>>>(F, (int)rows, part, (int)nb);
    count_launch();
    gram(F, rows, G);
  }
  // T[k][i][r] = sum_j X[k][i][j] B[j][r]
  void pass_T() const {
    GemmArgs g{};
    g.A = X; g.ta = xt; g.sAm = J; g.sAk = 1;
    g.B = B; g.tb = Elem::F32; g.sBn = 1; g.sBk = RT;
    g.D = T; g.sDm = RT; g.sDn = 1;
    g.M = (int)(K * I); g.N = RT; g.K = (int)J; g.batch = 1; g.alpha = 1.f; g.beta = 0.f;
    g.split_scratch = splitk; g.split_scratch_floats = splitk_floats;
    gemm_strided(g, st);
  }
  // U[k][j][r] = sum_i X[k][i][j] A[i][r]   (one GEMM per k)
  void pass_U() const {
    GemmArgs g{};
    g.A = X; g.ta = xt; g.sAz = I * J; g.sAm = 1; g.sAk = J;
    g.B = A; g.tb = Elem::F32; g.sBz = 0; g.sBn = 1; g.sBk = RT;
    g.D = U; g.sDz = J * RT; g.sDm = RT; g.sDn = 1;
    g.M = (int)J; g.N = RT; g.K = (int)I; g.batch = (int)K; g.alpha = 1.f; g.beta = 0.f;
    gemm_strided(g, st);
  }
  void reduce(const float *src, int64_t s_row, int64_t s_t, int64_t nrows, int64_t nterms,
              const float *F) const {
    dense_reduce_kernel<RT><<<blocks(nrows * RT), 256, 0, st>>>(src, s_row, s_t, (int)nrows,
                                                                (int)nterms, F, M);
    count_launch();
  }
  void c_update() const {
    pass_T();
    reduce(T, I * RT, RT, K, I, A);                 // M_C[k] = sum_i A[i] T[k][i]
    solve(C, K, GA, GB, false, GC);
  }
  void run(const float *A0, const float *B0, int iters) const {
    unit_columns(A0, I, A, GA);
    unit_columns(B0, J, B, GB);
    for (int it = 0; it < iters; ++it) {
      c_update();
      reduce(T, RT, I * RT, I, K, C);               // M_A[i] = sum_k C[k] T[k][i]
      solve(A, I, GB, GC, true, GA);
      pass_U();
      reduce(U, RT, J * RT, J, K, C);               // M_B[j] = sum_k C[k] U[k][j]
      solve(B, J, GA, GC, true, GB);
    }
    c_update();
  }
};

template <int RT>
void run_dense(const DenseCpArgs &a) {
  DenseCp<RT> d{a.X, a.xt, a.K, a.I, a.J, a.R,
                a.work, a.work + a.I * RT, a.work + (a.I + a.J) * RT,
                nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr,
                a.splitk, a.splitk_floats, a.status, a.st};
  float *w = a.work + (a.I + a.J + a.K) * RT;
  d.T = w; w += a.K * a.I * RT;
  d.U = w; w += a.K * a.J * RT;
  const int64_t mx = a.I > a.J ? (a.I > a.K ? a.I : a.K) : (a.J > a.K ? a.J : a.K);
  d.M = w; w += mx * RT;
  d.GA = w; w += RT * RT;
  d.GB = w; w += RT * RT;
  d.GC = w; w += RT * RT;
  d.L = w; w += factor_floats<RT>();
  d.part = w;
  d.run(a.A0, a.B0, a.iters);
  unpad_kernel<<<blocks(a.I * a.R), 256, 0, a.st>>>(d.A, a.I, a.R, RT, a.A_out);
  unpad_kernel<<<blocks(a.J * a.R), 256, 0, a.st>>>(d.B, a.J, a.R, RT, a.B_out);
  unpad_kernel<<<blocks(a.K * a.R), 256, 0, a.st>>>(d.C, a.K, a.R, RT, a.C_out);
  count_launch();
  count_launch();
  count_launch();
}

constexpr size_t kNSplitkFloats = size_t(1) << 20;   // Gram split-K scratch

int64_t n_mpart_rows(int64_t maxdim) { return maxdim + 304; }

// The N-way sweeps of the replica CP-ALS reading (time mode first, then every
// non-temporal mode in order, normalised; a final time update), each update
// F_n = M_n (Hadamard product of the other modes' Grams)^-1 with the fp64
// L D L^T of the replica solve.
template <int RT>
struct DenseCpN {
  const void *X;
  Elem xt;
  int NN, R;
  int64_t dim[kMaxNModes], stride[kMaxNModes], total;
  float *F[kMaxNModes], *G[kMaxNModes];
  float *M, *Hp, *L, *part, *mpart, *splitk;
  int *status;
  cudaStream_t st;

  void gram(const float *Fm, int64_t rows, float *Gm) const {
    GemmArgs g{};
    g.A = Fm; g.ta = Elem::F32; g.sAm = 1; g.sAk = RT;
    g.B = Fm; g.tb = Elem::F32; g.sBn = 1; g.sBk = RT;
    g.D = Gm; g.sDm = RT; g.sDn = 1;
    g.M = RT; g.N = RT; g.K = (int)rows; g.batch = 1; g.alpha = 1.f; g.beta = 0.f;
    g.split_scratch = splitk; g.split_scratch_floats = kNSplitkFloats;
    gemm_strided(g, st);
  }
  void mttkrp(int mode) const {
    NDenseShape sh{};
    for (int m = 0; m < NN; ++m) {
      sh.F[m] = F[m];
      sh.dim[m] = dim[m];
      sh.stride[m] = stride[m];
    }
    sh.NN = NN;
    const int64_t rows = dim[mode], others = total / rows;
    int64_t nsplit = (304 + rows - 1) / rows;          // about two CTAs per SM
    if (nsplit > others / 256) nsplit = others / 256;  // at least a CTA's worth each
    if (nsplit < 1) nsplit = 1;
    const int64_t per = (others + nsplit - 1) / nsplit;
    const dim3 grid((unsigned)rows, (unsigned)nsplit);
    if (xt == Elem::BF16)
      nmttkrp_kernel<RT, Elem::BF16><<<grid, 256, 0, st>>>(X, sh, mode, per, mpart);
    else
      nmttkrp_kernel<RT, Elem::F32><<<grid, 256, 0, st>>>(X, sh, mode, per, mpart);
    count_launch();
    nsplit_sum_kernel<RT><<<blocks(rows * RT), 256, 0, st>>>(mpart, rows, (int)nsplit, M);
    count_launch();
  }
  void update(int mode, bool normalize) const {
    mttkrp(mode);
    const int last = mode == NN - 1 ? NN - 2 : NN - 1;
    NGrams gs{};
    for (int m = 0; m < NN; ++m) gs.G[m] = G[m];
    gram_product_kernel<RT><<<blocks(RT * RT), 256, 0, st>>>(gs, NN, mode, last, Hp);
    count_launch();
    dense_factor_kernel<RT><<<1, 128, 0, st>>>(Hp, G[last], R, L, status);
    count_launch();
    const int64_t rows = dim[mode];
    const unsigned nb = blocks(rows);
    dense_rows_kernel<RT><<<nb, 256, 0, st>>>(M, nullptr, R, (int)rows, L, F[mode],
                                              normalize ? part : nullptr);
    count_launch();
    if (normalize) {
      dense_scale_kernel<RT><<<blocks(rows * RT), 256, 0, st>>>(F[mode], (int)rows, part,
                                                               (int)nb);
      count_launch();
    }
    gram(F[mode], rows, G[mode]);
  }
  void unit_columns(const float *F0, int m) const {
    const int64_t rows = dim[m];
    const unsigned nb = blocks(rows);
    dense_rows_kernel<RT><<<nb, 256, 0, st>>>(nullptr, F0, R, (int)rows, nullptr, F[m], part);
    count_launch();
    dense_scale_kernel<RT><<<blocks(rows * RT), 256, 0, st>>>(F[m], (int)rows, part, (int)nb);
    count_launch();
    gram(F[m], rows, G[m]);
  }
};

template <int RT>
void run_dense_n(const DenseCpNArgs &a) {
  DenseCpN<RT> d{};
  d.X = a.X; d.xt = a.xt; d.NN = a.NN; d.R = a.R; d.status = a.status; d.st = a.st;
  int64_t maxdim = 1;
  d.total = 1;
  for (int m = 0; m < a.NN; ++m) {
    d.dim[m] = a.dims[m];
    d.total *= a.dims[m];
    if (a.dims[m] > maxdim) maxdim = a.dims[m];
  }
  int64_t str = 1;
  for (int m = a.NN - 1; m >= 0; --m) {
    d.stride[m] = str;
    str *= a.dims[m];
  }
  float *w = a.work;
  for (int m = 0; m < a.NN; ++m) { d.F[m] = w; w += a.dims[m] * RT; }
  for (int m = 0; m < a.NN; ++m) { d.G[m] = w; w += RT * RT; }
  d.Hp = w; w += RT * RT;
  d.M = w; w += maxdim * RT;
  d.L = w; w += factor_floats<RT>();
  d.part = w; w += ((maxdim + 255) / 256) * RT;
  d.mpart = w; w += n_mpart_rows(maxdim) * RT;
  d.splitk = w;
  for (int m = 1; m < a.NN; ++m) d.unit_columns(a.A0[m - 1], m);
  for (int it = 0; it < a.iters; ++it) {
    d.update(0, false);
    for (int m = 1; m < a.NN; ++m) d.update(m, true);
  }
  d.update(0, false);
  for (int m = 1; m < a.NN; ++m) {
    unpad_kernel<<<blocks(a.dims[m] * a.R), 256, 0, a.st>>>(d.F[m], a.dims[m], a.R, RT,
                                                            a.A_out[m - 1]);
    count_launch();
  }
  unpad_kernel<<<blocks(a.dims[0] * a.R), 256, 0, a.st>>>(d.F[0], a.dims[0], a.R, RT, a.C_out);
  count_launch();
}

}  // namespace

size_t dense_cp_n_work_floats(int NN, const int64_t *dims, int RT) {
  int64_t maxdim = 1, sum = 0;
  for (int m = 0; m < NN; ++m) {
    sum += dims[m];
    if (dims[m] > maxdim) maxdim = dims[m];
  }
  return (size_t)(sum * RT + (NN + 1) * RT * RT + maxdim * RT + 2 * RT * RT + RT +
                  ((maxdim + 255) / 256) * RT + n_mpart_rows(maxdim) * RT) +
         kNSplitkFloats;
}

void dense_cp_n(const DenseCpNArgs &a, int RT) {
  if (RT == 8) run_dense_n<8>(a);
  else if (RT == 16) run_dense_n<16>(a);
  else run_dense_n<32>(a);
}

size_t dense_cp_work_floats(int64_t K, int64_t I, int64_t J, int RT) {
  const int64_t mx = I > J ? (I > K ? I : K) : (J > K ? J : K);
  return (size_t)((I + J + K) * RT + K * I * RT + K * J * RT + mx * RT + 3 * RT * RT +
                  2 * RT * RT + RT + ((mx + 255) / 256) * RT);
}

void dense_cp(const DenseCpArgs &a, int RT) {
  if (RT == 8) run_dense<8>(a);
  else if (RT == 16) run_dense<16>(a);
  else run_dense<32>(a);
}

}  // namespace octen
