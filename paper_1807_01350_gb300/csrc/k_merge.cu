// Merge of the replica factors: anchor match (Sec. "Factor match for
// identifiability", Eq. 5, fp64), the lift of A and B through the stacked
// projections (Sec. "Update results", Eq. 6-7), the least-squares solve of the
// new rows of C, and the dense fp32 Cholesky / triangular solves that build the
// lift operators once per stream.
#include "k_match.cuh"

namespace octen {

// ---------------------------------------------------------------------------
// Anchor match.  ref_a = PA rows [0, S) (= u^T A_prev).
//   sim[r][s] = |cos(At[:S, r], ref_a[:, s])| + |cos(Bt[:S, r], ref_b[:, s])|
// greedy: largest similarity among unmatched pairs, ties to lowest s then r;
// d_a[s] = <At[:S, pi(s)], ref_a[:, s]> / ||ref_a[:, s]||^2 (0 -> 1), same for b.
// Dot products, norms, similarities and scales are fp64.  An fp64 warp
// instruction costs ~64 cycles on this GPU, so the S-term dot products are
// spread over P * RT CTAs (one per replica and column r) before one CTA per
// replica matches; the greedy scan compares the similarities through their
// bit patterns (ordered like the values for non-negative doubles) with integer
// instructions.
// ---------------------------------------------------------------------------

// Scratch layout per replica p (doubles): dA[RT][RT], dB[RT][RT], then
// nta[RT], ntb[RT], nra[RT], nrb[RT].
template <int RT>
__host__ __device__ constexpr int align_scratch_per_replica() { return 2 * RT * RT + 4 * RT; }

// grid (RT, P), 96 threads: warp 0 row r of dA, warp 1 row r of dB, warp 2 the
// four squared norms of column r.
template <int RT>
__global__ void __launch_bounds__(96)
    align_dots_kernel(const float *__restrict__ At, const float *__restrict__ Bt,
                      const float *__restrict__ PA, const float *__restrict__ PB, int Q, int S,
                      int R, double *__restrict__ scratch) {
  const int r = blockIdx.x, p = blockIdx.y, warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  double *sc = scratch + (int64_t)p * align_scratch_per_replica<RT>();
  const float *at = At + (int64_t)p * Q * RT, *bt = Bt + (int64_t)p * Q * RT;
  if (warp < 2) {
    const float *t = warp == 0 ? at : bt;
    const float *ref = warp == 0 ? PA : PB;
    double acc = 0.0;
    if (r < R && lane < R)
      for (int q = 0; q < S; ++q)
        acc = fma((double)t[q * RT + r], (double)ref[(int64_t)q * R + lane], acc);
    if (lane < RT) sc[warp * RT * RT + r * RT + lane] = acc;
  } else {
    double a1 = 0.0, a2 = 0.0, a3 = 0.0, a4 = 0.0;
    if (r < R) {
      for (int q = lane; q < S; q += 32) {
        const double ta = at[q * RT + r], tb = bt[q * RT + r];
        const double ra = PA[(int64_t)q * R + r], rb = PB[(int64_t)q * R + r];
        a1 = fma(ta, ta, a1); a2 = fma(tb, tb, a2); a3 = fma(ra, ra, a3); a4 = fma(rb, rb, a4);
      }
    }
    for (int o = 16; o > 0; o >>= 1) {
      a1 += __shfl_xor_sync(0xffffffffu, a1, o);
      a2 += __shfl_xor_sync(0xffffffffu, a2, o);
      a3 += __shfl_xor_sync(0xffffffffu, a3, o);
      a4 += __shfl_xor_sync(0xffffffffu, a4, o);
    }
    if (lane == 0) {
      double *n = sc + 2 * RT * RT;
      n[r] = a1; n[RT + r] = a2; n[2 * RT + r] = a3; n[3 * RT + r] = a4;
    }
  }
}

// grid P, 256 threads: similarities, greedy matching (warp 0), scales, and the
// aligned replica factors Ah = At[:, pi] / d_a, Bh = Bt[:, pi] / d_b,
// Ch = Ct[:, pi] d_a d_b (the scales applied as fp32 factors).
template <int RT>
__global__ void __launch_bounds__(256)
    align_match_kernel(const float *__restrict__ At, const float *__restrict__ Bt,
                       const float *__restrict__ Ct, const double *__restrict__ scratch, int Q,
                       int R, float *__restrict__ Ah, float *__restrict__ Bh,
                       float *__restrict__ Ch, int *__restrict__ perm_out,
                       double *__restrict__ scales_out) {
  __shared__ double dA[RT * RT], dB[RT * RT], nrm[4 * RT], sq[4 * RT];
  __shared__ unsigned long long key[RT * RT];
  __shared__ float fa[RT], fb[RT], fc[RT];
  __shared__ int perm[RT];
  const int p = blockIdx.x;
  const double *sc = scratch + (int64_t)p * align_scratch_per_replica<RT>();
  for (int e = threadIdx.x; e < RT * RT; e += blockDim.x) {
    dA[e] = sc[e];
    dB[e] = sc[RT * RT + e];
  }
  if (threadIdx.x < 4 * RT) {
    const double v = sc[2 * RT * RT + threadIdx.x];
    nrm[threadIdx.x] = v;
    sq[threadIdx.x] = sqrt(v);   // nta, ntb, nra, nrb -> their square roots
  }
  __syncthreads();
  const double *nta = sq, *ntb = sq + RT, *nra = sq + 2 * RT, *nrb = sq + 3 * RT;
  for (int e = threadIdx.x; e < RT * RT; e += blockDim.x) {
    const int r = e / RT, s = e % RT;
    double v = 0.0;
    if (r < R && s < R) {
      const double den_a = nta[r] * nra[s];
      const double den_b = ntb[r] * nrb[s];
      if (den_a > 0.0) v += fabs(dA[e]) / den_a;
      if (den_b > 0.0) v += fabs(dB[e]) / den_b;
      if (!isfinite(v)) v = 0.0;   // a diverged replica still gets a valid matching
    }
    key[e] = static_cast<unsigned long long>(__double_as_longlong(v));   // v >= 0
  }
  __syncthreads();
  if (threadIdx.x < 32) {
    const int lane = threadIdx.x;
    greedy_match_warp<RT>(key, R, perm);
    if (lane < R) {
      const int s = lane, r = perm[s];
      const double n2a = nrm[2 * RT + s], n2b = nrm[3 * RT + s];
      double a = n2a > 0.0 ? dA[r * RT + s] / n2a : 0.0;
      double b = n2b > 0.0 ? dB[r * RT + s] / n2b : 0.0;
      if (a == 0.0) a = 1.0;
      if (b == 0.0) b = 1.0;
      fa[s] = (float)(1.0 / a);
      fb[s] = (float)(1.0 / b);
      fc[s] = (float)(a * b);
      perm_out[p * R + s] = r;
      scales_out[(int64_t)p * 2 * R + s] = a;
      scales_out[(int64_t)p * 2 * R + R + s] = b;
    }
  }
  __syncthreads();
  const float *at = At + (int64_t)p * Q * RT, *bt = Bt + (int64_t)p * Q * RT;
  const float *ct = Ct + (int64_t)p * Q * RT;
  for (int e = threadIdx.x; e < Q * RT; e += blockDim.x) {
    const int q = e / RT, s = e % RT;
    float va = 0.f, vb = 0.f, vc = 0.f;
    if (s < R) {
      const int r = perm[s];
      va = at[q * RT + r] * fa[s];
      vb = bt[q * RT + r] * fb[s];
      vc = ct[q * RT + r] * fc[s];
    }
    const int64_t o = (int64_t)p * Q * RT + e;
    Ah[o] = va;
    Bh[o] = vb;
    Ch[o] = vc;
  }
}

template <int RT>
static void align_launch(const float *At, const float *Bt, const float *Ct, const float *PA,
                         const float *PB, int P, int Q, int S, int R, float *Ah, float *Bh,
                         float *Ch, int *perm, double *scales, double *scratch, cudaStream_t st) {
  align_dots_kernel<RT><<<dim3(RT, P), 96, 0, st>>>(At, Bt, PA, PB, Q, S, R, scratch);
  count_launch();
  align_match_kernel<RT><<<P, 256, 0, st>>>(At, Bt, Ct, scratch, Q, R, Ah, Bh, Ch, perm, scales);
  count_launch();
}

size_t align_scratch_doubles(int P, int RT) {
  return (size_t)P * (RT == 8    ? align_scratch_per_replica<8>()
                      : RT == 16 ? align_scratch_per_replica<16>()
                                 : align_scratch_per_replica<32>());
}

void align_replicas(const float *At, const float *Bt, const float *Ct, const float *PA,
                    const float *PB, int P, int Q, int S, int R, int RT, float *Ah,
                    float *Bh, float *Ch, int *perm, double *scales, double *scratch,
                    cudaStream_t st) {
  if (RT == 8)
    align_launch<8>(At, Bt, Ct, PA, PB, P, Q, S, R, Ah, Bh, Ch, perm, scales, scratch, st);
  else if (RT == 16)
    align_launch<16>(At, Bt, Ct, PA, PB, P, Q, S, R, Ah, Bh, Ch, perm, scales, scratch, st);
  else
    align_launch<32>(At, Bt, Ct, PA, PB, P, Q, S, R, Ah, Bh, Ch, perm, scales, scratch, st);
}

// ---------------------------------------------------------------------------
// Right-hand side of the lift: residual of every replica block against the
// projected previous factor, reduced to the Qd distinct rows of the stack.
//   anchor row c < S:  sum_p (or mean_p) (Fh_p[c] - PF[c])
//   private row c:     Fh_p[b] - PF[c] with p, b the owner of column c
// ---------------------------------------------------------------------------
__global__ void lift_rhs_kernel(const float *__restrict__ Fh, const float *__restrict__ PF,
                                int P, int Q, int S, int R, int RT, int Qd, int sum_mode,
                                float *__restrict__ e) {
  const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (idx >= (int64_t)Qd * R) return;
  const int c = (int)(idx / R), r = (int)(idx % R);
  const float pf = PF[idx];
  float v;
  if (c < S) {
    float s = 0.f;
    for (int p = 0; p < P; ++p) s += Fh[((int64_t)p * Q + c) * RT + r] - pf;
    v = sum_mode ? s : s / (float)P;
  } else {
    const int p = (c - S) / (Q - S);
    const int b = S + (c - S) - p * (Q - S);
    v = Fh[((int64_t)p * Q + b) * RT + r] - pf;
  }
  e[idx] = v;
}

void lift_rhs(const float *Fh, const float *PF, int P, int Q, int S, int R, int RT, int Qd,
              int sum_mode, float *e, cudaStream_t st) {
  const int64_t n = (int64_t)Qd * R;
  lift_rhs_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(Fh, PF, P, Q, S, R, RT, Qd,
                                                                sum_mode, e);
  count_launch();
}

// ---------------------------------------------------------------------------
// New rows of C.  The stacked system (W_new,p^T) C_new = Ch_p - G_p has normal
// equations (sum_p W_p W_p^T) C_new = sum_p W_p (Ch_p - G_p).  Both sides are
// reduced over the Qd distinct columns of W_all (anchor columns weighted P):
// chunks of kCChunk columns give partial sums, added in chunk order by the
// solve, which factors the t x t system by fp64 Cholesky (t <= 64) in one CTA.
// ---------------------------------------------------------------------------
constexpr int kCChunk = 64;

size_t c_solve_scratch_floats(int64_t t, int Qd, int R) {
  return (size_t)((Qd + kCChunk - 1) / kCChunk) * (size_t)(t * t + t * R);
}

// Chunk j of the columns c (grid ceil(Qd / kCChunk), 256 threads):
//   part[j][k][l]         = sum_c w_c W[k][c] W[l][c]      (w_c = P for c < S, else 1)
//   part[j][t t + k R + r] = sum_c W[k][c] E[c][r],
// E[c][r] = sum over the replicas holding column c of Ch_p[b][r] - G_p[b][r]
// (all P for an anchor column c = b < S, else the one replica p with
// c = S + p (Q - S) + b - S), each sum in increasing c.
__global__ void __launch_bounds__(256)
    c_normal_kernel(const float *__restrict__ W, const float *__restrict__ Ch,
                    const float *__restrict__ G, int t, int P, int Q, int S, int Qd, int R,
                    int RT, float *__restrict__ part) {
  __shared__ float Ws[64][kCChunk + 1];
  __shared__ float Es[kCChunk][33];
  const int c0 = blockIdx.x * kCChunk;
  const int nc = Qd - c0 < kCChunk ? Qd - c0 : kCChunk;
  for (int e = threadIdx.x; e < t * kCChunk; e += blockDim.x) {
    const int k = e / kCChunk, cc = e % kCChunk;
    Ws[k][cc] = cc < nc ? W[(int64_t)k * Qd + c0 + cc] : 0.f;
  }
  for (int e = threadIdx.x; e < kCChunk * R; e += blockDim.x) {
    const int cc = e / R, r = e % R, c = c0 + cc;
    float v = 0.f;
    if (cc < nc) {
      if (c < S) {
        for (int p = 0; p < P; ++p)
          v += Ch[((int64_t)p * Q + c) * RT + r] - G[((int64_t)p * Q + c) * R + r];
      } else {
        const int p = (c - S) / (Q - S);
        const int b = S + (c - S) - p * (Q - S);
        v = Ch[((int64_t)p * Q + b) * RT + r] - G[((int64_t)p * Q + b) * R + r];
      }
    }
    Es[cc][r] = v;
  }
  __syncthreads();
  float *out = part + (int64_t)blockIdx.x * (t * t + t * R);
  const float wS = (float)P;
  for (int e = threadIdx.x; e < t * t; e += blockDim.x) {
    const int k = e / t, l = e % t;
    float acc = 0.f;
    for (int cc = 0; cc < nc; ++cc) {
      const float w = c0 + cc < S ? wS : 1.f;
      acc = fmaf(w * Ws[k][cc], Ws[l][cc], acc);
    }
    out[e] = acc;
  }
  for (int e = threadIdx.x; e < t * R; e += blockDim.x) {
    const int k = e / R, r = e % R;
    float acc = 0.f;
    for (int cc = 0; cc < nc; ++cc) acc = fmaf(Ws[k][cc], Es[cc][r], acc);
    out[t * t + e] = acc;
  }
}

// Reciprocal square root of a Cholesky pivot.  ok is cleared unless d is
// positive, normal and finite.  For d in [2^-100, 2^100]: the fp32 value of d
// assembled from its bits (mantissa truncated to 23 bits), rsqrt.approx of it
// (relative error < 2^-22), widened to fp64 from its bits, and one Newton step
// for 1 / sqrt(d), y <- y + y (1 - d y^2) / 2, which squares the relative error
// (< 2^-42).  Outside that range the fp64 square root and division are used.
__device__ __forceinline__ double pivot_rsqrt(double d, bool &ok) {
  const int hi = __double2hiint(d);
  const unsigned lo = static_cast<unsigned>(__double2loint(d));
  const int be = (hi >> 20) & 0x7ff;
  if (hi < 0 || be == 0 || be == 0x7ff) {
    ok = false;
    return 0.0;
  }
  if (be < 1023 - 100 || be > 1023 + 100) return 1.0 / sqrt(d);
  const float f = __int_as_float(((be - 1023 + 127) << 23) | ((hi & 0xfffff) << 3) |
                                 static_cast<int>(lo >> 29));
  float y;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(f));
  const int yb = __float_as_int(y);
  const int ye = (yb >> 23) & 0xff;
  const int ym = yb & 0x7fffff;
  const double y0 = __hiloint2double(((ye - 127 + 1023) << 20) | (ym >> 3), ym << 29);
  const double e = fma(-d * y0, y0, 1.0);
  return fma(0.5 * y0, e, y0);
}

// Gram (t x t, t <= 64) = L L^T by right-looking Cholesky in fp64 (the pivot
// column scaled by the reciprocal square root of the pivot, then the trailing
// lower triangle updated by all threads), then L L^T X = rhs for the R
// columns of rhs, forward and backward by columns with the updates of the
// remaining rows in parallel.  A pivot that is not positive: the diagonal is
// loaded by 1e-12 trace / t and the factorisation repeated once; if that fails
// as well, status gets kDevCholesky and C_new = 0.
__global__ void __launch_bounds__(256)
    c_solve_kernel(const float *__restrict__ part, int nchunks, int t, int R,
                   float *__restrict__ C_new, int *status) {
  __shared__ double L[64 * 64];
  __shared__ double X[64 * 32];
  __shared__ double rinv[64];
  __shared__ int ok_s;
  const int tid = threadIdx.x, nt = blockDim.x;
  const int per = t * t + t * R;
  // the chunks' partial sums, added in chunk order (the system's entries
  // e < t t, its right-hand side after them)
  auto entry = [&](int e) {
    float v = 0.f;
    for (int j = 0; j < nchunks; ++j) v += part[(int64_t)j * per + e];
    return v;
  };
  for (int e = tid; e < per; e += nt) {
    const float v = entry(e);
    if (e < t * t) L[e] = v;
    else X[e - t * t] = v;
  }
  if (tid == 0) ok_s = 1;
  __syncthreads();
  for (int attempt = 0; attempt < 2; ++attempt) {
    for (int j = 0; j < t; ++j) {
      if (tid == 0) {
        bool ok = true;
        const double d = L[j * t + j];
        const double y = pivot_rsqrt(d, ok);
        if (ok) {
          L[j * t + j] = d * y;
          rinv[j] = y;
        } else {
          ok_s = 0;
        }
      }
      __syncthreads();
      if (!ok_s) break;
      for (int i = j + 1 + tid; i < t; i += nt) L[i * t + j] *= rinv[j];
      __syncthreads();
      const int m = t - j - 1;   // trailing block rows / columns j + 1 ..
      for (int e = tid; e < m * m; e += nt) {
        const int i = j + 1 + e / m, k = j + 1 + e % m;
        if (k <= i) L[i * t + k] = fma(-L[i * t + j], L[k * t + j], L[i * t + k]);
      }
      __syncthreads();
    }
    if (ok_s || attempt == 1) break;
    __syncthreads();
    for (int e = tid; e < t * t; e += nt) L[e] = entry(e);
    __syncthreads();
    if (tid == 0) {
      double tr = 0.0;
      for (int k = 0; k < t; ++k) tr += L[k * t + k];
      for (int k = 0; k < t; ++k) L[k * t + k] += 1e-12 * tr / t;
      ok_s = 1;
    }
    __syncthreads();
  }
  if (!ok_s) {
    if (tid == 0) atomicOr(status, kDevCholesky);
    for (int e = tid; e < t * R; e += nt) C_new[e] = 0.f;
    return;
  }
  // L z = rhs: z_k = b_k / L_kk, then b_i -= L_ik z_k below it
  for (int k = 0; k < t; ++k) {
    for (int r = tid; r < R; r += nt) X[k * R + r] *= rinv[k];
    __syncthreads();
    const int n = (t - k - 1) * R;
    for (int e = tid; e < n; e += nt) {
      const int i = k + 1 + e / R, r = e % R;
      X[i * R + r] = fma(-L[i * t + k], X[k * R + r], X[i * R + r]);
    }
    __syncthreads();
  }
  // L^T x = z: x_k = z_k / L_kk, then z_i -= L_ki x_k above it
  for (int k = t - 1; k >= 0; --k) {
    for (int r = tid; r < R; r += nt) X[k * R + r] *= rinv[k];
    __syncthreads();
    const int n = k * R;
    for (int e = tid; e < n; e += nt) {
      const int i = e / R, r = e % R;
      X[i * R + r] = fma(-L[k * t + i], X[k * R + r], X[i * R + r]);
    }
    __syncthreads();
  }
  for (int e = tid; e < t * R; e += nt) C_new[e] = (float)X[e];
}

__global__ void scale_columns_kernel(const float *__restrict__ in, int64_t rows, int cols,
                                     int S, float w, float *__restrict__ out) {
  const int64_t n = rows * cols;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int c = (int)(i % cols);
    out[i] = c < S ? in[i] * w : in[i];
  }
}

void scale_columns(const float *in, int64_t rows, int cols, int S, float w_shared, float *out,
                   cudaStream_t st) {
  const int64_t n = rows * cols;
  if (n <= 0) return;
  const unsigned blocks = (unsigned)((n + 255) / 256 < 8192 ? (n + 255) / 256 : 8192);
  scale_columns_kernel<<<blocks, 256, 0, st>>>(in, rows, cols, S, w_shared, out);
  count_launch();
}

// scratch: c_solve_scratch_floats(t, Qd, R) floats of chunk partials.
void solve_c_new(const float *W, const float *Ch, const float *G, int64_t t, int P, int Q,
                 int S, int Qd, int R, int RT, float *scratch, float *C_new, int *status,
                 cudaStream_t st) {
  const int nchunks = (Qd + kCChunk - 1) / kCChunk;
  c_normal_kernel<<<nchunks, 256, 0, st>>>(W, Ch, G, (int)t, P, Q, S, Qd, R, RT, scratch);
  count_launch();
  c_solve_kernel<<<1, 256, 0, st>>>(scratch, nchunks, (int)t, R, C_new, status);
  count_launch();
}

// G[p][b][r] += sum_k W[k][col_p(b)] C_new[k][r]
__global__ void update_g_kernel(const float *__restrict__ W, const float *__restrict__ Cn,
                                int t, int P, int Q, int S, int Qd, int R,
                                float *__restrict__ G) {
  const int p = blockIdx.y;
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= Q * R) return;
  const int b = e / R, r = e % R;
  const int col = b < S ? b : S + p * (Q - S) + (b - S);
  float acc = 0.f;
  for (int k = 0; k < t; ++k) acc = fmaf(W[(int64_t)k * Qd + col], Cn[(int64_t)k * R + r], acc);
  G[((int64_t)p * Q + b) * R + r] += acc;
}

void update_g(const float *W, const float *C_new, int64_t t, int P, int Q, int S, int Qd,
              int R, float *G, cudaStream_t st) {
  dim3 grid((Q * R + 255) / 256, P);
  update_g_kernel<<<grid, 256, 0, st>>>(W, C_new, (int)t, P, Q, S, Qd, R, G);
  count_launch();
}

// ---------------------------------------------------------------------------
// Dense SPD factorisation A = L L^T (row-major n x n, lower triangle written,
// fp32) by 32-wide column blocks: fp64 factor of the diagonal block, fp32
// triangular solve of the panel below, fp32 trailing update by the SIMT GEMM.
// ---------------------------------------------------------------------------
constexpr int kNB = 32;

__global__ void chol_diag_kernel(float *A, int n, int j0, int jb, int *status) {
  __shared__ double Ls[kNB * kNB];
  __shared__ int ok_s;
  for (int e = threadIdx.x; e < jb * jb; e += blockDim.x) {
    const int r = e / jb, c = e % jb;
    Ls[e] = A[(int64_t)(j0 + r) * n + j0 + c];
  }
  if (threadIdx.x == 0) ok_s = 1;
  __syncthreads();
  for (int j = 0; j < jb; ++j) {
    if (threadIdx.x == 0) {
      double d = Ls[j * jb + j];
      for (int k = 0; k < j; ++k) d -= Ls[j * jb + k] * Ls[j * jb + k];
      if (d > 0.0) Ls[j * jb + j] = sqrt(d);
      else { Ls[j * jb + j] = 1.0; ok_s = 0; }
    }
    __syncthreads();
    const int i = j + 1 + threadIdx.x;
    if (i < jb) {
      double s = Ls[i * jb + j];
      for (int k = 0; k < j; ++k) s -= Ls[i * jb + k] * Ls[j * jb + k];
      Ls[i * jb + j] = s / Ls[j * jb + j];
    }
    __syncthreads();
  }
  if (!ok_s && threadIdx.x == 0) atomicOr(status, kDevCholesky);
  for (int e = threadIdx.x; e < jb * jb; e += blockDim.x) {
    const int r = e / jb, c = e % jb;
    A[(int64_t)(j0 + r) * n + j0 + c] = c <= r ? (float)Ls[e] : 0.f;
  }
}

// rows i >= j0 + jb:  L[i][j0 : j0+jb] = A[i][j0 : j0+jb] L11^-T
__global__ void chol_panel_kernel(float *A, int n, int j0, int jb) {
  __shared__ float L11[kNB * kNB];
  for (int e = threadIdx.x; e < jb * jb; e += blockDim.x)
    L11[e] = A[(int64_t)(j0 + e / jb) * n + j0 + e % jb];
  __syncthreads();
  const int64_t i = (int64_t)j0 + jb + blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  float x[kNB];
  float *row = A + i * n + j0;
  for (int k = 0; k < jb; ++k) {
    float s = row[k];
    for (int l = 0; l < k; ++l) s = fmaf(-x[l], L11[k * jb + l], s);
    x[k] = s / L11[k * jb + k];
  }
  for (int k = 0; k < jb; ++k) row[k] = x[k];
}

void cholesky_f32(float *Gm, int n, int *status, cudaStream_t st) {
  for (int j0 = 0; j0 < n; j0 += kNB) {
    const int jb = n - j0 < kNB ? n - j0 : kNB;
    chol_diag_kernel<<<1, 64, 0, st>>>(Gm, n, j0, jb, status);
    count_launch();
    const int rest = n - j0 - jb;
    if (rest <= 0) continue;
    chol_panel_kernel<<<(rest + 127) / 128, 128, 0, st>>>(Gm, n, j0, jb);
    count_launch();
    GemmArgs g{};
    g.A = Gm + (int64_t)(j0 + jb) * n + j0; g.ta = Elem::F32; g.sAz = 0; g.sAm = n; g.sAk = 1;
    g.B = g.A; g.tb = Elem::F32; g.sBz = 0; g.sBn = n; g.sBk = 1;
    g.D = Gm + (int64_t)(j0 + jb) * n + j0 + jb; g.sDz = 0; g.sDm = n; g.sDn = 1;
    g.M = rest; g.N = rest; g.K = jb; g.batch = 1; g.alpha = -1.f; g.beta = 1.f;
    gemm_strided(g, st);
  }
}

// Block triangular solves with m right-hand sides (row-major n x m, in place).
__global__ void trsv_fwd_block_kernel(const float *L, int n, int j0, int jb, float *Bm, int m) {
  __shared__ float L11[kNB * kNB];
  for (int e = threadIdx.x; e < jb * jb; e += blockDim.x)
    L11[e] = L[(int64_t)(j0 + e / jb) * n + j0 + e % jb];
  __syncthreads();
  const int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (c >= m) return;
  float x[kNB];
  for (int k = 0; k < jb; ++k) {
    float s = Bm[(int64_t)(j0 + k) * m + c];
    for (int l = 0; l < k; ++l) s = fmaf(-L11[k * jb + l], x[l], s);
    x[k] = s / L11[k * jb + k];
  }
  for (int k = 0; k < jb; ++k) Bm[(int64_t)(j0 + k) * m + c] = x[k];
}

__global__ void trsv_bwd_block_kernel(const float *L, int n, int j0, int jb, float *Bm, int m) {
  __shared__ float L11[kNB * kNB];
  for (int e = threadIdx.x; e < jb * jb; e += blockDim.x)
    L11[e] = L[(int64_t)(j0 + e / jb) * n + j0 + e % jb];
  __syncthreads();
  const int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (c >= m) return;
  float x[kNB];
  for (int k = jb - 1; k >= 0; --k) {
    float s = Bm[(int64_t)(j0 + k) * m + c];
    for (int l = k + 1; l < jb; ++l) s = fmaf(-L11[l * jb + k], x[l], s);
    x[k] = s / L11[k * jb + k];
  }
  for (int k = 0; k < jb; ++k) Bm[(int64_t)(j0 + k) * m + c] = x[k];
}

void chol_solve_f32(const float *L, int n, float *Bm, int m, cudaStream_t st) {
  const unsigned blocks = (unsigned)((m + 127) / 128);
  for (int j0 = 0; j0 < n; j0 += kNB) {          // L Y = B
    const int jb = n - j0 < kNB ? n - j0 : kNB;
    trsv_fwd_block_kernel<<<blocks, 128, 0, st>>>(L, n, j0, jb, Bm, m);
    count_launch();
    const int rest = n - j0 - jb;
    if (rest <= 0) continue;
    GemmArgs g{};
    g.A = L + (int64_t)(j0 + jb) * n + j0; g.ta = Elem::F32; g.sAm = n; g.sAk = 1;
    g.B = Bm + (int64_t)j0 * m; g.tb = Elem::F32; g.sBn = 1; g.sBk = m;
    g.D = Bm + (int64_t)(j0 + jb) * m; g.sDm = m; g.sDn = 1;
    g.M = rest; g.N = m; g.K = jb; g.batch = 1; g.alpha = -1.f; g.beta = 1.f;
    gemm_strided(g, st);
  }
  const int last = ((n - 1) / kNB) * kNB;
  for (int j0 = last; j0 >= 0; j0 -= kNB) {     // L^T X = Y
    const int jb = n - j0 < kNB ? n - j0 : kNB;
    trsv_bwd_block_kernel<<<blocks, 128, 0, st>>>(L, n, j0, jb, Bm, m);
    count_launch();
    if (j0 == 0) continue;
    GemmArgs g{};
    // Y[0:j0] -= L[j0:j0+jb, 0:j0]^T X[j0:j0+jb]
    g.A = L + (int64_t)j0 * n; g.ta = Elem::F32; g.sAm = 1; g.sAk = n;
    g.B = Bm + (int64_t)j0 * m; g.tb = Elem::F32; g.sBn = 1; g.sBk = m;
    g.D = Bm; g.sDm = m; g.sDn = 1;
    g.M = j0; g.N = m; g.K = jb; g.batch = 1; g.alpha = -1.f; g.beta = 1.f;
    gemm_strided(g, st);
  }
}

__global__ void transpose_kernel(const float *__restrict__ in, int64_t rows, int64_t cols,
                                 float *__restrict__ out) {
  __shared__ float tile[32][33];
  const int64_t r0 = (int64_t)blockIdx.y * 32, c0 = (int64_t)blockIdx.x * 32;
  for (int yy = threadIdx.y; yy < 32; yy += 8) {
    const int64_t r = r0 + yy, c = c0 + threadIdx.x;
    tile[yy][threadIdx.x] = (r < rows && c < cols) ? in[r * cols + c] : 0.f;
  }
  __syncthreads();
  for (int yy = threadIdx.y; yy < 32; yy += 8) {
    const int64_t c = c0 + yy, r = r0 + threadIdx.x;
    if (c < cols && r < rows) out[c * rows + r] = tile[threadIdx.x][yy];
  }
}

void transpose_f32(const float *in, int64_t rows, int64_t cols, float *out, cudaStream_t st) {
  dim3 grid((unsigned)((cols + 31) / 32), (unsigned)((rows + 31) / 32));
  transpose_kernel<<<grid, dim3(32, 8), 0, st>>>(in, rows, cols, out);
  count_launch();
}

}  // namespace octen
