// Kernels of the N-mode extension (Sec. "Extending to Higher-Order Tensors"):
// a tensor with N - 1 non-temporal modes I_1 x ... x I_{N-1} growing in its
// N-th (time) mode.  Every replica p compresses every mode with its own
// projection (first S columns shared, Eq. 1), keeps the N-way summary
// Y_p[q_1]...[q_{N-1}][c] (X_p = Y_p + Z_p), decomposes it by CP-ALS, and the
// replica factors are matched on their anchor rows in every non-temporal mode
// before each factor is lifted as in Eq. 7.
//
// Compression of a chunk of t slices X[k][i_1]...[i_{N-1}] (fp32) as a chain
// of skinny GEMMs that each contract the innermost index and write their
// result transposed, so that the next index to contract becomes innermost:
//   X [(k, i_1..i_{N-2})][i_{N-1}]         x U_{N-1} of all replicas (N = P Q)
//     -> T [p][q_{N-1}][(k, i_1..i_{N-2})]
//   T [p][(q_{m+1}.., k, i_1..i_{m-1})][i_m] x U_m,p      (batched over p)
//     -> T [p][q_m][(q_{m+1}.., k, i_1..i_{m-1})]
//   ... down to m = 1, leaving T [p][(q_1..q_{N-1})][k];
//   Y_p[(q_1..q_{N-1})][c] += sum_k T[p][(q..)][k] W_p[k][c].
// The first product reads every slice once for all replicas (the anchor
// columns are computed once per replica, as in the 3-mode mode-2 pass); the
// later ones work on tensors already shrunk by Q / I_m per step.
#include "k_match.cuh"
#include "k_solve.cuh"

namespace octen {

namespace {

constexpr int kNThreads = 256;

__host__ __device__ inline int64_t ipow(int64_t b, int e) {
  int64_t r = 1;
  for (int i = 0; i < e; ++i) r *= b;
  return r;
}

// The Khatri-Rao form of the MTTKRP keeps the product of the outer factors'
// rows for every outer index combination (Q^(NN-2) x RT floats) and their X
// offsets; it applies for Q <= 32 while that table stays small.
constexpr int kKrMaxFloats = 8192;
__host__ __device__ inline bool nals_use_kr(int NN, int Q, int RT) {
  return Q <= 32 && ipow(Q, NN - 2) * RT <= kKrMaxFloats;
}

// Shared floats of the replica ALS: X Q^NN (if it is kept in shared memory,
// rounded up to a multiple of 4) | F NN Q RT | M Q RT | Mp max(Q, 128) RT |
// G NN RT^2 | Hp, Lc, Lr RT^2 each | rf RT | red 8 RT | scl RT | with the
// Khatri-Rao form: KRo Q^(NN-2) RT | Oo Q^(NN-2) ints (rounded up to 4).
// Every array after X has a length that is a multiple of 4 (RT is a multiple
// of 8).
size_t nals_floats(int NN, int Q, int RT, bool x_in_smem) {
  const size_t q = (size_t)Q, rt = (size_t)RT;
  const size_t x = x_in_smem ? (((size_t)ipow(Q, NN) + 3) & ~size_t(3)) : 0;
  const size_t mp = (q > 128 ? q : 128) * rt;
  size_t kr = 0;
  if (nals_use_kr(NN, Q, RT)) {
    const size_t no = (size_t)ipow(Q, NN - 2);
    kr = no * rt + ((no + 3) & ~size_t(3));
  }
  return x + (size_t)NN * q * rt + q * rt + mp + (size_t)NN * rt * rt + 3 * rt * rt +
         10 * rt + kr;
}

__device__ __forceinline__ void nals_mttkrp_barrier() {
  asm volatile("bar.sync 2, 128;" ::: "memory");
}

// MTTKRP of mode n by the 128 threads u = 0..127 (warps 4..7):
//   M[q][r] = sum over the other indices of X[..q..] prod_{m != n} F_m[idx_m][r].
// The other modes are split into an inner mode ml (the last one other than n)
// and the outer ones.  A work item is one (q, r < R) and a contiguous range of
// the outer index combinations (the range split into `ns` parts when Q R is
// below 128, so that every thread has work; the parts are summed in order
// afterwards).  Per outer combination: the product of the outer factors' rows
// (once) and the inner sum over ml; the outer digits advance like an odometer
// (no divisions in the loop).  Entries r >= R of M are left untouched (zero).
template <int RT, int NN>
__device__ void nals_mttkrp(const float *X, const float *F, int Q, int R, int n, float *M,
                            float *Mp, int u) {
  int pw[NN];
  pw[NN - 1] = 1;
#pragma unroll
  for (int m = NN - 2; m >= 0; --m) pw[m] = pw[m + 1] * Q;
  const int ml = n == NN - 1 ? NN - 2 : NN - 1;
  int sl = 0, pwn = 0;   // strides of modes ml and n (selected without indexing pw at run time)
#pragma unroll
  for (int m = 0; m < NN; ++m) {
    if (m == ml) sl = pw[m];
    if (m == n) pwn = pw[m];
  }
  const int items = Q * R;
  const int ns = items >= 128 ? 1 : 128 / items;
  const int nouter = (int)ipow(Q, NN - 2);
  const int chunk = (nouter + ns - 1) / ns;
  for (int w = u; w < items * ns; w += 128) {
    const int part = w / items, e = w - part * items;
    const int q = e / R, r = e - q * R;
    const int o0 = part * chunk;
    const int o1 = o0 + chunk < nouter ? o0 + chunk : nouter;
    float acc = 0.f;
    if (o0 < o1) {
      int dig[NN];
      int rem = o0;
#pragma unroll
      for (int m = NN - 1; m >= 0; --m) {
        dig[m] = 0;
        if (m == n || m == ml) continue;
        dig[m] = rem % Q;
        rem /= Q;
      }
      const float *fl = F + (size_t)ml * Q * RT + r;
      const float *xq = X + q * pwn;
      for (int o = o0; o < o1; ++o) {
        int off = 0;
        float pr = 1.f;
#pragma unroll
        for (int m = 0; m < NN; ++m) {
          if (m == n || m == ml) continue;
          off += dig[m] * pw[m];
          pr *= F[(m * Q + dig[m]) * RT + r];
        }
        const float *xp = xq + off;
        float s = 0.f;
        for (int d = 0; d < Q; ++d) s = fmaf(xp[d * sl], fl[d * RT], s);
        acc = fmaf(pr, s, acc);
#pragma unroll
        for (int m = NN - 1; m >= 0; --m) {
          if (m == n || m == ml) continue;
          if (++dig[m] < Q) break;
          dig[m] = 0;
        }
      }
    }
    if (ns == 1) M[q * RT + r] = acc;
    else Mp[w] = acc;
  }
  if (ns > 1) {
    nals_mttkrp_barrier();
    for (int e = u; e < items; e += 128) {
      float s = 0.f;
      for (int part = 0; part < ns; ++part) s += Mp[part * items + e];
      M[(e / R) * RT + e % R] = s;
    }
  }
}

// MTTKRP of mode n in Khatri-Rao form by warps 4..7 (u = 0..127), Q <= 32.
// First the outer modes' (all but n and the inner mode ml) row products
// KRo[o][r] and the X offsets Oo[o] of every outer combination o; then
//  - non-temporal n (ml = the time mode, stride 1): a warp per q at a time,
//    lanes over (phase s, inner index d): acc[r] = sum over the phase's o of
//    X[q, o, d] KRo[o][r], times F_ml[d][r], summed over the warp;
//  - time mode n (ml = the last non-temporal mode): lanes over (s, c), 4 nsw
//    groups over o: t[r] = sum_d X[o, d, c] F_ml[d][r], acc[r] += KRo[o][r] t[r];
//    the groups' partials are summed in order.
// Lanes read consecutive X addresses (the stride-1 index runs across them).
template <int RT, int NN>
__device__ void nals_mttkrp_kr(const float *X, const float *F, int Q, int n, float *M,
                               float *Mp, float *KRo, int *Oo, int u) {
  int pw[NN];
  pw[NN - 1] = 1;
#pragma unroll
  for (int m = NN - 2; m >= 0; --m) pw[m] = pw[m + 1] * Q;
  const int ml = n == NN - 1 ? NN - 2 : NN - 1;
  int sl = 0, pwn = 0;
#pragma unroll
  for (int m = 0; m < NN; ++m) {
    if (m == ml) sl = pw[m];
    if (m == n) pwn = pw[m];
  }
  const int nouter = (int)ipow(Q, NN - 2);
  for (int o = u; o < nouter; o += 128) {
    int rem = o, off = 0;
    float4 pr[RT / 4];
#pragma unroll
    for (int r4 = 0; r4 < RT / 4; ++r4) pr[r4] = make_float4(1.f, 1.f, 1.f, 1.f);
#pragma unroll
    for (int m = NN - 1; m >= 0; --m) {
      if (m == n || m == ml) continue;
      const int dg = rem % Q;
      rem /= Q;
      off += dg * pw[m];
      const float4 *f = reinterpret_cast<const float4 *>(F + (m * Q + dg) * RT);
#pragma unroll
      for (int r4 = 0; r4 < RT / 4; ++r4) {
        const float4 v = f[r4];
        pr[r4].x *= v.x; pr[r4].y *= v.y; pr[r4].z *= v.z; pr[r4].w *= v.w;
      }
    }
    float4 *k = reinterpret_cast<float4 *>(KRo + o * RT);
#pragma unroll
    for (int r4 = 0; r4 < RT / 4; ++r4) k[r4] = pr[r4];
    Oo[o] = off;
  }
  nals_mttkrp_barrier();
  const int w = u >> 5, lane = u & 31;
  const int nsw = 32 / Q;
  const int s = lane / Q, i = lane - s * Q;
  const bool active = s < nsw;
  const float *Fl = F + (size_t)ml * Q * RT;
  float acc[RT];
  if (n != NN - 1) {
    for (int q = w; q < Q; q += 4) {
#pragma unroll
      for (int r = 0; r < RT; ++r) acc[r] = 0.f;
      if (active) {
        const float *xq = X + q * pwn + i;
#pragma unroll 4
        for (int o = s; o < nouter; o += nsw) {
          const float x = xq[Oo[o]];
          const float4 *kr = reinterpret_cast<const float4 *>(KRo + o * RT);
#pragma unroll
          for (int r4 = 0; r4 < RT / 4; ++r4) {
            const float4 k = kr[r4];
            acc[4 * r4] = fmaf(x, k.x, acc[4 * r4]);
            acc[4 * r4 + 1] = fmaf(x, k.y, acc[4 * r4 + 1]);
            acc[4 * r4 + 2] = fmaf(x, k.z, acc[4 * r4 + 2]);
            acc[4 * r4 + 3] = fmaf(x, k.w, acc[4 * r4 + 3]);
          }
        }
        const float4 *f = reinterpret_cast<const float4 *>(Fl + i * RT);
#pragma unroll
        for (int r4 = 0; r4 < RT / 4; ++r4) {
          const float4 v = f[r4];
          acc[4 * r4] *= v.x;
          acc[4 * r4 + 1] *= v.y;
          acc[4 * r4 + 2] *= v.z;
          acc[4 * r4 + 3] *= v.w;
        }
      }
#pragma unroll
      for (int r = 0; r < RT; ++r)
        for (int o = 16; o > 0; o >>= 1) acc[r] += __shfl_xor_sync(0xffffffffu, acc[r], o);
      if (lane < RT) {
        float v = 0.f;
#pragma unroll
        for (int r = 0; r < RT; ++r)
          if (r == lane) v = acc[r];
        M[q * RT + lane] = v;
      }
    }
  } else {
    const int ng = 4 * nsw;
#pragma unroll
    for (int r = 0; r < RT; ++r) acc[r] = 0.f;
    if (active) {
      const int g = w * nsw + s;
#pragma unroll 2
      for (int o = g; o < nouter; o += ng) {
        const float *xo = X + Oo[o] + i;
        float t[RT];
#pragma unroll
        for (int r = 0; r < RT; ++r) t[r] = 0.f;
#pragma unroll 4
        for (int d = 0; d < Q; ++d) {
          const float x = xo[d * sl];
          const float4 *f = reinterpret_cast<const float4 *>(Fl + d * RT);
#pragma unroll
          for (int r4 = 0; r4 < RT / 4; ++r4) {
            const float4 v = f[r4];
            t[4 * r4] = fmaf(x, v.x, t[4 * r4]);
            t[4 * r4 + 1] = fmaf(x, v.y, t[4 * r4 + 1]);
            t[4 * r4 + 2] = fmaf(x, v.z, t[4 * r4 + 2]);
            t[4 * r4 + 3] = fmaf(x, v.w, t[4 * r4 + 3]);
          }
        }
        const float4 *kr = reinterpret_cast<const float4 *>(KRo + o * RT);
#pragma unroll
        for (int r4 = 0; r4 < RT / 4; ++r4) {
          const float4 k = kr[r4];
          acc[4 * r4] = fmaf(k.x, t[4 * r4], acc[4 * r4]);
          acc[4 * r4 + 1] = fmaf(k.y, t[4 * r4 + 1], acc[4 * r4 + 1]);
          acc[4 * r4 + 2] = fmaf(k.z, t[4 * r4 + 2], acc[4 * r4 + 2]);
          acc[4 * r4 + 3] = fmaf(k.w, t[4 * r4 + 3], acc[4 * r4 + 3]);
        }
      }
      float4 *mp = reinterpret_cast<float4 *>(Mp + ((size_t)g * Q + i) * RT);
#pragma unroll
      for (int r4 = 0; r4 < RT / 4; ++r4)
        mp[r4] = make_float4(acc[4 * r4], acc[4 * r4 + 1], acc[4 * r4 + 2], acc[4 * r4 + 3]);
    }
    nals_mttkrp_barrier();
    for (int e = u; e < Q * RT; e += 128) {
      float sum = 0.f;
      for (int g = 0; g < ng; ++g) sum += Mp[(size_t)g * Q * RT + e];
      M[e] = sum;
    }
  }
}

}  // namespace

// grid P, 256 threads.  Per replica: the CP of the N-way summary X_p by
// alternating least squares in the order of the oracle's CP sweep: the time
// factor, then every non-temporal factor normalised to unit l2, `iters` times,
// and a final time-factor update.  Warps 0..3 factor the normal equations
// (fp64 L D L^T of the Hadamard product of the other factors' Grams) while
// warps 4..7 form the MTTKRP; the whole CTA then substitutes.
struct NAlsArgs {
  const float *Y;                  // P x Q^NN summaries
  float *F[kMaxNModes];            // in: warm starts of modes 0..NN-2; out: all NN factors
  const float *G0[kMaxNModes];     // Grams of the warm starts (P x RT x RT)
  int Q, R, iters, x_in_smem;
  int *status;
};

template <int RT, int NN>
__global__ void __launch_bounds__(kNThreads, 1) nals_kernel(NAlsArgs a) {
  extern __shared__ __align__(16) float sm[];
  __shared__ double Craw[RT * (RT + 1)], Rs[RT];
  __shared__ int fail_s;
  const int p = blockIdx.x, tid = threadIdx.x, Q = a.Q, R = a.R;
  const int64_t nx = ipow(Q, NN);
  const float *X = a.Y + (size_t)p * nx;
  float *base = sm;
  if (a.x_in_smem) {
    for (int64_t e = tid; e < nx; e += blockDim.x) base[e] = X[e];
    X = base;
    base += (nx + 3) & ~int64_t(3);
  }
  float *F = base;                                   // [NN][Q][RT]
  float *M = F + (size_t)NN * Q * RT;                // [Q][RT]
  float *Mp = M + Q * RT;                            // MTTKRP partials
  float *G = Mp + (Q > 128 ? Q : 128) * RT;          // [NN][RT][RT]
  float *Hp = G + NN * RT * RT;
  float *Lc = Hp + RT * RT, *Lr = Lc + RT * RT, *rf = Lr + RT * RT;
  float *red = rf + RT, *scl = red + 8 * RT;
  const bool use_kr = nals_use_kr(NN, Q, RT);
  float *KRo = scl + RT;                                        // [Q^(NN-2)][RT]
  int *Oo = reinterpret_cast<int *>(KRo + ipow(Q, NN - 2) * RT);
  for (int e = tid; e < Q * RT; e += blockDim.x) M[e] = 0.f;   // columns r >= R stay zero
#pragma unroll
  for (int m = 0; m < NN - 1; ++m) {
    for (int e = tid; e < Q * RT; e += blockDim.x)
      F[(size_t)m * Q * RT + e] = a.F[m][(size_t)p * Q * RT + e];
    for (int e = tid; e < RT * RT; e += blockDim.x)
      G[m * RT * RT + e] = a.G0[m][(size_t)p * RT * RT + e];
  }
  __syncthreads();

  auto update = [&](int n, bool normalize) {
    const int ml = n == NN - 1 ? NN - 2 : NN - 1;
    if (tid < 128) {
      for (int e = tid; e < RT * RT; e += 128) {
        float h = 1.f;
#pragma unroll
        for (int m = 0; m < NN; ++m)
          if (m != n && m != ml) h *= G[m * RT * RT + e];
        Hp[e] = h;
      }
      factor_barrier();
      ldl_factor<RT>(Hp, G + ml * RT * RT, R, Craw, Rs, Lc, Lr, rf, &fail_s);
    } else {
      if (use_kr) nals_mttkrp_kr<RT, NN>(X, F, Q, n, M, Mp, KRo, Oo, tid - 128);
      else nals_mttkrp<RT, NN>(X, F, Q, R, n, M, Mp, tid - 128);
    }
    __syncthreads();
    if (fail_s && tid == 0) atomicOr(a.status, kDevCholesky);
    solve_rows_smem<RT>(M, F + (size_t)n * Q * RT, Q, normalize, Lc, Lr, rf, red, scl);
    __syncthreads();
    smem_gram<RT>(F + (size_t)n * Q * RT, Q, G + n * RT * RT);
    __syncthreads();
  };

  for (int it = 0; it < a.iters; ++it) {
    update(NN - 1, false);
    for (int n = 0; n < NN - 1; ++n) update(n, true);
  }
  update(NN - 1, false);
#pragma unroll
  for (int m = 0; m < NN; ++m)
    for (int e = tid; e < Q * RT; e += blockDim.x)
      a.F[m][(size_t)p * Q * RT + e] = F[(size_t)m * Q * RT + e];
}

namespace {

template <int RT, int NN>
bool nals_launch(const NAlsArgs &a, int P, size_t smem, cudaStream_t st) {
  if (cudaFuncSetAttribute(nals_kernel<RT, NN>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)smem) != cudaSuccess)
    return false;
  nals_kernel<RT, NN><<<P, kNThreads, smem, st>>>(a);
  if (cudaGetLastError() != cudaSuccess) return false;
  count_launch();
  return true;
}

template <int RT>
bool nals_dispatch(int NN, const NAlsArgs &a, int P, size_t smem, cudaStream_t st) {
  switch (NN) {
    case 3: return nals_launch<RT, 3>(a, P, smem, st);
    case 4: return nals_launch<RT, 4>(a, P, smem, st);
    case 5: return nals_launch<RT, 5>(a, P, smem, st);
    case 6: return nals_launch<RT, 6>(a, P, smem, st);
    default: return false;
  }
}

constexpr size_t kNalsSmemLimit = 200 * 1024;

}  // namespace

bool nals_fits(int NN, int Q, int RT) {
  return Q <= kNThreads && nals_floats(NN, Q, RT, false) * sizeof(float) <= kNalsSmemLimit;
}

bool nals_run(const NAlsInput &in, cudaStream_t st) {
  const int NN = in.NN, RT = in.RT;
  if (NN < 3 || NN > kMaxNModes || !nals_fits(NN, in.Q, RT)) return false;
  NAlsArgs a{};
  a.Y = in.Y;
  for (int m = 0; m < NN; ++m) a.F[m] = in.F[m];
  for (int m = 0; m < NN - 1; ++m) a.G0[m] = in.G0[m];
  a.Q = in.Q; a.R = in.R; a.iters = in.iters; a.status = in.status;
  const bool xs = nals_floats(NN, in.Q, RT, true) * sizeof(float) <= kNalsSmemLimit;
  a.x_in_smem = xs ? 1 : 0;
  const size_t smem = nals_floats(NN, in.Q, RT, xs) * sizeof(float);
  if (RT == 8) return nals_dispatch<8>(NN, a, in.P, smem, st);
  if (RT == 16) return nals_dispatch<16>(NN, a, in.P, smem, st);
  return nals_dispatch<32>(NN, a, in.P, smem, st);
}

// ---------------------------------------------------------------------------
// Anchor match of the N-mode replicas (fp64), the 3-mode rule mode by mode:
//   sim[r][s] = sum over the non-temporal modes of |cos(F_n[:S, r], ref_n[:, s])|
// (ref_n = rows [0, S) of U_n^T A_n, a cosine with a zero norm counts 0), the
// greedy one-to-one matching, per-mode anchor scales
//   d_n[s] = <F_n[:S, pi(s)], ref_n[:, s]> / ||ref_n[:, s]||^2   (0 -> 1),
// and the aligned factors F_n[:, pi] / d_n, C[:, pi] prod_n d_n.
// grid P, 256 threads.
// ---------------------------------------------------------------------------
struct NAlignArgs {
  const float *F[kMaxNModes];    // raw replica factors, non-temporal modes then time
  const float *PF[kMaxNModes];   // U_n^T A_n, Qd x R (non-temporal modes)
  float *Fh[kMaxNModes];         // aligned factors, same layout as F
  int nm, Q, S, R;
  int *perm;                     // P x R
  double *scales;                // P x nm x R
};

template <int RT>
__global__ void __launch_bounds__(kNThreads) n_align_kernel(NAlignArgs a) {
  __shared__ double sim[RT * RT], nt[RT], nr[RT], prod[RT];
  __shared__ unsigned long long key[RT * RT];
  __shared__ int perm[RT];
  __shared__ float fs[RT];
  const int p = blockIdx.x, tid = threadIdx.x, Q = a.Q, S = a.S, R = a.R;
  for (int e = tid; e < RT * RT; e += blockDim.x) sim[e] = 0.0;
  for (int n = 0; n < a.nm; ++n) {
    const float *F = a.F[n] + (size_t)p * Q * RT;
    const float *ref = a.PF[n];
    __syncthreads();   // the previous mode's norms are consumed
    if (tid < RT) {
      double v = 0.0;
      if (tid < R)
        for (int q = 0; q < S; ++q) {
          const double x = F[q * RT + tid];
          v = fma(x, x, v);
        }
      nt[tid] = sqrt(v);
    } else if (tid < 2 * RT) {
      const int s = tid - RT;
      double v = 0.0;
      if (s < R)
        for (int q = 0; q < S; ++q) {
          const double x = ref[(size_t)q * R + s];
          v = fma(x, x, v);
        }
      nr[s] = sqrt(v);
    }
    __syncthreads();
    for (int e = tid; e < RT * RT; e += blockDim.x) {
      const int r = e / RT, s = e % RT;
      if (r >= R || s >= R) continue;
      double dot = 0.0;
      for (int q = 0; q < S; ++q)
        dot = fma((double)F[q * RT + r], (double)ref[(size_t)q * R + s], dot);
      const double den = nt[r] * nr[s];
      if (den > 0.0) sim[e] += fabs(dot) / den;
    }
  }
  __syncthreads();
  for (int e = tid; e < RT * RT; e += blockDim.x) {
    const int r = e / RT, s = e % RT;
    double v = (r < R && s < R) ? sim[e] : 0.0;
    if (!isfinite(v)) v = 0.0;   // a diverged replica still gets a valid matching
    key[e] = static_cast<unsigned long long>(__double_as_longlong(v));
  }
  if (tid < RT) prod[tid] = 1.0;
  __syncthreads();
  if (tid < 32) greedy_match_warp<RT>(key, R, perm);
  __syncthreads();
  for (int n = 0; n < a.nm; ++n) {
    const float *F = a.F[n] + (size_t)p * Q * RT;
    const float *ref = a.PF[n];
    if (tid < R) {
      const int s = tid, r = perm[s];
      double dot = 0.0, n2 = 0.0;
      for (int q = 0; q < S; ++q) {
        const double x = ref[(size_t)q * R + s];
        dot = fma((double)F[q * RT + r], x, dot);
        n2 = fma(x, x, n2);
      }
      double d = n2 > 0.0 ? dot / n2 : 0.0;
      if (d == 0.0) d = 1.0;
      prod[s] *= d;
      fs[s] = (float)(1.0 / d);
      a.scales[((size_t)p * a.nm + n) * R + s] = d;
    }
    __syncthreads();
    float *Fh = a.Fh[n] + (size_t)p * Q * RT;
    for (int e = tid; e < Q * RT; e += blockDim.x) {
      const int q = e / RT, s = e % RT;
      Fh[e] = s < R ? F[q * RT + perm[s]] * fs[s] : 0.f;
    }
    __syncthreads();   // fs is rewritten by the next mode
  }
  {
    const float *C = a.F[a.nm] + (size_t)p * Q * RT;
    float *Ch = a.Fh[a.nm] + (size_t)p * Q * RT;
    for (int e = tid; e < Q * RT; e += blockDim.x) {
      const int q = e / RT, s = e % RT;
      Ch[e] = s < R ? C[q * RT + perm[s]] * (float)prod[s] : 0.f;
    }
    if (tid < R) a.perm[p * R + tid] = perm[tid];
  }
}

void n_align(const NAlignInput &in, cudaStream_t st) {
  NAlignArgs a{};
  for (int n = 0; n <= in.nm; ++n) {
    a.F[n] = in.F[n];
    a.Fh[n] = in.Fh[n];
  }
  for (int n = 0; n < in.nm; ++n) a.PF[n] = in.PF[n];
  a.nm = in.nm; a.Q = in.Q; a.S = in.S; a.R = in.R; a.perm = in.perm; a.scales = in.scales;
  if (in.RT == 8) n_align_kernel<8><<<in.P, kNThreads, 0, st>>>(a);
  else if (in.RT == 16) n_align_kernel<16><<<in.P, kNThreads, 0, st>>>(a);
  else n_align_kernel<32><<<in.P, kNThreads, 0, st>>>(a);
  count_launch();
}

// ---------------------------------------------------------------------------
// Fitness (Sec. "Evaluation Measures"): per slice k the sums of X_k^2 and of
// (X_k - sum_r C[k][r] A_1[:, r] o ... o A_nm[:, r])^2, the residual formed
// element by element in fp64 (no cancellation against ||X||^2).  grid
// (blocks per slice, slices), 256 threads; partial[k][block][2] doubles.
// ---------------------------------------------------------------------------
struct NFitArgs {
  const void *X;                   // nk slices, [k][i_1]...[i_nm], fp32 or bf16
  int xbf16;
  const float *A[kMaxNModes];      // I_n x R
  const float *C;                  // nk x R (the chunk's rows)
  int64_t dims[kMaxNModes];
  int64_t E;                       // elements per slice
  int nm, R;
  double *partial;
};

__global__ void __launch_bounds__(256) n_fit_kernel(NFitArgs a) {
  __shared__ double red[2][8];
  const int k = blockIdx.y, tid = threadIdx.x;
  const float *x = static_cast<const float *>(a.X) + (int64_t)k * a.E;
  const __nv_bfloat16 *xh = static_cast<const __nv_bfloat16 *>(a.X) + (int64_t)k * a.E;
  const float *c = a.C + (int64_t)k * a.R;
  double s0 = 0.0, s1 = 0.0;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + tid; e < a.E;
       e += (int64_t)gridDim.x * blockDim.x) {
    int64_t idx[kMaxNModes];
    int64_t rem = e;
    for (int n = a.nm - 1; n >= 0; --n) {
      idx[n] = rem % a.dims[n];
      rem /= a.dims[n];
    }
    double model = 0.0;
    for (int r = 0; r < a.R; ++r) {
      double pr = c[r];
      for (int n = 0; n < a.nm; ++n) pr *= (double)a.A[n][idx[n] * a.R + r];
      model += pr;
    }
    const double xv = a.xbf16 ? (double)__bfloat162float(xh[e]) : (double)x[e];
    const double d = xv - model;
    s0 = fma(xv, xv, s0);
    s1 = fma(d, d, s1);
  }
  for (int o = 16; o > 0; o >>= 1) {
    s0 += __shfl_xor_sync(0xffffffffu, s0, o);
    s1 += __shfl_xor_sync(0xffffffffu, s1, o);
  }
  if ((tid & 31) == 0) {
    red[0][tid >> 5] = s0;
    red[1][tid >> 5] = s1;
  }
  __syncthreads();
  if (tid == 0) {
    double t0 = 0.0, t1 = 0.0;
    for (int w = 0; w < 8; ++w) {
      t0 += red[0][w];
      t1 += red[1][w];
    }
    double *pp = a.partial + ((int64_t)k * gridDim.x + blockIdx.x) * 2;
    pp[0] = t0;
    pp[1] = t1;
  }
}

int n_fit_blocks(int64_t E) {
  const int64_t b = (E + 256 * 8 - 1) / (256 * 8);
  return (int)(b < 1 ? 1 : (b > 1024 ? 1024 : b));
}

void n_fit_sums(const void *X, Elem xt, int64_t nk, const float *const *A, const float *C,
                const int64_t *dims, int nm, int R, double *partial, cudaStream_t st) {
  NFitArgs a{};
  a.X = X; a.xbf16 = xt == Elem::BF16; a.C = C; a.nm = nm; a.R = R; a.partial = partial;
  a.E = 1;
  for (int n = 0; n < nm; ++n) {
    a.A[n] = A[n];
    a.dims[n] = dims[n];
    a.E *= dims[n];
  }
  n_fit_kernel<<<dim3((unsigned)n_fit_blocks(a.E), (unsigned)nk), 256, 0, st>>>(a);
  count_launch();
}

// ---------------------------------------------------------------------------
// Compression chain (see the top of the file).
// ---------------------------------------------------------------------------
int64_t ncompress_rows_max(int nm, const int64_t *dims, int Q, int64_t t) {
  int64_t rows = t;
  for (int n = 0; n + 1 < nm; ++n) rows *= dims[n];   // first product: (k, i_1..i_{N-2})
  int64_t best = rows;
  // per-replica elements after the first product: Q rows; contracting mode m
  // leaves rows_out = elements_in / I_m * Q ... tracked as elements
  int64_t elems = rows * Q;
  for (int m = nm - 2; m >= 0; --m) {
    const int64_t rin = elems / dims[m];
    if (rin > best) best = rin;
    elems = rin * Q;
    if (elems > best) best = elems;
  }
  return best;
}

int64_t ncompress_buf_floats(int nm, const int64_t *dims, int P, int Q, int64_t t) {
  int64_t rows = t;
  for (int n = 0; n + 1 < nm; ++n) rows *= dims[n];
  int64_t best = rows * Q;
  int64_t elems = rows * Q;
  for (int m = nm - 2; m >= 0; --m) {
    elems = elems / dims[m] * Q;
    if (elems > best) best = elems;
  }
  return best * P;
}

void ncompress_chunk(const NCompressInput &c, const void *X, Elem xt, int64_t t,
                     const float *Wt, float *Y, cudaStream_t st, const void *Ut16,
                     int *status) {
  const int nm = c.nm, P = c.P, Q = c.Q;
  // 1. innermost mode, all replicas at once: bufA[(p, q)][row] = sum_i
  // X[row][i] Ut[(p, q)][i].  bf16 slices: on the tensor cores as the product
  // Ut . X^T (A = Ut, B = the slice rows, both K-major; the [(p, q)][row]
  // output is row-major in the GEMM's own terms), else on the SIMT kernels.
  int64_t rows = t;
  for (int n = 0; n + 1 < nm; ++n) rows *= c.dims[n];
  const int64_t Il = c.dims[nm - 1];
  bool done = false;
  if (xt == Elem::BF16 && Ut16 && rows <= (int64_t(1) << 30)) {
    TcStoreArgs g{};
    g.A = Ut16; g.a_inner = Il; g.a_rows = (int64_t)P * Q; g.a_rows_per_z = 0;
    g.B = X; g.b_inner = Il; g.b_rows = rows; g.b_rows_per_z = 0;
    g.M = P * Q; g.N = (int)rows; g.K = (int)Il; g.BN = rows >= 256 ? 256 : 128;
    g.batch = 1; g.ksplit = 1;
    g.D = c.bufA; g.s_split = 0; g.s_z = 0; g.s_m = rows;
    g.katoms = 1;
    done = tc_gemm_store(g, status, st);
    if (!done) cudaGetLastError();
  }
  if (!done) {
    GemmArgs g{};
    g.A = X; g.ta = xt; g.sAm = Il; g.sAk = 1;
    g.B = c.Ut[nm - 1]; g.tb = Elem::F32; g.sBn = Il; g.sBk = 1;
    g.D = c.bufA; g.sDm = 1; g.sDn = rows;
    g.M = (int)rows; g.N = P * Q; g.K = (int)Il; g.batch = 1; g.alpha = 1.f; g.beta = 0.f;
    gemm_strided(g, st);
  }
  float *in = c.bufA, *out = c.bufB;
  int64_t elems = rows * Q;   // per replica
  // 2. the other non-temporal modes, innermost first, per replica
  for (int m = nm - 2; m >= 0; --m) {
    const int64_t Im = c.dims[m];
    const int64_t rin = elems / Im;
    GemmArgs g{};
    g.A = in; g.ta = Elem::F32; g.sAz = elems; g.sAm = Im; g.sAk = 1;
    g.B = c.Ut[m]; g.tb = Elem::F32; g.sBz = (int64_t)Q * Im; g.sBn = Im; g.sBk = 1;
    g.D = out; g.sDz = rin * Q; g.sDm = 1; g.sDn = rin;
    g.M = (int)rin; g.N = Q; g.K = (int)Im; g.batch = P; g.alpha = 1.f; g.beta = 0.f;
    g.skinny_batch = true;
    gemm_strided(g, st);
    elems = rin * Q;
    float *tmp = in; in = out; out = tmp;
  }
  // 3. time mode into the summaries
  const int64_t nq = elems / t;   // Q^(N-1)
  GemmArgs g{};
  g.A = in; g.ta = Elem::F32; g.sAz = elems; g.sAm = t; g.sAk = 1;
  g.B = Wt; g.tb = Elem::F32; g.sBz = (int64_t)Q * t; g.sBn = t; g.sBk = 1;
  g.D = Y; g.sDz = nq * Q; g.sDm = Q; g.sDn = 1;
  g.M = (int)nq; g.N = Q; g.K = (int)t; g.batch = P; g.alpha = 1.f; g.beta = 1.f;
  g.skinny_batch = true;
  gemm_strided(g, st);
}

}  // namespace octen
