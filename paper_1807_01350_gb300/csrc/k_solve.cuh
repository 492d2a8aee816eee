// The R x R normal-equation solve of the replica ALS (Algorithm 1's CP(X_p, R)
// step): F_p = M_p (G1_p * G2_p)^-1, with G1, G2 the Grams of the two factors
// that stay fixed in the update and M_p the MTTKRP.
//
// The Hadamard product G = G1 * G2 is factored as G = L D L^T (L unit lower
// triangular) in fp64, then every row of M is solved by fp32 forward and
// backward substitution with L and D^-1 rounded to fp32.
//
// fp64 arithmetic on this GPU issues one warp instruction per ~64 cycles per
// warp (its latency is the same), while the SM as a whole sustains about one
// fp64 warp instruction per ~19 cycles.  The factorisation is therefore spread
// over four warps, one per SM sub-partition, with the dependent chain kept
// apart from the bulk of the arithmetic:
//   warp 0 (pivot warp) owns the diagonal.  At step j it applies column j to
//     the diagonal and forms the next pivot's reciprocal r_{j+1} = 1 / D_{j+1}
//     (fp32 estimate from the bits of D, one Newton step in fp64);
//   warps 1..3 (update warps) own the strictly lower entries, 96 threads with a
//     fixed set of entries each, kept in registers.  At step j every owner of an
//     entry (i, k), k > j, subtracts c_ij c_kj r_j from it; the owners of
//     column j + 1 publish its final (unscaled) values c_{i,j+1} to shared memory.
// One named barrier over the four warps closes each step.
//
// The factor of an update depends only on factors that are already final, so
// it is a kernel of its own (als_ldl_kernel) that runs beside the MTTKRP of the
// update; the solve proper (als_apply_kernel) sums the MTTKRP's partials,
// substitutes, and forms the Gram of the factor it writes (for the factors of
// the next updates), with a cluster of CTAs per replica.
#pragma once

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

// Gram of the Q x RT factor held in shared memory: Gout[r][s] = sum_q F[q][r] F[q][s].
// Thread t < (RT/2)^2 accumulates the 2 x 2 block at rows 2 (t / (RT/2)), columns
// 2 (t % (RT/2)) with two 8-byte shared loads per row of F.
template <int RT>
__device__ __forceinline__ void smem_gram(const float *Fs, int Q, float *Gout) {
  constexpr int H = RT / 2;
  const int t = threadIdx.x;
  if (t >= H * H) return;
  const int r0 = 2 * (t / H), c0 = 2 * (t % H);
  float a00 = 0.f, a01 = 0.f, a10 = 0.f, a11 = 0.f;
#pragma unroll 4
  for (int q = 0; q < Q; ++q) {
    const float2 x = *reinterpret_cast<const float2 *>(Fs + q * RT + r0);
    const float2 y = *reinterpret_cast<const float2 *>(Fs + q * RT + c0);
    a00 = fmaf(x.x, y.x, a00);
    a01 = fmaf(x.x, y.y, a01);
    a10 = fmaf(x.y, y.x, a10);
    a11 = fmaf(x.y, y.y, a11);
  }
  Gout[r0 * RT + c0] = a00;
  Gout[r0 * RT + c0 + 1] = a01;
  Gout[(r0 + 1) * RT + c0] = a10;
  Gout[(r0 + 1) * RT + c0 + 1] = a11;
}

// Reciprocal of a pivot.  ok is cleared unless d is positive, normal and finite.
// For d in [2^-100, 2^100] (every pivot of a Gram of bounded columns): the
// fp32 value of d is assembled from its bits (mantissa truncated to 23 bits,
// relative error < 2^-23), its reciprocal taken with rcp.approx (relative
// error < 2^-23), the result widened to fp64 from its bits, and one Newton
// step y <- y + y (1 - d y) squares the relative error (< 2^-43).  No fp64
// conversion instructions sit on the chain; outside that range the fp64
// division is used.
__device__ __forceinline__ double pivot_rcp(double d, bool &ok) {
  const int hi = __double2hiint(d);
  const unsigned lo = static_cast<unsigned>(__double2loint(d));
  const int be = (hi >> 20) & 0x7ff;   // biased exponent of |d|
  if (hi < 0 || be == 0 || be == 0x7ff) {
    ok = false;   // negative, zero, subnormal, infinite or NaN
    return 0.0;
  }
  if (be < 1023 - 100 || be > 1023 + 100) return 1.0 / d;
  const float f = __int_as_float(((be - 1023 + 127) << 23) | ((hi & 0xfffff) << 3) |
                                 static_cast<int>(lo >> 29));
  float y;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(f));
  const int yb = __float_as_int(y);
  const int ye = (yb >> 23) & 0xff;
  const int ym = yb & 0x7fffff;
  const double y0 = __hiloint2double(((ye - 127 + 1023) << 20) | (ym >> 3), ym << 29);
  const double e = fma(-d, y0, 1.0);
  return fma(y0, e, y0);
}

__device__ __forceinline__ void factor_barrier() { asm volatile("bar.sync 1, 128;" ::: "memory"); }

// Warps 0..3: G = G1 * G2 (fp64) = L D L^T.  On return (after a barrier over
// the four warps) Lc[k][i] = Lr[i][k] = L[i][k] for i > k (fp32, zero elsewhere)
// and rf[k] = 1 / D[k] (fp32, zero for k >= R).  If a pivot is not positive the
// diagonal is loaded by 1e-12 trace / R and the factorisation repeated once; if
// that fails as well, L = I and rf = 1 (the solve returns M) and *fail = 1.
template <int RT>
__device__ void ldl_factor(const float *__restrict__ g1, const float *__restrict__ g2, int R,
                           double *Craw /*[RT][RT+1]*/, double *Rs /*[RT]*/, float *Lc,
                           float *Lr, float *rf, int *fail) {
  constexpr int LD = RT + 1;
  constexpr int NU = 96;                                   // update threads
  constexpr int NS = (RT * (RT - 1) / 2 + NU - 1) / NU;    // entries per update thread
  const unsigned full = 0xffffffffu;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  for (int e = tid; e < RT * RT; e += 128) {
    Lc[e] = 0.f;
    Lr[e] = 0.f;
  }
  // entries of update thread u: the strict lower triangle listed by column k
  // descending (column R-2 first), entry e = s * NU + u in slot s.  Group g >= 1
  // of that list is column k = R-1-g with rows k+1 .. R-1.
  const int u = tid - 32;
  const int nent = R * (R - 1) / 2;
  int ei[NS > 0 ? NS : 1], ek[NS > 0 ? NS : 1];
  double a[NS > 0 ? NS : 1];
#pragma unroll
  for (int s = 0; s < NS; ++s) {
    ei[s] = 0;
    ek[s] = -1;
    a[s] = 0.0;
    const int e = s * NU + u;
    if (warp > 0 && e < nent) {
      int g = 1;
      while ((g + 1) * g / 2 <= e) ++g;
      const int k = R - 1 - g;
      ek[s] = k;
      ei[s] = k + 1 + (e - g * (g - 1) / 2);
    }
  }
  bool ok = true;
  for (int attempt = 0; attempt < 2; ++attempt) {
    ok = true;
    if (warp == 0) {
      // pivot warp: lane t holds diagonal entry t
      double diag = lane < R ? (double)g1[lane * (RT + 1)] * (double)g2[lane * (RT + 1)] : 1.0;
      if (attempt == 1) {
        double tr = lane < R ? diag : 0.0;
        for (int o = 16; o > 0; o >>= 1) tr += __shfl_xor_sync(full, tr, o);
        diag += 1e-12 * tr / R;
      }
      double rj = pivot_rcp(__shfl_sync(full, diag, 0), ok);
      if (lane == 0) Rs[0] = rj;
      factor_barrier();   // column 0 and r_0 published
      for (int j = 0; j + 1 < R; ++j) {
        const double ct = (lane > j && lane < R) ? Craw[lane * LD + j] : 0.0;
        diag = fma(-ct, ct * rj, diag);
        rj = pivot_rcp(__shfl_sync(full, diag, j + 1), ok);
        if (!ok) rj = 0.0;
        if (lane == 0) Rs[j + 1] = rj;
        factor_barrier();
      }
      if (lane == 0) *fail = ok ? 0 : 1;
    } else {
      // update warps: entries in registers, column j + 1 published at step j
#pragma unroll
      for (int s = 0; s < NS; ++s) {
        if (ek[s] >= 0) {
          const int i = ei[s], k = ek[s];
          a[s] = (double)g1[i * RT + k] * (double)g2[i * RT + k];
          if (k == 0) Craw[i * LD] = a[s];
        }
      }
      factor_barrier();
      for (int j = 0; j + 1 < R; ++j) {
        const double rj = Rs[j];
        const double ct = (lane > j && lane < R) ? Craw[lane * LD + j] : 0.0;
        const double st = ct * rj;
        const int na = (R - 2 - j) * (R - 1 - j) / 2;   // entries with column > j
#pragma unroll
        for (int s = 0; s < NS; ++s) {
          if (s * NU + (warp - 1) * 32 < na) {   // warp-uniform
            const double ci = __shfl_sync(full, ct, ei[s]);
            const double sk = __shfl_sync(full, st, ek[s] < 0 ? 0 : ek[s]);
            if (s * NU + u < na) {
              a[s] = fma(-ci, sk, a[s]);
              if (ek[s] == j + 1) Craw[ei[s] * LD + ek[s]] = a[s];
            }
          }
        }
        factor_barrier();
      }
    }
    factor_barrier();   // *fail visible to the four warps
    if (!*fail) break;
  }
  ok = !*fail;
  if (warp == 0) {
    if (lane < RT) rf[lane] = lane < R ? (ok ? (float)Rs[lane] : 1.f) : 0.f;
  } else if (ok) {
#pragma unroll
    for (int s = 0; s < NS; ++s) {
      if (ek[s] >= 0) {
        const float l = (float)(a[s] * Rs[ek[s]]);
        Lc[ek[s] * RT + ei[s]] = l;
        Lr[ei[s] * RT + ek[s]] = l;
      }
    }
  }
}

// y <- y (L D L^T)^-1 for one row y (the matrix symmetric): forward
// substitution with the unit lower L (column-major Lc[k][i] = L[i][k]), scaling
// by rf = 1/D, backward substitution with L^T (row-major Lr[k][i] = L[k][i]).
// Entries beyond the rank are zero in Lc, Lr and rf, so padded columns stay 0.
template <int RT>
__device__ __forceinline__ void ldl_substitute(float (&y)[RT], const float *Lc, const float *Lr,
                                               const float *rf) {
#pragma unroll
  for (int k = 0; k < RT; ++k) {
    const float yk = y[k];
    const float4 *lc = reinterpret_cast<const float4 *>(Lc + k * RT);
#pragma unroll
    for (int i4 = (k + 1) / 4; i4 < RT / 4; ++i4) {
      const float4 l = lc[i4];
      if (4 * i4 + 0 > k) y[4 * i4 + 0] = fmaf(-l.x, yk, y[4 * i4 + 0]);
      if (4 * i4 + 1 > k) y[4 * i4 + 1] = fmaf(-l.y, yk, y[4 * i4 + 1]);
      if (4 * i4 + 2 > k) y[4 * i4 + 2] = fmaf(-l.z, yk, y[4 * i4 + 2]);
      if (4 * i4 + 3 > k) y[4 * i4 + 3] = fmaf(-l.w, yk, y[4 * i4 + 3]);
    }
  }
#pragma unroll
  for (int r4 = 0; r4 < RT / 4; ++r4) {
    const float4 d = reinterpret_cast<const float4 *>(rf)[r4];
    y[4 * r4] *= d.x; y[4 * r4 + 1] *= d.y; y[4 * r4 + 2] *= d.z; y[4 * r4 + 3] *= d.w;
  }
#pragma unroll
  for (int k = RT - 1; k > 0; --k) {
    const float fk = y[k];
    const float4 *lr = reinterpret_cast<const float4 *>(Lr + k * RT);
#pragma unroll
    for (int i4 = 0; i4 <= (k - 1) / 4; ++i4) {
      const float4 l = lr[i4];
      if (4 * i4 + 0 < k) y[4 * i4 + 0] = fmaf(-l.x, fk, y[4 * i4 + 0]);
      if (4 * i4 + 1 < k) y[4 * i4 + 1] = fmaf(-l.y, fk, y[4 * i4 + 1]);
      if (4 * i4 + 2 < k) y[4 * i4 + 2] = fmaf(-l.z, fk, y[4 * i4 + 2]);
      if (4 * i4 + 3 < k) y[4 * i4 + 3] = fmaf(-l.w, fk, y[4 * i4 + 3]);
    }
  }
}

// Per replica: the packed factor written by als_ldl_kernel and read by
// als_apply_kernel, [Lc (RT x RT) | Lr (RT x RT) | rf (RT)] floats.
template <int RT>
__host__ __device__ constexpr int factor_floats() { return 2 * RT * RT + RT; }

// Whole CTA (Q <= blockDim.x, a multiple of 32): rows q < Q of M (Q x RT,
// shared) solved against the factor in (Lc, Lr, rf) into F; with `normalize`
// the columns are scaled to unit l2 (norms over the CTA).
template <int RT>
__device__ void solve_rows_smem(const float *M, float *F, int Q, bool normalize,
                                const float *Lc, const float *Lr, const float *rf, float *red,
                                float *scl) {
  const int tid = threadIdx.x;
  const bool own = tid < Q;
  float y[RT];
#pragma unroll
  for (int r = 0; r < RT; ++r) y[r] = own ? M[tid * RT + r] : 0.f;
  if (own) ldl_substitute<RT>(y, Lc, Lr, rf);
  if (normalize) {
    float sq[RT];
#pragma unroll
    for (int r = 0; r < RT; ++r) sq[r] = y[r] * y[r];
    block_sum_rows<RT>(sq, red, scl);
    if (tid < RT) {
      const float n = sqrtf(scl[tid]);
      red[tid] = n > 0.f ? 1.f / n : 1.f;   // reciprocal norm per column
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < RT; ++r) y[r] *= red[r];
  }
  if (own) {
#pragma unroll
    for (int r = 0; r < RT; ++r) F[tid * RT + r] = y[r];
  }
}

// L D L^T factor of Gnew_p * Gother_p -> Lout_p (the Grams of the two factors
// that stay fixed in the update, already formed by the solves that wrote
// them).  It depends only on factors that are already final, so it runs beside
// the MTTKRP of the same update.  grid P, 128 threads (the four factor warps).
template <int RT>
__global__ void __launch_bounds__(128)
    als_ldl_kernel(const float *__restrict__ Gnew, const float *__restrict__ Gother, int R,
                   float *__restrict__ Lout, int *status) {
  __shared__ __align__(16) float G1[RT * RT], G2[RT * RT];
  __shared__ double Craw[RT * (RT + 1)], Rs[RT];
  __shared__ __align__(16) float Lc[RT * RT], Lr[RT * RT], rf[RT];
  __shared__ int fail_s;
  const int p = blockIdx.x, tid = threadIdx.x;
  const float4 *g1 = reinterpret_cast<const float4 *>(Gnew + (int64_t)p * RT * RT);
  const float4 *g2 = reinterpret_cast<const float4 *>(Gother + (int64_t)p * RT * RT);
  for (int e = tid; e < RT * RT / 4; e += blockDim.x) {
    reinterpret_cast<float4 *>(G1)[e] = g1[e];
    reinterpret_cast<float4 *>(G2)[e] = g2[e];
  }
  __syncthreads();
  ldl_factor<RT>(G1, G2, R, Craw, Rs, Lc, Lr, rf, &fail_s);
  __syncthreads();
  if (fail_s && tid == 0) atomicOr(status, kDevCholesky);
  float *lo = Lout + (int64_t)p * factor_floats<RT>();
  for (int e = tid; e < RT * RT; e += blockDim.x) {
    lo[e] = Lc[e];
    lo[RT * RT + e] = Lr[e];
  }
  if (tid < RT) lo[2 * RT * RT + tid] = rf[tid];
}

__device__ __forceinline__ uint32_t cluster_rank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}
__device__ __forceinline__ uint32_t cluster_size() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_nctarank;" : "=r"(r));
  return r;
}
__device__ __forceinline__ void cluster_barrier() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::
                   : "memory");
}
// fp32 at the same shared-memory offset in CTA `rank` of the cluster
__device__ __forceinline__ float ld_cluster(const float *p, uint32_t rank) {
  const uint32_t a = static_cast<uint32_t>(__cvta_generic_to_shared(p));
  uint32_t ra;
  float v;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(ra) : "r"(a), "r"(rank));
  asm volatile("ld.shared::cluster.f32 %0, [%1];" : "=f"(v) : "r"(ra) : "memory");
  return v;
}

// Rows [row0, row0 + nrows) of M_p summed over `nsplit` partial MTTKRPs into
// Ms (nrows x RT): row q of split s at M + s * split_stride + (p * Q + q) *
// row_stride, or with segQ > 0 the segmented partials m1_part[p][j][2][RT] of
// the blocks j of 32 rows (q', i) that hold rows of q (segment 0 if the block
// starts in q).  RT / 4 threads per row, a float4 of columns each.
template <int RT>
__device__ __forceinline__ void sum_partial_rows(const float *__restrict__ M, int nsplit,
                                                 int64_t split_stride, int64_t row_stride,
                                                 int segQ, int p, int Q, int row0, int nrows,
                                                 float *Ms) {
  constexpr int TPR = RT / 4;
  for (int e = threadIdx.x; e < nrows * TPR; e += blockDim.x) {
    const int rr = e / TPR, c4 = e - (e / TPR) * TPR;
    if (segQ > 0) {
      const int q = row0 + rr;
      const int64_t nblk = ((int64_t)segQ * segQ + 31) / 32;
      const int64_t first = (int64_t)q * segQ, last = first + segQ - 1;
      float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
      for (int64_t j = first / 32; j <= last / 32; ++j) {
        const int sgm = (32 * j) / segQ == q ? 0 : 1;
        const float4 v = *reinterpret_cast<const float4 *>(
            M + (((int64_t)p * nblk + j) * 2 + sgm) * RT + 4 * c4);
        acc.x += v.x; acc.y += v.y; acc.z += v.z; acc.w += v.w;
      }
      *reinterpret_cast<float4 *>(Ms + rr * RT + 4 * c4) = acc;
      continue;
    }
    const float *base = M + ((int64_t)p * Q + row0 + rr) * row_stride + 4 * c4;
    float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
    int sp = 0;
    for (; sp + 4 <= nsplit; sp += 4) {
      const float4 v0 = *reinterpret_cast<const float4 *>(base + (sp + 0) * split_stride);
      const float4 v1 = *reinterpret_cast<const float4 *>(base + (sp + 1) * split_stride);
      const float4 v2 = *reinterpret_cast<const float4 *>(base + (sp + 2) * split_stride);
      const float4 v3 = *reinterpret_cast<const float4 *>(base + (sp + 3) * split_stride);
      acc.x += (v0.x + v1.x) + (v2.x + v3.x);
      acc.y += (v0.y + v1.y) + (v2.y + v3.y);
      acc.z += (v0.z + v1.z) + (v2.z + v3.z);
      acc.w += (v0.w + v1.w) + (v2.w + v3.w);
    }
    for (; sp < nsplit; ++sp) {
      const float4 v = *reinterpret_cast<const float4 *>(base + sp * split_stride);
      acc.x += v.x; acc.y += v.y; acc.z += v.z; acc.w += v.w;
    }
    *reinterpret_cast<float4 *>(Ms + rr * RT + 4 * c4) = acc;
  }
}

// y = row `threadIdx.x` of Ms solved against L D L^T (zero for threads past
// the CTA's rows).
template <int RT>
__device__ __forceinline__ void solve_own_row(const float *Ms, bool own, const float *Lc,
                                              const float *Lr, const float *rf, float (&y)[RT]) {
#pragma unroll
  for (int r = 0; r < RT; ++r) y[r] = 0.f;
  if (own) {
    const float4 *mr = reinterpret_cast<const float4 *>(Ms + threadIdx.x * RT);
#pragma unroll
    for (int r4 = 0; r4 < RT / 4; ++r4) {
      const float4 v = mr[r4];
      y[4 * r4] = v.x; y[4 * r4 + 1] = v.y; y[4 * r4 + 2] = v.z; y[4 * r4 + 3] = v.w;
    }
    ldl_substitute<RT>(y, Lc, Lr, rf);
  }
}

template <int RT>
__device__ __forceinline__ void store_row(float *dst, const float (&y)[RT]) {
  float4 *o = reinterpret_cast<float4 *>(dst);
#pragma unroll
  for (int r4 = 0; r4 < RT / 4; ++r4)
    o[r4] = make_float4(y[4 * r4], y[4 * r4 + 1], y[4 * r4 + 2], y[4 * r4 + 3]);
}

// Column norms and Gram of the solved rows over the cluster.  One reduction
// serves both: the Gram of the unnormalised rows (per CTA into Gp, then summed
// over the cluster in rank order) has the squared column norms on its
// diagonal, and the Gram of the normalised factor is that Gram scaled by
// 1 / (n_r n_s).  On return scale[r] = 1 / n_r (1 for a zero column) and this
// CTA's share of the normalised Gram, entries [e0, e1) with e0 = rank * RT^2 /
// size, is in Gout_p; peers may still be reading Gp, so the caller closes with
// a cluster barrier before Gp is written again or the CTA exits.
template <int RT>
__device__ __forceinline__ void cluster_gram_scale(const float (&y)[RT], bool own, float *Ms,
                                                   int nrows, float *Gp, float *scale,
                                                   float *__restrict__ Gout_p, uint32_t crank,
                                                   uint32_t ncta) {
  const int tid = threadIdx.x;
  __syncthreads();   // every row of Ms has been read
  if (own) store_row<RT>(Ms + tid * RT, y);
  __syncthreads();
  smem_gram<RT>(Ms, nrows, Gp);
  cluster_barrier();   // every CTA's partial Gram is in place
  if (tid < RT) {
    float tot = 0.f;
    for (uint32_t c = 0; c < ncta; ++c) tot += ld_cluster(Gp + tid * (RT + 1), c);
    const float n = sqrtf(tot);
    scale[tid] = n > 0.f ? 1.f / n : 1.f;   // reciprocal norm per column
  }
  __syncthreads();   // scale visible CTA-wide
  const int e0 = (int)(crank * (RT * RT) / ncta), e1 = (int)((crank + 1) * (RT * RT) / ncta);
  for (int e = e0 + tid; e < e1; e += blockDim.x) {
    float g = 0.f;
    for (uint32_t c = 0; c < ncta; ++c) g += ld_cluster(Gp + e, c);
    Gout_p[e] = g * scale[e / RT] * scale[e % RT];
  }
}

// Row q of F_p (and, with Ft, column q of its bf16 transpose [NP][Q], rows >= RT zero).
template <int RT>
__device__ __forceinline__ void store_factor_row(const float (&y)[RT], float *__restrict__ F,
                                                 __nv_bfloat16 *__restrict__ Ft, int NP, int p,
                                                 int Q, int q) {
  store_row<RT>(F + ((int64_t)p * Q + q) * RT, y);
  if (Ft) {
#pragma unroll
    for (int r = 0; r < RT; ++r) Ft[((int64_t)p * NP + r) * Q + q] = __float2bfloat16_rn(y[r]);
    for (int r = RT; r < NP; ++r) Ft[((int64_t)p * NP + r) * Q + q] = __float2bfloat16_rn(0.f);
  }
}

// F_p = M_p (L D L^T)^-1 for rows [rank * rows_per_cta, ...) of replica p,
// M_p the sum of `nsplit` partial MTTKRPs (sum_partial_rows).  A cluster of
// CTAs shares a replica (grid P * cluster size); with `normalize` the column
// norms are summed over the cluster through distributed shared memory and the
// columns scaled to unit l2.  Writes F_p and, if Ft is given, a bf16 copy
// transposed to [NP][Q] (rows >= R zero) for the tensor-core passes; with Gout
// the Gram F_p^T F_p (each CTA's rows, then the partials summed over the
// cluster in rank order).  256 threads; dynamic smem rows_per_cta * RT floats.
template <int RT>
__global__ void __launch_bounds__(256)
    als_apply_kernel(const float *__restrict__ M, int nsplit, int64_t split_stride,
                     int64_t row_stride, const float *__restrict__ Lin, float *__restrict__ F,
                     __nv_bfloat16 *__restrict__ Ft, int NP, int Q, int rows_per_cta,
                     int normalize, float *__restrict__ Gout, int segQ) {
  extern __shared__ __align__(16) float Ms[];   // [rows_per_cta][RT]
  __shared__ __align__(16) float Lc[RT * RT], Lr[RT * RT], rf[RT], Gp[RT * RT];
  __shared__ float red[8 * RT], part[RT], scale[RT];
  pdl_trigger();
  pdl_wait();   // the MTTKRP partials are the previous kernel's
  const int tid = threadIdx.x;
  const uint32_t ncta = cluster_size(), crank = cluster_rank();
  const int p = blockIdx.x / ncta;
  const int row0 = crank * rows_per_cta;
  const int nrows = Q - row0 < rows_per_cta ? (Q - row0 > 0 ? Q - row0 : 0) : rows_per_cta;
  {
    const float4 *li = reinterpret_cast<const float4 *>(Lin + (int64_t)p * factor_floats<RT>());
    float4 *lc = reinterpret_cast<float4 *>(Lc), *lr = reinterpret_cast<float4 *>(Lr);
    for (int e = tid; e < RT * RT / 4; e += blockDim.x) {
      lc[e] = li[e];
      lr[e] = li[RT * RT / 4 + e];
    }
    if (tid < RT) rf[tid] = Lin[(int64_t)p * factor_floats<RT>() + 2 * RT * RT + tid];
  }
  sum_partial_rows<RT>(M, nsplit, split_stride, row_stride, segQ, p, Q, row0, nrows, Ms);
  __syncthreads();

  // f = M row solved against L D L^T: forward with L, scale by 1/D, backward with L^T
  const bool own = tid < nrows;
  float y[RT];
  solve_own_row<RT>(Ms, own, Lc, Lr, rf, y);
  if (normalize && Gout) {
    cluster_gram_scale<RT>(y, own, Ms, nrows, Gp, scale, Gout + (int64_t)p * RT * RT, crank, ncta);
    cluster_barrier();   // peers are done reading Gp
#pragma unroll
    for (int r = 0; r < RT; ++r) y[r] *= scale[r];
    if (own) store_factor_row<RT>(y, F, Ft, NP, p, Q, row0 + tid);
    return;
  }
  if (normalize) {
    // column sums of squares over this CTA's rows, then over the cluster
    float sq[RT];
#pragma unroll
    for (int r = 0; r < RT; ++r) sq[r] = y[r] * y[r];
    block_sum_rows<RT>(sq, red, part);
    cluster_barrier();   // every CTA's partial sums are in place
    if (tid < RT) {
      float tot = 0.f;
      for (uint32_t c = 0; c < ncta; ++c) tot += ld_cluster(part + tid, c);
      const float n = sqrtf(tot);
      scale[tid] = n > 0.f ? 1.f / n : 1.f;   // reciprocal norm per column
    }
    cluster_barrier();   // peers are done reading `part`; `scale` visible CTA-wide
#pragma unroll
    for (int r = 0; r < RT; ++r) y[r] *= scale[r];
  }
  if (own) store_factor_row<RT>(y, F, Ft, NP, p, Q, row0 + tid);
  if (Gout) {
    __syncthreads();   // every row of Ms has been read
    if (own) store_row<RT>(Ms + tid * RT, y);
    __syncthreads();
    smem_gram<RT>(Ms, nrows, Gp);
    cluster_barrier();   // every CTA's partial Gram is in place
    const int e0 = (int)(crank * (RT * RT) / ncta), e1 = (int)((crank + 1) * (RT * RT) / ncta);
    for (int e = e0 + tid; e < e1; e += blockDim.x) {
      float g = 0.f;
      for (uint32_t c = 0; c < ncta; ++c) g += ld_cluster(Gp + e, c);
      Gout[(int64_t)p * RT * RT + e] = g;
    }
    cluster_barrier();   // peers are done reading Gp
  }
}

}  // namespace octen
