// Tensor-core contractions of the compression step (Sec. "Parallel
// Compression and Decomposition": the mode-2 and mode-1 products of
// Z_p = X x1 U_p^T x2 V_p^T x3 W_p^T) on sm_103a: tcgen05.mma with the
// accumulator in tensor memory, operands staged by TMA (128-byte swizzle) in
// a multi-stage shared-memory ring, one CTA per 128 x BN output tile.
//
//   warp 0 lane 0 : TMA producer   (full[s] <- bytes landed)
//   warp 1 lane 0 : MMA issuer     (empty[s] <- tcgen05.commit, acc <- last commit)
//   warps 0..3    : epilogue, each reading its 32 TMEM lanes with tcgen05.ld
//
// Every wait on an mbarrier is bounded by a clock budget; on expiry the CTA
// raises kDevTimeout in the status word, skips the rest of its work, still
// waits (bounded) for the MMAs it issued and frees its tensor memory.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <array>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>

#include "octen_internal.cuh"

namespace octen {

namespace {

constexpr int kBM = 128;          // UMMA M (cta_group::1)
constexpr int kRowBytes = 128;    // one 128-byte swizzle row of K per operand row
constexpr long long kWaitBudget = 4000000000LL;   // ~2 s at 2 GHz

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Bounded wait; false after `budget` clock cycles or when another role raised
// the abort flag.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity,
                                          volatile int *abort_flag, long long budget) {
  const long long t0 = clock64();
  while (!mbar_try_wait(bar, parity)) {
    if (*abort_flag) return false;
    if (clock64() - t0 > budget) return false;
  }
  return true;
}

__device__ __forceinline__ void tma_load_2d(void *dst, const CUtensorMap *map, uint64_t *bar,
                                            int x, int y) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3}], [%4];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_u32(bar))
      : "memory");
}

// Same load with an L2 cache policy (from createpolicy) attached.
__device__ __forceinline__ void tma_load_2d_policy(void *dst, const CUtensorMap *map, uint64_t *bar,
                                                   int x, int y, uint64_t policy) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint"
      " [%0], [%1, {%2, %3}], [%4], %5;" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_u32(bar)), "l"(policy)
      : "memory");
}

// L2 policy that keeps the lines it touches in the L2 as long as it can (an
// output that the next kernel reads again).
__device__ __forceinline__ uint64_t policy_evict_last() {
  uint64_t p;
  asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
  return p;
}

// 16-byte global store with an L2 cache policy attached.
__device__ __forceinline__ void st_global_v4_policy(void *ptr, uint4 v, uint64_t pol) {
  asm volatile("st.global.L2::cache_hint.v4.u32 [%0], {%1, %2, %3, %4}, %5;" ::"l"(ptr),
               "r"(v.x), "r"(v.y), "r"(v.z), "r"(v.w), "l"(pol)
               : "memory");
}

__device__ __forceinline__ uint64_t policy_evict_first() {
  uint64_t p;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
  return p;
}

__device__ __forceinline__ void tmem_alloc(uint32_t *holder, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                   smem_u32(holder)),
               "r"(ncols));
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
}

__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols));
}

__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

template <int KIND>
__device__ __forceinline__ void mma_issue(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc,
                                          uint32_t idesc, uint32_t accumulate) {
  if constexpr (KIND == 0) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem_d),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate));
  } else {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem_d),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate));
  }
}

__device__ __forceinline__ void mma_commit(uint64_t *bar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
          smem_u32(bar))
      : "memory");
}

// 32 lanes x 32 columns of fp32 from tensor memory (lane = warp quadrant + lane id).
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&r)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
      "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
      "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]),
        "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]),
        "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// Shared-memory matrix descriptor of a K-major operand tile stored as 128-byte
// rows with the 128-byte swizzle (TMA SWIZZLE_128B): 8-row groups 1024 B apart.
__device__ __forceinline__ uint64_t make_desc_sw128(uint32_t saddr) {
  uint64_t d = 0;
  d |= static_cast<uint64_t>((saddr & 0x3FFFFu) >> 4);   // start address
  d |= static_cast<uint64_t>(1) << 16;                    // leading offset (unused here)
  d |= static_cast<uint64_t>(1024 >> 4) << 32;            // stride offset: 8 rows x 128 B
  d |= static_cast<uint64_t>(1) << 46;                    // descriptor version
  d |= static_cast<uint64_t>(2) << 61;                    // 128-byte swizzle
  return d;
}

// Instruction descriptor: fp32 accumulate, both operands K-major, M = 128.
// KIND 0: bf16 x bf16 (kind::f16); KIND 1: e4m3 x e4m3 (kind::f8f6f4).
__host__ __device__ constexpr uint32_t make_idesc(int KIND, int N) {
  return (1u << 4) |                                   // D format f32
         ((KIND == 0 ? 1u : 0u) << 7) |                 // A format: bf16 / e4m3
         ((KIND == 0 ? 1u : 0u) << 10) |                // B format: bf16 / e4m3
         (static_cast<uint32_t>(N >> 3) << 17) |        // N / 8
         (static_cast<uint32_t>(kBM >> 4) << 24);       // M / 16
}

struct TcShape {
  int M, N, K;          // per batch item (K in elements)
  int BN;               // tile N (multiple of 32, <= 256)
  int stages;
  int tmem_cols;        // power of two >= BN
  int zdiv;             // batch index z -> rows (z / zdiv) * hi + (z % zdiv) * lo
  int a_hi, a_lo, b_hi, b_lo;
  int ksplit;           // > 1: blockIdx.x is the K split (a single N tile)
  int a_stream;         // A is read once: load it with an L2 evict-first policy
  int katoms;           // 128-byte K atoms per pipeline stage (1, 2 or 4)
  long long wait_budget;   // clock cycles a pipeline wait may take before the CTA
                           // gives up (the drains after a give-up keep kWaitBudget)
};

// Plain store: D[split * s_split + z * s_z + m * s_m + n] (split-K partials), in
// fp32, or rounded to bf16 at the same offsets of Dh when Dh is given.
struct TcStoreEpi {
  static constexpr bool kRowMajor = true;   // rows are contiguous in n
  static constexpr bool kSeg = false;
  static constexpr bool kBf16Rows = true;   // may store bf16 rows (Dh)
  float *D;
  int64_t s_split, s_z, s_m;
  // optional fused reduction (replica ALS): with rows m = a * Q + b, every warp
  // block of 32 rows (one a, 32 consecutive b) also writes
  //   part[z][m / 32][n] = sum_{i < 32} D(m + i, n) * Bfac[z][b + i][n]
  const float *Bfac;
  float *part;
  int Q, RT;
  __nv_bfloat16 *Dh;
  int seg;    // segmented partials (32 does not divide Q)
  int keep;   // bf16 rows stored with an L2 evict-last policy (read again soon)
  __device__ __forceinline__ bool stores() const { return D != nullptr || Dh != nullptr; }
  __device__ __forceinline__ void store(int z, int split, int m, int n, float v) const {
    const int64_t o = (int64_t)split * s_split + (int64_t)z * s_z + (int64_t)m * s_m + n;
    if (Dh) Dh[o] = __float2bfloat16_rn(v);
    else D[o] = v;
  }
  // 8 bf16 values of row m from column n (n % 8 == 0; strides multiples of 8)
  __device__ __forceinline__ void store_bf16x8(int z, int split, int m, int n, uint4 v) const {
    const int64_t o = (int64_t)split * s_split + (int64_t)z * s_z + (int64_t)m * s_m + n;
    if (keep) st_global_v4_policy(Dh + o, v, policy_evict_last());
    else *reinterpret_cast<uint4 *>(Dh + o) = v;
  }
};

// Mode-2 epilogue: row m = k * I + i, column c of V_all -> every replica owning c.
struct Mode2TcEpi {
  static constexpr bool kRowMajor = false;
  static constexpr bool kSeg = true;   // 16-byte segments along i when I % 8 == 0
  __nv_bfloat16 *T;
  const float *scale;
  int64_t I;
  int P, Q, S;
  bool seg;
  __device__ __forceinline__ float row_scale(int64_t m) const {
    return scale ? scale[m / I] : 1.f;
  }
  // A warp's 32 rows (m_w .. m_w + 31) x 32 columns (c_base ..) staged as bf16
  // in stg[column][row]: lane l writes rows m_w + 8 (l % 4) .. + 7 of columns
  // c_base + 8 q + l / 4, q < 4, as one 16-byte store per replica that owns the
  // column.  With I % 8 == 0 those 8 rows lie in one slice and start 16-byte
  // aligned in T.
  __device__ __forceinline__ void store_chunk(const __nv_bfloat16 *stg, int64_t m_w, int c_base,
                                              int64_t M, int N, int lane) const {
    const int sg = lane & 3;
    const int64_t mseg = m_w + 8 * sg;
    if (mseg >= M) return;
    const int64_t k = mseg / I, i = mseg - k * I;
    __nv_bfloat16 *Tk = T + (k * P * Q) * I + i;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int j = 8 * q + (lane >> 2);
      const int c = c_base + j;
      if (c >= N) continue;
      const uint4 v = *reinterpret_cast<const uint4 *>(stg + j * 32 + 8 * sg);
      if (c < S) {
        for (int p = 0; p < P; ++p)
          *reinterpret_cast<uint4 *>(Tk + ((int64_t)p * Q + c) * I) = v;
      } else {
        const int p = (c - S) / (Q - S);
        const int b = S + (c - S) - p * (Q - S);
        *reinterpret_cast<uint4 *>(Tk + ((int64_t)p * Q + b) * I) = v;
      }
    }
  }
  __device__ __forceinline__ void operator()(int, int, int m, int c, float v) const {
    const int64_t k = m / I, i = m - k * I;
    if (scale) v *= scale[k];
    const __nv_bfloat16 h = __float2bfloat16_rn(v);
    if (c < S) {
      for (int p = 0; p < P; ++p) T[((k * P + p) * Q + c) * I + i] = h;
    } else {
      const int p = (c - S) / (Q - S);
      const int b = S + (c - S) - p * (Q - S);
      T[((k * P + p) * Q + b) * I + i] = h;
    }
  }
};

// Mode-1 epilogue: batch z = k * P + p, row a, column b -> T2[p][k][a][b].
struct Mode1TcEpi {
  static constexpr bool kRowMajor = true;
  static constexpr bool kSeg = false;
  static constexpr bool kBf16Rows = false;
  float *T2;
  int64_t t;
  int P, Q;
  const float *Bfac = nullptr;   // no fused reduction
  float *part = nullptr;
  int RT = 0, seg = 0;
  __device__ __forceinline__ bool stores() const { return true; }
  __device__ __forceinline__ void store(int z, int, int a, int b, float v) const {
    const int k = z / P, p = z - k * P;
    T2[(((int64_t)p * t + k) * Q + a) * Q + b] = v;
  }
};

__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// Persistent GEMM: one CTA per SM walks the tiles (N fastest, then M, then the
// batch index); tensor memory holds two accumulators so the epilogue of one
// tile overlaps the main loop of the next.
//   warp 0 lane 0 : TMA producer        full[s]  <- TMA bytes,  waits empty[s]
//   warp 1 lane 0 : MMA issuer          empty[s] <- commit,     acc_full[b] <- commit
//   warps 2..5    : epilogue (lane quadrant = warp % 4), acc_empty[b] <- 4 arrivals
template <int KIND, class Epi, int KATOMS>
__global__ void __launch_bounds__(192, 1)
    tc_gemm_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                   const TcShape sh, const Epi epi, int batch, int *status) {
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  uint8_t *smem = reinterpret_cast<uint8_t *>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
  const int stages = sh.stages;
  // a stage holds `katoms` 128-byte K atoms of each operand, atom after atom
  constexpr int katoms = KATOMS;
  const uint32_t a_atom = kBM * kRowBytes, b_atom = sh.BN * kRowBytes;
  const uint32_t a_bytes = a_atom * katoms;
  const uint32_t b_bytes = b_atom * katoms;
  uint8_t *sA = smem;
  uint8_t *sB = smem + stages * a_bytes;
  uint64_t *full = reinterpret_cast<uint64_t *>(sB + stages * b_bytes);
  uint64_t *empty = full + stages;
  uint64_t *acc_full = empty + stages;     // [2]
  uint64_t *acc_empty = acc_full + 2;      // [2]
  uint64_t *drain = acc_empty + 2;
  uint32_t *tmem_holder = reinterpret_cast<uint32_t *>(drain + 1);
  volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_holder + 1);
  // row-major epilogues stage each warp's 32 x 32 block here to store whole rows
  float *stage_all = reinterpret_cast<float *>(
      (reinterpret_cast<uintptr_t>(tmem_holder + 2) + 15) & ~static_cast<uintptr_t>(15));

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  constexpr int kElemsPerRow = KIND == 0 ? 64 : 128;   // 128 bytes of K
  const int kStageElems = kElemsPerRow * katoms;
  const int nk_all = (sh.K + kStageElems - 1) / kStageElems;   // stages of K
  const int tiles_n = sh.ksplit > 1 ? sh.ksplit : (sh.N + sh.BN - 1) / sh.BN;
  const int tiles_m = (sh.M + kBM - 1) / kBM;
  const int total = tiles_n * tiles_m * batch;         // work items (tiles)
  const int per_split = sh.ksplit > 1 ? (nk_all + sh.ksplit - 1) / sh.ksplit : nk_all;
  const int item0 = (int)blockIdx.x;
  const int nitems = (int)gridDim.x;

  if (threadIdx.x == 0) {
    for (int s = 0; s < stages; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&acc_full[b], 1);
      mbar_init(&acc_empty[b], 4);
    }
    mbar_init(drain, 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) tmem_alloc(tmem_holder, sh.tmem_cols);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_holder;
  // everything above is setup: the operands and outputs of the update are
  // touched only once the previous kernel of the chain has completed
  pdl_trigger();
  pdl_wait();

  // work item -> (z, m0, n0 or split, first K block, K blocks)
  auto decode = [&](int tile, int &z, int &m0, int &n0, int &split, int &kb0, int &nk) {
    const int nt = tile % tiles_n;
    const int rest = tile / tiles_n;
    m0 = (rest % tiles_m) * kBM;
    z = rest / tiles_m;
    if (sh.ksplit > 1) {
      split = nt; n0 = 0; kb0 = nt * per_split; nk = min(per_split, nk_all - kb0);
    } else {
      split = 0; n0 = nt * sh.BN; kb0 = 0; nk = nk_all;
    }
  };

  if (warp == 0 && lane == 0) {
    // TMA producer
    const uint64_t a_policy = sh.a_stream ? policy_evict_first() : 0;
    uint32_t it = 0;
    bool aborted = false;
    for (int tile = item0; tile < total && !aborted; tile += nitems) {
      int z, m0, n0, split, kb0, nk;
      decode(tile, z, m0, n0, split, kb0, nk);
      const int a_row = (z / sh.zdiv) * sh.a_hi + (z % sh.zdiv) * sh.a_lo + m0;
      const int b_row = (z / sh.zdiv) * sh.b_hi + (z % sh.zdiv) * sh.b_lo + n0;
      for (int kb = 0; kb < nk; ++kb, ++it) {
        const int s = it % stages;
        const uint32_t ph = (it / stages) & 1u;
        if (!mbar_wait(&empty[s], ph ^ 1u, abort_flag, sh.wait_budget)) {
          *abort_flag = 1;
          atomicOr(status, kDevTimeout);
          aborted = true;
          break;
        }
        mbar_expect_tx(&full[s], a_bytes + b_bytes);
#pragma unroll
        for (int at = 0; at < katoms; ++at) {
          // K atoms past the end are filled with zeros by the TMA unit
          const int kx = ((kb0 + kb) * katoms + at) * kElemsPerRow;
          if (sh.a_stream)
            tma_load_2d_policy(sA + s * a_bytes + at * a_atom, &tmA, &full[s], kx, a_row,
                               a_policy);
          else
            tma_load_2d(sA + s * a_bytes + at * a_atom, &tmA, &full[s], kx, a_row);
          tma_load_2d(sB + s * b_bytes + at * b_atom, &tmB, &full[s], kx, b_row);
        }
      }
    }
    if (aborted) {
      // wait (bounded) for the copies still in flight before the CTA can exit
      const uint32_t first = it > (uint32_t)stages ? it - stages : 0u;
      for (uint32_t j = first; j < it; ++j) {
        const long long t0 = clock64();
        while (!mbar_try_wait(&full[j % stages], (j / stages) & 1u) &&
               clock64() - t0 < kWaitBudget) {
        }
      }
    }
  } else if (warp == 1 && lane == 0) {
    // MMA issuer
    const uint32_t idesc = make_idesc(KIND, sh.BN);
    uint32_t it = 0, local = 0;
    bool aborted = false;
    for (int tile = item0; tile < total && !aborted; tile += nitems, ++local) {
      int z, m0, n0, split, kb0, nk;
      decode(tile, z, m0, n0, split, kb0, nk);
      const uint32_t buf = local & 1u, use = local >> 1;
      if (!mbar_wait(&acc_empty[buf], (use & 1u) ^ 1u, abort_flag, sh.wait_budget)) {
        *abort_flag = 1;
        atomicOr(status, kDevTimeout);
        break;
      }
      tc_fence_after();
      const uint32_t d = tmem + buf * static_cast<uint32_t>(sh.BN);
      for (int kb = 0; kb < nk; ++kb, ++it) {
        const int s = it % stages;
        const uint32_t ph = (it / stages) & 1u;
        if (!mbar_wait(&full[s], ph, abort_flag, sh.wait_budget)) {
          *abort_flag = 1;
          atomicOr(status, kDevTimeout);
          aborted = true;
          break;
        }
        tc_fence_after();
        // the stage's descriptors once; an MMA's operands lie at byte offsets
        // within the stage, which add to the 16-byte start-address field
        // (shared addresses stay below 2^18, so the field does not carry)
        const uint64_t da = make_desc_sw128(smem_u32(sA + s * a_bytes));
        const uint64_t db = make_desc_sw128(smem_u32(sB + s * b_bytes));
#pragma unroll
        for (int at = 0; at < katoms; ++at) {
#pragma unroll
          for (int kk = 0; kk < kRowBytes / 32; ++kk) {
            mma_issue<KIND>(d, da + ((at * a_atom + kk * 32) >> 4),
                            db + ((at * b_atom + kk * 32) >> 4), idesc,
                            (kb > 0 || at > 0 || kk > 0) ? 1u : 0u);
          }
        }
        mma_commit(&empty[s]);
      }
      mma_commit(&acc_full[buf]);
    }
    // every MMA this thread issued has completed once the drain barrier flips
    mma_commit(drain);
    const long long t0 = clock64();
    while (!mbar_try_wait(drain, 0) && clock64() - t0 < kWaitBudget) {
    }
  } else if (warp >= 2) {
    // epilogue
    const int quad = warp & 3;
    uint32_t local = 0;
    for (int tile = item0; tile < total; tile += nitems, ++local) {
      int z, m0, n0, split, kb0, nk;
      decode(tile, z, m0, n0, split, kb0, nk);
      const uint32_t buf = local & 1u, use = local >> 1;
      const bool ok = mbar_wait(&acc_full[buf], use & 1u, abort_flag, sh.wait_budget);
      if (!__all_sync(0xffffffffu, ok && !*abort_flag)) {
        if (lane == 0) {
          *abort_flag = 1;
          atomicOr(status, kDevTimeout);
        }
        break;
      }
      tc_fence_after();
      const int m = m0 + quad * 32 + lane;
      for (int c0 = 0; c0 < sh.BN; c0 += 32) {
        uint32_t r[32];
        tmem_ld32(tmem + (static_cast<uint32_t>(quad * 32) << 16) + buf * sh.BN + c0, r);
        if constexpr (Epi::kRowMajor) {
          // transpose through shared memory: instruction `i` stores row i of the
          // warp's block, lanes covering 32 consecutive columns
          float *stg = stage_all + (warp - 2) * 32 * 33;
#pragma unroll
          for (int j = 0; j < 32; ++j) stg[lane * 33 + j] = __uint_as_float(r[j]);
          __syncwarp();
          const int n = n0 + c0 + lane;
          bool stored = false;
          if constexpr (Epi::kBf16Rows) {
            if (epi.Dh && sh.N % 8 == 0) {
              // bf16 rows: lane l packs columns 8 (l % 4) .. + 7 of rows l / 4 + 8 q
              const int c8 = 8 * (lane & 3);
#pragma unroll
              for (int q = 0; q < 4; ++q) {
                const int i = (lane >> 2) + 8 * q;
                const int mi = m0 + quad * 32 + i;
                const int nb = n0 + c0 + c8;
                if (mi < sh.M && nb < sh.N) {
                  const float *src = stg + i * 33 + c8;
                  __align__(16) __nv_bfloat162 h[4];
#pragma unroll
                  for (int e = 0; e < 4; ++e) h[e] = __floats2bfloat162_rn(src[2 * e], src[2 * e + 1]);
                  epi.store_bf16x8(z, split, mi, nb, *reinterpret_cast<const uint4 *>(h));
                }
              }
              stored = true;
            }
          }
          if (!stored && epi.stores()) {   // else only the fused reduction below
            for (int i = 0; i < 32; ++i) {
              const int mi = m0 + quad * 32 + i;
              if (mi < sh.M && n < sh.N) epi.store(z, split, mi, n, stg[i * 33 + lane]);
            }
          }
          if (epi.part != nullptr) {
            const int mb = m0 + quad * 32;   // 32 rows of one a when 32 divides Q
            if (mb < sh.M && n < sh.N) {
              const int b0 = mb % epi.Q;
              if (!epi.seg) {
                const float *bf = epi.Bfac + ((int64_t)z * epi.Q + b0) * epi.RT + n;
                float acc = 0.f;
                for (int i = 0; i < 32; ++i) acc = fmaf(stg[i * 33 + lane], bf[i * epi.RT], acc);
                epi.part[((int64_t)z * (sh.M / 32) + mb / 32) * epi.RT + n] = acc;
              } else {
                // rows [0, Q - b0) belong to the block's first m / Q, the rest
                // (Q >= 32: at most one more) to the next
                const float *bf = epi.Bfac + (int64_t)z * epi.Q * epi.RT + n;
                const int nv = sh.M - mb < 32 ? sh.M - mb : 32;
                const int cut = epi.Q - b0;   // the same for the whole warp
                float a0 = 0.f, a1 = 0.f;
                if (cut >= 32 && nv == 32) {   // most blocks: one segment
                  const float *w = bf + b0 * epi.RT;
#pragma unroll
                  for (int i = 0; i < 32; ++i) a0 = fmaf(stg[i * 33 + lane], w[i * epi.RT], a0);
                } else {
                  const int n0 = cut < nv ? cut : nv;
                  for (int i = 0; i < n0; ++i)
                    a0 = fmaf(stg[i * 33 + lane], bf[(b0 + i) * epi.RT], a0);
                  for (int i = n0; i < nv; ++i)
                    a1 = fmaf(stg[i * 33 + lane], bf[(b0 + i - epi.Q) * epi.RT], a1);
                }
                const int64_t nblk = (sh.M + 31) / 32;
                float *pp = epi.part + (((int64_t)z * nblk + mb / 32) * 2) * epi.RT + n;
                pp[0] = a0;
                pp[epi.RT] = a1;
              }
            }
          }
          __syncwarp();
        } else {
          bool done = false;
          if constexpr (Epi::kSeg) {
            if (epi.seg) {
              // bf16 block [32 columns][32 rows] per warp, then 16-byte segments
              __nv_bfloat16 *stg =
                  reinterpret_cast<__nv_bfloat16 *>(stage_all) + (warp - 2) * 32 * 32;
              const float sc = m < sh.M ? epi.row_scale(m) : 1.f;
#pragma unroll
              for (int j = 0; j < 32; ++j)
                stg[j * 32 + lane] = __float2bfloat16_rn(__uint_as_float(r[j]) * sc);
              __syncwarp();
              epi.store_chunk(stg, m0 + quad * 32, n0 + c0, sh.M, sh.N, lane);
              __syncwarp();
              done = true;
            }
          }
          if (!done && m < sh.M) {
#pragma unroll
            for (int j = 0; j < 32; ++j) {
              const int n = n0 + c0 + j;
              if (n < sh.N) epi(z, split, m, n, __uint_as_float(r[j]));
            }
          }
        }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&acc_empty[buf]);
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) tmem_dealloc(tmem, sh.tmem_cols);
}

// The driver's tensor-map encoder, looked up once per process (the static's
// initialisation is thread-safe).
PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static const PFN_cuTensorMapEncodeTiled_v12000 fn = [] {
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      return reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    return static_cast<PFN_cuTensorMapEncodeTiled_v12000>(nullptr);
  }();
  return fn;
}

// 2-D map over a row-major [rows][inner] operand, 128-byte boxes along K.
bool make_map(CUtensorMap *m, const void *base, bool fp8, uint64_t inner, uint64_t rows,
              uint32_t box_rows) {
  PFN_cuTensorMapEncodeTiled_v12000 fn = encode_fn();
  if (!fn) return false;
  const uint64_t esz = fp8 ? 1 : 2;
  if ((reinterpret_cast<uintptr_t>(base) & 15) || ((inner * esz) & 15)) return false;
  cuuint64_t dims[2] = {inner, rows};
  cuuint64_t strides[1] = {inner * esz};
  cuuint32_t box[2] = {static_cast<cuuint32_t>(kRowBytes / esz), box_rows};
  cuuint32_t estr[2] = {1, 1};
  return fn(m, fp8 ? CU_TENSOR_MAP_DATA_TYPE_UINT8 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2,
            const_cast<void *>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
            CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

int pow2_at_least(int n) {
  int p = 32;
  while (p < n) p <<= 1;
  return p;
}

int sm_count() {
  static const int n = [] {
    int dev = 0, c = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&c, cudaDevAttrMultiProcessorCount, dev);
    return c > 0 ? c : 1;
  }();
  return n;
}

// Clock budget of the pipeline waits: kWaitBudget (about 2 s), or the cycle
// count in OCTEN_WAIT_BUDGET_CYCLES (between 1 and kWaitBudget), a debug setting
// read at every launch with which a test makes the waits run out before their
// data lands, so that the timeout path (abort, drain, status word) runs
// without anything on the device hanging.
long long wait_budget_cycles() {
  const char *v = getenv("OCTEN_WAIT_BUDGET_CYCLES");
  if (!v || !*v) return kWaitBudget;
  char *end = nullptr;
  const long long n = strtoll(v, &end, 10);
  if (end == v || n < 1) return kWaitBudget;
  return n < kWaitBudget ? n : kWaitBudget;
}

template <int KIND, class Epi>
bool launch_tc(const CUtensorMap &ma, const CUtensorMap &mb, TcShape sh, int batch,
               const Epi &epi, int *status, cudaStream_t st, int smem_reserve = 0,
               int max_ctas = 0, int max_stages = 0, bool pdl = false) {
  sh.wait_budget = wait_budget_cycles();
  sh.tmem_cols = pow2_at_least(2 * sh.BN);       // two accumulators
  if (sh.tmem_cols > 512) return false;
  if (sh.katoms != 2 && sh.katoms != 4) sh.katoms = 1;   // kernels for 1, 2 and 4 atoms
  const size_t per_stage = static_cast<size_t>(kBM + sh.BN) * kRowBytes * sh.katoms;
  const size_t stage_bytes = Epi::kRowMajor ? 4 * 32 * 33 * sizeof(float) + 16
                             : Epi::kSeg   ? 4 * 32 * 32 * sizeof(__nv_bfloat16) + 16
                                           : 0;
  const int64_t room = 220 * 1024 - (int64_t)stage_bytes - smem_reserve;
  sh.stages = room > 0 ? static_cast<int>(room / (int64_t)per_stage) : 0;
  if (sh.stages > 8) sh.stages = 8;
  if (max_stages >= 2 && sh.stages > max_stages) sh.stages = max_stages;
  if (sh.stages < 2) return false;
  const size_t smem = 1024 + per_stage * sh.stages + (2 * sh.stages + 5) * 8 + 16 + stage_bytes;
  auto kern = sh.katoms == 4   ? tc_gemm_kernel<KIND, Epi, 4>
              : sh.katoms == 2 ? tc_gemm_kernel<KIND, Epi, 2>
                               : tc_gemm_kernel<KIND, Epi, 1>;
  if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           static_cast<int>(smem)) != cudaSuccess)
    return false;
  const int tiles_n = sh.ksplit > 1 ? sh.ksplit : (sh.N + sh.BN - 1) / sh.BN;
  const int64_t items = (int64_t)tiles_n * ((sh.M + kBM - 1) / kBM) * batch;
  if (items <= 0 || items > (int64_t)1 << 30) return false;
  cudaLaunchConfig_t cfg = {};
  cfg.blockDim = dim3(192);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  if (pdl) {
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
  }
  const int slots = max_ctas > 0 && max_ctas < sm_count() ? max_ctas : sm_count();
  const int grid_items = (int)(items < slots ? items : slots);
  cfg.gridDim = dim3(grid_items);
  if (cudaLaunchKernelEx(&cfg, kern, ma, mb, sh, epi, batch, status) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  count_launch();
  count_tc_launch();
  return true;
}

// ---------------------------------------------------------------------------
// Autotuner.  For every GEMM shape the first call (outside stream capture)
// times the candidate launch configurations with CUDA events on the caller's
// stream and keeps the fastest for the rest of the process.  Only choices that
// leave every output bit unchanged are tuned: the K atoms per pipeline stage
// (the MMAs run in the same order either way) and, for mode 2, the N tile (each
// output's K sum is the same sequence whatever tile it falls in).  The split-K
// count, which changes the summation, is fixed by the caller.  The timing
// launches write the same outputs as the final one and are not counted as
// launches.  OCTEN_AUTOTUNE=0 keeps the defaults.
struct TuneChoice {
  int katoms, BN;
  int stages = 0;   // pipeline stages at most (0: as many as fit)
};

std::mutex g_tune_mu;
std::map<std::array<int64_t, 8>, TuneChoice> g_tune;

bool autotune_enabled() {
  const char *v = getenv("OCTEN_AUTOTUNE");
  return !(v && strcmp(v, "0") == 0);
}

bool stream_capturing(cudaStream_t st) {
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(st, &cs) != cudaSuccess) {
    cudaGetLastError();
    return true;   // be safe: no synchronising work
  }
  return cs != cudaStreamCaptureStatusNone;
}

// launch(choice) issues one GEMM with that choice and returns false if refused.
template <class Launch>
TuneChoice tuned(const std::array<int64_t, 8> &key, const TuneChoice *cand, int ncand,
                 cudaStream_t st, Launch launch) {
  {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    auto it = g_tune.find(key);
    if (it != g_tune.end()) return it->second;
  }
  if (ncand < 2 || !autotune_enabled() || stream_capturing(st)) return cand[0];
  const uint64_t l0 = octen_launch_count(), t0 = octen_tc_launch_count();
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  // time on an otherwise idle device (work on other streams, such as a factor
  // kernel beside the GEMM, would slow whichever candidate it overlaps), in
  // two rounds over the candidates, keeping each candidate's best
  cudaDeviceSynchronize();
  constexpr int kMaxCand = 6;
  float cand_ms[kMaxCand];
  bool runs[kMaxCand];
  for (int c = 0; c < ncand && c < kMaxCand; ++c) {
    cand_ms[c] = 3.4e38f;
    runs[c] = launch(cand[c]);   // warm-up (and the check that it runs)
    if (!runs[c]) cudaGetLastError();
  }
  for (int round = 0; round < 2; ++round) {
    for (int c = 0; c < ncand && c < kMaxCand; ++c) {
      if (!runs[c]) continue;
      cudaEventRecord(e0, st);
      const bool ok = launch(cand[c]) && launch(cand[c]);
      cudaEventRecord(e1, st);
      float ms = 0.f;
      if (!ok || cudaEventSynchronize(e1) != cudaSuccess ||
          cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
        cudaGetLastError();
        runs[c] = false;
        continue;
      }
      if (ms < cand_ms[c]) cand_ms[c] = ms;
    }
  }
  TuneChoice best = cand[0];
  float best_ms = 3.4e38f;
  for (int c = 0; c < ncand && c < kMaxCand; ++c) {
    if (runs[c] && cand_ms[c] < best_ms) {
      best_ms = cand_ms[c];
      best = cand[c];
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (getenv("OCTEN_AUTOTUNE_LOG")) {   // diagnostics: the timings behind each choice
    fprintf(stderr, "octen autotune key");
    for (int64_t v : key) fprintf(stderr, " %lld", (long long)v);
    for (int c = 0; c < ncand && c < kMaxCand; ++c)
      fprintf(stderr, " | katoms %d BN %d stages %d: %.4f ms%s", cand[c].katoms, cand[c].BN,
              cand[c].stages, runs[c] ? cand_ms[c] / 2 : -1.f,
              cand[c].katoms == best.katoms && cand[c].BN == best.BN &&
                      cand[c].stages == best.stages
                  ? " *"
                  : "");
    fprintf(stderr, "\n");
  }
  adjust_launch_counts(-(int64_t)(octen_launch_count() - l0),
                       -(int64_t)(octen_tc_launch_count() - t0));
  std::lock_guard<std::mutex> lock(g_tune_mu);
  g_tune[key] = best;
  return best;
}

}  // namespace

bool tc_supported() {
  int dev = 0, major = 0, minor = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return false;
  cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev);
  cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev);
  return major == 10 && minor == 3 && encode_fn() != nullptr;
}

bool mode2_tc(const Mode2Args &a, int *status, cudaStream_t st) {
  if (a.tt != Elem::BF16 || !(a.tx == Elem::BF16 || a.tx == Elem::E4M3) || a.tv != a.tx)
    return false;
  const bool fp8 = a.tx == Elem::E4M3;
  const int64_t M = a.t * a.I;
  if (M > (1 << 30) || a.J > (1 << 30)) return false;
  CUtensorMap ma, mb256, mb128;
  if (!make_map(&ma, a.X, fp8, a.J, M, kBM) || !make_map(&mb256, a.Vt, fp8, a.J, a.Qd, 256) ||
      !make_map(&mb128, a.Vt, fp8, a.J, a.Qd, 128))
    return false;
  Mode2TcEpi epi{static_cast<__nv_bfloat16 *>(a.T), a.slice_scale, a.I, a.P, a.Q, a.S,
                 a.I % 8 == 0};
  auto launch = [&](const TuneChoice &c) {
    TcShape sh{};
    sh.ksplit = 1;
    sh.M = static_cast<int>(M); sh.N = a.Qd; sh.K = static_cast<int>(a.J); sh.BN = c.BN;
    sh.zdiv = 1; sh.a_hi = 0; sh.a_lo = 0; sh.b_hi = 0; sh.b_lo = 0;
    sh.a_stream = 1;   // the slices are read once
    sh.katoms = c.katoms;
    const CUtensorMap &mb = c.BN == 256 ? mb256 : mb128;
    return fp8 ? launch_tc<1>(ma, mb, sh, 1, epi, status, st)
               : launch_tc<0>(ma, mb, sh, 1, epi, status, st);
  };
  static const TuneChoice cand[] = {{1, 256}, {2, 128}, {1, 128}};
  const std::array<int64_t, 8> key{2, fp8 ? 1 : 0, M, a.Qd, a.J, a.I, a.P, a.Q};
  return launch(tuned(key, cand, 3, st, launch));
}

bool mode1_tc(const Mode1Args &a, int *status, cudaStream_t st) {
  if (a.te != Elem::BF16) return false;
  CUtensorMap ma, mb, mb128;
  const int BN = (a.Q + 31) / 32 * 32;
  if (BN > 256) return false;
  const int64_t rowsA = static_cast<int64_t>(a.P) * a.Q;
  const int64_t rowsB = a.t * a.P * a.Q;
  if (rowsB > (1 << 30)) return false;
  if (!make_map(&ma, a.Ut, false, a.I, rowsA, kBM) || !make_map(&mb, a.T, false, a.I, rowsB, BN))
    return false;
  const bool two_n = BN > 128 && make_map(&mb128, a.T, false, a.I, rowsB, 128);
  Mode1TcEpi epi{a.T2, a.t, a.P, a.Q};
  auto launch = [&](const TuneChoice &c) {
    TcShape sh{};
    sh.ksplit = 1;
    sh.M = a.Q; sh.N = a.Q; sh.K = static_cast<int>(a.I); sh.BN = c.BN;
    sh.zdiv = a.P;                   // z = k * P + p
    sh.a_hi = 0; sh.a_lo = a.Q;      // A rows: p * Q
    sh.b_hi = a.P * a.Q; sh.b_lo = a.Q;   // B rows: (k * P + p) * Q
    sh.katoms = c.katoms;
    return launch_tc<0>(ma, c.BN == 128 && two_n ? mb128 : mb, sh, static_cast<int>(a.t * a.P),
                        epi, status, st, 0, 0, c.stages);
  };
  // the N tile (one or two tiles of the Q columns) and the K atoms per stage
  // leave every output's K order unchanged
  const TuneChoice cand[] = {{1, BN}, {2, BN}, {1, 128}, {2, 128}};
  const std::array<int64_t, 8> key{3, a.t, a.I, a.P, a.Q, 0, 0, 0};
  return launch(tuned(key, cand, two_n ? 4 : 2, st, launch));
}

bool tc_gemm_store(const TcStoreArgs &g, int *status, cudaStream_t st) {
  if (g.BN % 32 || g.BN > 256 || g.BN < 32) return false;
  CUtensorMap ma, mb;
  if (!make_map(&ma, g.A, false, g.a_inner, g.a_rows, kBM) ||
      !make_map(&mb, g.B, false, g.b_inner, g.b_rows, g.BN))
    return false;
  // the split count is fixed by the caller's K atoms (it sets the summation)
  const int katoms0 = g.katoms == 2 || g.katoms == 4 ? g.katoms : 1;
  const int ks = tc_gemm_splits(g.K, g.ksplit, katoms0);
  const bool seg = g.m1_part && g.m1_seg;
  if (g.m1_part && (g.BN != 32 || ks > 1 || (seg ? g.Q < 32 : g.Q % 32 != 0))) return false;
  if (ks > 1 && (g.N > g.BN)) return false;
  TcStoreEpi epi{g.D, ks > 1 ? g.s_split : 0, g.s_z, g.s_m, g.m1_B, g.m1_part, g.Q, g.RT, g.Dh,
                 seg ? 1 : 0, g.d_keep ? 1 : 0};
  auto launch = [&](const TuneChoice &c) {
    TcShape sh{};
    sh.M = g.M; sh.N = g.N; sh.K = g.K; sh.BN = g.BN;
    sh.zdiv = 1; sh.a_hi = g.a_rows_per_z; sh.a_lo = 0; sh.b_hi = g.b_rows_per_z; sh.b_lo = 0;
    sh.a_stream = g.a_stream ? 1 : 0;
    sh.katoms = c.katoms;
    sh.ksplit = ks;
    return launch_tc<0>(ma, mb, sh, g.batch, epi, status, st, g.smem_reserve, g.max_ctas,
                        c.stages, g.pdl);
  };
  // candidates: the caller's K atoms per stage with as many pipeline stages
  // as fit or three (fewer bytes in flight per SM, more room beside the
  // GEMM), and the other atom counts (1, 2, 4: with four, a tile's rows of
  // K = 256 arrive as whole 512-byte rows); with split-K another atom count
  // only if it cuts K at the same places (the splits set the summation)
  auto split_elems = [&](int k) {
    const int nk = (g.K + 64 * k - 1) / (64 * k);
    return ((nk + ks - 1) / ks) * 64 * k;
  };
  TuneChoice cand[5] = {{katoms0, g.BN, 0}, {katoms0, g.BN, 3}};
  int ncand = 2;
  for (int k : {1, 2, 4})
    if (k != katoms0 && (ks == 1 || split_elems(k) == split_elems(katoms0)))
      cand[ncand++] = TuneChoice{k, g.BN, 0};
  const std::array<int64_t, 8> key{1 + 16 * (int64_t)g.max_ctas, g.M, g.N, g.K, g.batch, ks,
                                   g.Dh != nullptr, g.m1_part != nullptr};
  return launch(tuned(key, cand, ncand, st, launch));
}

int tc_gemm_splits(int K, int ksplit, int katoms) {
  const int nk = (K + 64 * katoms - 1) / (64 * katoms);   // pipeline stages of K
  int ks = ksplit < 1 ? 1 : (ksplit > nk ? nk : ksplit);
  const int per = (nk + ks - 1) / ks;
  return (nk + per - 1) / per;   // every split gets at least one stage
}

}  // namespace octen
