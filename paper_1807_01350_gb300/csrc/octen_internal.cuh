// Internal declarations shared by the translation units of the CUDA library.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp8.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <cstdio>
#include <string>

#include "../../include/octen.h"

namespace octen {

// Bit flags a kernel may raise in the context's device status word.
enum DevFlag : int {
  kDevCholesky = 1,   // a Cholesky pivot stayed non-positive after loading
  kDevTimeout = 2,    // a bounded wait ran out
};

// Element types of the slice batch and of the contraction operands.
enum class Elem : int { F32 = 0, BF16 = 1, E4M3 = 2 };

inline size_t elem_size(Elem e) { return e == Elem::F32 ? 4 : (e == Elem::BF16 ? 2 : 1); }

// Programmatic dependent launch inside the replica CP-ALS chain: a kernel
// launched with cudaLaunchAttributeProgrammaticStreamSerialization may start
// while its predecessor on the stream is still running.  pdl_trigger lets the
// next kernel of the chain launch early (its CTAs then do their setup beside
// this one); pdl_wait blocks until the predecessor has completed and its
// writes are visible.  Every kernel of the chain calls both before it touches
// any data of the update, so the chain's order of reads and writes is the
// stream's.  Without the attribute both are no-ops.
__device__ __forceinline__ void pdl_trigger() {
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

// Asks for the largest shared-memory part of the SMs' on-chip memory when
// kernel f runs.  An SM holds one split between L1 and shared memory at a
// time and the tensor-core GEMMs take the largest shared part, so a kernel
// meant to run beside them (or beside another such kernel) must prefer the
// same split; with another preference it waits for their CTAs to leave the
// SMs.  Call once per kernel (the setting persists).
template <class Kernel>
inline void prefer_max_shared(Kernel *f) {
  if (cudaFuncSetAttribute(f, cudaFuncAttributePreferredSharedMemoryCarveout,
                           cudaSharedmemCarveoutMaxShared) != cudaSuccess)
    cudaGetLastError();
}

// Brings the 128-byte line holding p into the L2 (a hint: nothing waits on it).
__device__ __forceinline__ void prefetch_l2(const void *p) {
  asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
}

// Counts every kernel launch issued through the launch helpers below.
void count_launch();
// Adds to the launch counters (negative: launches that did not do the work).
void adjust_launch_counts(int64_t n, int64_t ntc);

// Stages timed with CUDA events when a context has timing enabled.
enum Stage : int {
  kStQuant = 0, kStMode2, kStMode1, kStMode3, kStWarm, kStAlsGemm, kStAlsAux, kStAlsSolve,
  kStAlign, kStLift, kStCsolve, kStAlsFused, kNumStages
};

// Optional hook called around the kernels of a multi-kernel stage:
// fn(arg, stage, 1) before a launch, fn(arg, stage, 0) after it.
struct Marker {
  void (*fn)(void *, int, int) = nullptr;
  void *arg = nullptr;
  void operator()(int stage, int begin) const {
    if (fn) fn(arg, stage, begin);
  }
};

// ---------------------------------------------------------------------------
// Generic strided batched fp32-accumulate GEMM (SIMT FFMA):
//   D[z](m, n) = alpha * sum_k A[z](m, k) * B[z](n, k) + beta * D[z](m, n)
// with A(m, k) = A[z * sAz + m * sAm + k * sAk], and likewise for B and D.
// ---------------------------------------------------------------------------
struct GemmArgs {
  const void *A; Elem ta; int64_t sAz, sAm, sAk;
  const void *B; Elem tb; int64_t sBz, sBn, sBk;
  float *D; int64_t sDz, sDm, sDn;
  int M, N, K, batch;
  float alpha, beta;
  // optional scratch: lets a GEMM with few output tiles and a long K split K
  // over CTAs (partials reduced by a second kernel)
  float *split_scratch = nullptr;
  size_t split_scratch_floats = 0;
  // N <= 32 with several batch items: the skinny kernel per item (grid z)
  bool skinny_batch = false;
};
void gemm_strided(const GemmArgs &g, cudaStream_t st);

// Mode-2 contraction of the compression: T_rep[k][p][b][i] =
//   sum_j X[k][i][j] * V_all[j][col_p(b)] for every replica p,
// with Vt the transposed projection (Qd x J) in the operand type and T_rep in
// `tt` (fp32 or bf16).  X element type `tx`, optional per-slice scales.
struct Mode2Args {
  const void *X; Elem tx;
  const void *Vt; Elem tv;
  const float *slice_scale;  // nullable: per-slice multiplier (fp8 path)
  void *T; Elem tt;
  int64_t t, I, J;
  int P, Q, S, Qd;
};
void mode2_simt(const Mode2Args &a, cudaStream_t st);

// Mode-1 contraction: T2[p][k][a][b] = sum_i Ut_rep[p][a][i] * T_rep[k][p][b][i].
struct Mode1Args {
  const void *Ut; const void *T; Elem te;
  float *T2;
  int64_t t, I;
  int P, Q;
};
void mode1_simt(const Mode1Args &a, cudaStream_t st);

// tcgen05 versions of the two large contractions (bf16 / e4m3 operands).  They
// return false without launching when the device is not sm_103 or an operand
// violates the TMA alignment rules (row pitch a multiple of 16 bytes).
bool tc_supported();
bool mode2_tc(const Mode2Args &a, int *status, cudaStream_t st);
bool mode1_tc(const Mode1Args &a, int *status, cudaStream_t st);
void count_tc_launch();
// a wanted tensor-core launch that was refused (the SIMT kernels ran instead)
void count_tc_fallback(const char *what);

// Generic bf16 tcgen05 GEMM with a plain fp32 store, used by the replica ALS:
//   D[split][z](m, n) = sum_{k in split} A[z * a_rows_per_z + m][k] * B[z * b_rows_per_z + n][k]
// A and B are row-major bf16 [rows][inner] (K contiguous).  Stored at
// D + split * s_split + z * s_z + m * s_m + n for m < M, n < N.  With ksplit > 1
// the K blocks are divided among that many CTAs per tile (N <= BN then).
struct TcStoreArgs {
  const void *A; int64_t a_inner, a_rows; int a_rows_per_z;
  const void *B; int64_t b_inner, b_rows; int b_rows_per_z;
  int M, N, K, BN, batch, ksplit;
  float *D; int64_t s_split, s_z, s_m;
  __nv_bfloat16 *Dh = nullptr;   // if set: the output rounded to bf16 here instead of D
  // optional fused reduction for rows m = a * Q + b (needs BN == 32, Q % 32 == 0):
  // m1_part[z][m / 32][n] = sum over the 32 rows of D(m, n) * m1_B[z][b][n]
  // (with D and Dh both null only this reduction is written)
  const float *m1_B = nullptr;
  float *m1_part = nullptr;
  int Q = 0, RT = 0;
  // with 32 not dividing Q (Q >= 32) a warp's 32 rows may span two values of
  // m / Q: m1_seg writes both segments, m1_part[z][m / 32][2][n] (segment 0 the
  // rows of the block's first m / Q)
  bool m1_seg = false;
  // the bf16 output Dh is read again soon: stored with an L2 evict-last policy
  bool d_keep = false;
  // shared memory (bytes) to leave free on every SM for a kernel that runs
  // beside this GEMM (fewer pipeline stages)
  int smem_reserve = 0;
  // A is read once: its TMA loads carry an L2 evict-first policy so that it
  // does not push the reused operands and the fresh outputs out of the L2
  bool a_stream = false;
  // 128-byte K atoms per pipeline stage: 2 halves the barrier round trips and
  // commits per byte for the narrow (N = 32) GEMMs
  int katoms = 1;
  // at most this many CTAs (0: one per SM), so that another GEMM can run on
  // the other SMs at the same time
  int max_ctas = 0;
  // launched as a programmatic dependent of the previous kernel on the stream
  bool pdl = false;
};
bool tc_gemm_store(const TcStoreArgs &g, int *status, cudaStream_t st);
// the split count tc_gemm_store will use
int tc_gemm_splits(int K, int ksplit, int katoms = 1);
constexpr int kAlsKAtoms = 2;   // K atoms per stage of the replica-ALS GEMMs

// Mode-3 contraction and summary update: Y[p][a][b][c] +=
//   sum_k T2[p][k][a][b] * W_all[k][col_p(c)].
// With Xa and Xc given it may also write the bf16 layouts of the updated Y
// that the tensor-core CP-ALS reads (returns true if it did).
bool mode3_accumulate(const float *T2, const float *W, float *Y, int64_t t, int P, int Q,
                      int S, int Qd, cudaStream_t st, __nv_bfloat16 *Xa = nullptr,
                      __nv_bfloat16 *Xc = nullptr);

// Layout / precision conversions of the projections.
void make_replica_transpose(const float *M_all, int64_t rows, int P, int Q, int S, int Qd,
                            void *out, Elem te, cudaStream_t st);   // [p][q][row]
void make_transpose(const float *M_all, int64_t rows, int Qd, void *out, Elem te,
                    cudaStream_t st);                                 // [c][row]
void round_copy(const float *in, float *out, int64_t n, Elem te, cudaStream_t st);
void convert_slices(const void *in, Elem tin, void *out, Elem tout, int64_t n,
                    cudaStream_t st);
void quantize_e4m3(const __nv_bfloat16 *X, int64_t t, int64_t IJ, __nv_fp8_e4m3 *X8,
                   float *scale, cudaStream_t st);

// ---------------------------------------------------------------------------
// Replica CP-ALS (all P replicas in each launch).  Factors are P x Q x RT
// (RT = R rounded up to 8, padded columns zero).
// ---------------------------------------------------------------------------
constexpr int kAlsNP = 32;   // padded rank rows of the tensor-core ALS operands
constexpr int kMaxAlsGroups = 4;   // replica groups of the tensor-core CP-ALS

struct AlsBuffers {
  float *Af, *Bf, *Cf;   // current factors, P x Q x RT
  float *GA, *GB, *GC;   // their Grams, P x RT x RT
  float *M;              // MTTKRP result, P x Q x RT
  float *H;              // P x Q x Q x RT: SIMT pass-1 product (fp32), or the Tc GEMM
                         // output (bf16, first half of the buffer)
  int *status;
  // tensor-core path (bf16 / e4m3 modes, Q % 8 == 0)
  bool use_tc = false;
  __nv_bfloat16 *Xa = nullptr, *Xc = nullptr;   // P x Q^3 each
  __nv_bfloat16 *KR = nullptr;                  // P x kAlsNP x Q^2 (M3 operand when 32 does not divide Q)
  __nv_bfloat16 *Ct = nullptr;                  // P x kAlsNP x Q (C^T, the Tc operand)
  __nv_bfloat16 *Bt = nullptr;                  // P x kAlsNP x Q (B^T, the M3 operand)
  float *Mparts = nullptr;                      // partials: fused P x Q x Q/32 x RT, or split-K
                                                // ksplit x P x Q x RT
  int ksplit = 1;
  bool layouts_ready = false;                   // Xa, Xc already hold bf16(X_p)
  // the factor of every update runs on `side` beside the update's MTTKRP:
  // fork after the previous update, join before the solve
  cudaStream_t side = nullptr;                  // non-blocking
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  float *L = nullptr;                           // P x als_factor_floats(RT)
  // GEMM grid cap of this group's passes (0: one CTA per SM)
  int max_ctas = 0;
  // the chain's GEMMs, solves and reductions launched as programmatic
  // dependents of their predecessors (OCTEN_PDL=0: ordinary launches)
  bool pdl = false;
  // Q not a multiple of 8 (Q >= 32): the tensor-core passes run on X_p
  // zero-padded to Qp = the next multiple of 8 (the TMA row pitch of the bf16
  // copies), with factors Af_pad, Bf_pad, Cf_pad (P x Qp x RT, the rows past Q
  // zero, and zero after every update since their MTTKRP rows are zero), and
  // Xa, Xc, Ct, Bt, Mparts, M and the bf16 Tc sized for Qp.  0: no padding.
  int Qp = 0;
  float *Af_pad = nullptr, *Bf_pad = nullptr, *Cf_pad = nullptr;
  // Replica groups (tensor-core path, 32 <= Q): the replicas are split into
  // `groups` contiguous groups whose sweeps run as independent chains, group g
  // on gst[g] (group 0 on the caller's stream) with its factor kernels on
  // gside[g], each GEMM on at most SMs / groups CTAs, so that one group's
  // solves and reductions overlap another group's GEMMs.  Per replica the
  // arithmetic is the same as with one group.
  int groups = 1;
  cudaStream_t gst[kMaxAlsGroups] = {}, gside[kMaxAlsGroups] = {};
  cudaEvent_t gev_fork[kMaxAlsGroups] = {}, gev_join[kMaxAlsGroups] = {};
  cudaEvent_t gsplit = nullptr, gdone[kMaxAlsGroups] = {};
  // staggered start: group g's first launch waits for group g - 1's first
  // GEMM (gfirst[g - 1]), so that the groups' GEMMs and solves alternate
  // instead of running in lockstep
  cudaEvent_t gfirst[kMaxAlsGroups] = {};
  cudaEvent_t wait_first = nullptr, ev_first = nullptr;   // per group, set by the runner
};
int als_factor_floats(int RT);
// Returns false if a tensor-core launch was refused (the caller then reruns
// the SIMT path).
bool als_run(const float *Y, int P, int Q, int R, int RT, int iters, AlsBuffers &b,
             cudaStream_t st, const Marker &mk = Marker());
bool als_tc_eligible(int Q);
// Single-launch CP-ALS for replicas small enough to keep X_p and its pass-1
// product in shared memory (one CTA per replica); false if it does not apply.
bool als_fused_fits(int Q, int RT);
bool als_run_fused(const float *Y, int P, int Q, int R, int RT, int iters, AlsBuffers &b,
                   cudaStream_t st);
int als_tc_splits(int P, int Q, int desired);

// Warm start: F_p = unit columns of rows(p) of PF (Qd x R) into P x Q x RT, and
// the Gram of each F_p into G (P x RT x RT).
void warm_start(const float *PF, int P, int Q, int S, int R, int RT, float *F, float *G,
                cudaStream_t st);

// Anchor match (FP64).  ref rows = PA/PB rows [0, S).
void align_replicas(const float *At, const float *Bt, const float *Ct, const float *PA,
                    const float *PB, int P, int Q, int S, int R, int RT, float *Ah,
                    float *Bh, float *Ch, int *perm, double *scales, double *scratch,
                    cudaStream_t st);
// Dense CP-ALS of the existing tensor X (K x I x J, [k][i][j], element type
// xt) from the initial guesses A0 (I x R), B0 (J x R): `iters` sweeps as in the
// replica CP-ALS, results into A_out (I x R), B_out (J x R), C_out (K x R).
// `work` holds dense_cp_work_floats(K, I, J, RT) floats.
struct DenseCpArgs {
  const void *X; Elem xt;
  int64_t K, I, J;
  int R, iters;
  const float *A0, *B0;
  float *A_out, *B_out, *C_out;
  float *work;
  float *splitk; size_t splitk_floats;
  int *status;
  cudaStream_t st;
};
size_t dense_cp_work_floats(int64_t K, int64_t I, int64_t J, int RT);
void dense_cp(const DenseCpArgs &a, int RT);

// Dense N-way CP-ALS of the existing tensor X ([k][i_1]...[i_{NN-1}], fp32 or bf16;
// dims[0] = K, dims[m] = I_m) from the guesses A0[m - 1] (I_m x R): `iters`
// sweeps as in the N-mode replica CP-ALS (time mode, then every non-temporal
// mode normalised to unit l2, a final time update), results into A_out[m - 1]
// (I_m x R) and C_out (K x R).  `work` holds dense_cp_n_work_floats floats.
struct DenseCpNArgs {
  const void *X;
  Elem xt;
  int NN;
  const int64_t *dims;
  int R, iters;
  const float *const *A0;
  float *const *A_out;
  float *C_out;
  float *work;
  int *status;
  cudaStream_t st;
};
size_t dense_cp_n_work_floats(int NN, const int64_t *dims, int RT);
void dense_cp_n(const DenseCpNArgs &a, int RT);

// doubles of scratch align_replicas needs
size_t align_scratch_doubles(int P, int RT);

// e (Qd x R) for the lift: shared rows summed (sum_mode=1) or averaged.
void lift_rhs(const float *Fh, const float *PF, int P, int Q, int S, int R, int RT, int Qd,
              int sum_mode, float *e, cudaStream_t st);

// C_new (t x R, t <= 64) from the stacked W_new,p^T system, and the G update.
// scratch: c_solve_scratch_floats(t, Qd, R) floats.
size_t c_solve_scratch_floats(int64_t t, int Qd, int R);
void solve_c_new(const float *W, const float *Ch, const float *G, int64_t t, int P, int Q,
                 int S, int Qd, int R, int RT, float *scratch, float *C_new, int *status,
                 cudaStream_t st);
void update_g(const float *W, const float *C_new, int64_t t, int P, int Q, int S, int Qd,
              int R, float *G, cudaStream_t st);

// Dense fp32 SPD factor / solve (init-time lift operators).
// Lift of Eq. 7 for one non-temporal mode (k_lift.cu).
struct LiftEnv {
  int Qd, P, Q, S, R, RT;
  cudaStream_t st;
  int *status;
  float *e;                      // Qd x R right-hand side scratch
  float *splitk;
  size_t splitk_floats;
};
// L (rows x Qd or Qd x rows) for the rounded projection Ur (rows x Qd); false on
// allocation or CUDA failure (the stream is synchronised).
bool lift_build(const LiftEnv &v, const float *Ur, int64_t rows, float *L, int &over);
// F (rows x R) += L e, e from the aligned replica blocks Fh and the projected
// previous factor PF.
void lift_apply(const LiftEnv &v, const float *Fh, const float *PF, const float *L, int over,
                int64_t rows, float *F);
void cholesky_f32(float *Gm, int n, int *status, cudaStream_t st);
void chol_solve_f32(const float *L, int n, float *Bm, int m, cudaStream_t st);
void scale_columns(const float *in, int64_t rows, int cols, int S, float w_shared,
                   float *out, cudaStream_t st);
void transpose_f32(const float *in, int64_t rows, int64_t cols, float *out, cudaStream_t st);

// ---------------------------------------------------------------------------
// N-mode extension (k_nmode.cu): N - 1 <= 5 non-temporal modes plus time.
// ---------------------------------------------------------------------------
constexpr int kMaxNModes = 6;

// Upper bound on the rows of the time factor C a context grows to (its
// capacity doubles from 64 rows; 2^40 rows of even one fp32 column are beyond
// any device memory, so the bound only guards the doubling against overflow
// on a corrupt checkpoint header).
constexpr int64_t kCRowsMax = int64_t(1) << 40;

// Compression of fp32 slices X[k][i_1]...[i_{nm}] into the summaries
// Y[p][q_1]...[q_{nm}][c] (accumulated).  Ut[n] = [p][q][i] replica
// transposes of the projections; Wt = [p][c][k] of the chunk's time rows;
// bufA, bufB hold ncompress_buf_floats(...) floats each.
struct NCompressInput {
  int nm, P, Q;
  const int64_t *dims;
  const float *const *Ut;
  float *bufA, *bufB;
};
// X is fp32 or bf16 (xt); with bf16 slices the first contraction runs on the
// tensor cores when Ut16 (the innermost mode's replica transpose in bf16) is
// given and the rows meet the TMA rules, else on the SIMT kernels.
void ncompress_chunk(const NCompressInput &c, const void *X, Elem xt, int64_t t,
                     const float *Wt, float *Y, cudaStream_t st, const void *Ut16 = nullptr,
                     int *status = nullptr);
int64_t ncompress_rows_max(int nm, const int64_t *dims, int Q, int64_t t);
int64_t ncompress_buf_floats(int nm, const int64_t *dims, int P, int Q, int64_t t);

// CP-ALS of the P N-way summaries (one CTA per replica).  F[0..NN-2] hold the
// warm starts (P x Q x RT, unit columns) and G0 their Grams; on return F[0..NN-1]
// hold the replica factors (F[NN-1] the time factor).
struct NAlsInput {
  const float *Y;
  float *F[kMaxNModes];
  const float *G0[kMaxNModes];
  int NN, P, Q, R, RT, iters;
  int *status;
};
bool nals_fits(int NN, int Q, int RT);
bool nals_run(const NAlsInput &in, cudaStream_t st);

// Anchor match of the N-mode replica factors (fp64).
struct NAlignInput {
  const float *F[kMaxNModes];    // nm non-temporal factors, then time
  const float *PF[kMaxNModes];
  float *Fh[kMaxNModes];
  int nm, P, Q, S, R, RT;
  int *perm;
  double *scales;
};
void n_align(const NAlignInput &in, cudaStream_t st);

// Fitness sums of nk slices (see k_nmode.cu): partial[k][block][2] doubles,
// n_fit_blocks(E) blocks per slice of E elements.
int n_fit_blocks(int64_t E);
void n_fit_sums(const void *X, Elem xt, int64_t nk, const float *const *A, const float *C,
                const int64_t *dims, int nm, int R, double *partial, cudaStream_t st);

// true for device (or managed) memory
bool is_device_pointer(const void *p);

// Shape and precision limits of a 3-mode configuration (the limits octen_create
// states); EINVAL with the reason in `why`.
octen_status validate_config(const octen_config *c, std::string &why);

// Fit: sums of ||X_k||^2 and ||X_k - A diag(C[k]) B^T||^2 over all slices,
// written to out[0], out[1] (fp64).  partial: ceil(J/256)*ceil(I/32)*K*2 doubles.
void fit_sums(const void *X, Elem tx, int64_t K, int64_t I, int64_t J, const float *A,
              const float *B, const float *C, int R, double *partial, double *out,
              cudaStream_t st);
int64_t fit_partial_count(int64_t K, int64_t I, int64_t J);
// Largest y or z extent of a launch grid.
constexpr int64_t kGridYZMax = 65535;

// Largest K and I one fit_sums / n_fit_sums call takes (grid limits: slices
// and row tiles are grid dimensions of at most kGridYZMax blocks).
constexpr int64_t kFitSlicesMax = kGridYZMax;
int64_t fit_rows_max();

}  // namespace octen

#define OCTEN_CUDA_TRY(expr)                                                         \
  do {                                                                               \
    cudaError_t _e = (expr);                                                         \
    if (_e != cudaSuccess) {                                                         \
      fprintf(stderr, "octen: %s failed: %s (%s:%d)\n", #expr, cudaGetErrorString(_e), \
              __FILE__, __LINE__);                                                   \
    }                                                                                \
  } while (0)
