/*
 * octen.h - C ABI of the GB300 OCTen online CP update.
 *
 * The library keeps the state of one online CP decomposition of a 3-mode
 * tensor X (I x J x K) that grows along its third (time) mode, and updates it
 * batch by batch as the paper's Algorithm 1 does: each batch of new slices is
 * compressed into P small Q x Q x Q replicas (Sec. "Parallel Compression and
 * Decomposition", Eq. 1-2), every replica is decomposed by CP-ALS, the replica
 * factors are matched on their shared anchor rows (Sec. "Factor match for
 * identifiability", Eq. 5) and lifted back into the global factors A, B, C
 * (Sec. "Update results", Eq. 6-7).  The problem statement (Sec. "Problem
 * Formulation") fixes the calls: start from existing summaries and factors,
 * append a batch, read the factors and the fit.
 *
 * Conventions shared by every call:
 *  - Every array is row-major and dense.  A slice batch X is laid out
 *    [k][i][j] (t x I x J).  A is I x R, B is J x R, C is K x R.
 *  - Projection matrices: U_all (I x Qd), V_all (J x Qd), W_all (t x Qd) with
 *    Qd = S + P (Q - S).  Columns [0, S) are the anchors shared by every
 *    replica (the paper's u, v, w of Eq. 1); replica p owns columns
 *    [S + p (Q - S), S + (p + 1) (Q - S)).  The random draws are the caller's:
 *    the library never generates them.
 *  - Precision (octen_prec): FP32 computes everything in fp32 (fp32 FFMA, no
 *    TF32).  BF16 takes bf16 slices, rounds U and V to bf16 once, and runs the
 *    two large contractions in bf16 with fp32 accumulation.  FP8E4M3 takes
 *    bf16 slices, quantises each slice to e4m3 with a per-slice absmax scale,
 *    rounds V to e4m3 and U to bf16.  W stays fp32 in every mode.  The rounded
 *    values are the matrices used by every later step.
 *  - Pointers may be device memory or host memory (pageable or pinned); the
 *    library detects which and copies host inputs to the device (and device
 *    results to host outputs) on the context's stream.  The caller owns every
 *    buffer it passes; the library copies what it keeps.
 *  - Calls run on the stream given at creation and return once the work they
 *    enqueued has finished (the status of device-side checks is known then).
 *  - Errors are status codes; nothing is thrown across the ABI.  On a status
 *    other than OCTEN_OK, octen_last_error() describes it.  A context is not
 *    thread-safe.
 */
#ifndef OCTEN_H
#define OCTEN_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct octen_ctx octen_ctx;

typedef enum {
  OCTEN_OK = 0,
  OCTEN_EINVAL = 1,     /* bad argument or unsupported shape; state unchanged   */
  OCTEN_ENOMEM = 2,     /* device allocation failed                             */
  OCTEN_ECUDA = 3,      /* a CUDA runtime call failed                           */
  OCTEN_ETIMEOUT = 4,   /* a bounded device-side wait ran out                   */
  OCTEN_ENUMERIC = 5,   /* a Cholesky pivot was not positive even after loading */
  OCTEN_ESTATE = 6      /* call out of order (e.g. append before init)          */
} octen_status;

typedef enum { OCTEN_FP32 = 0, OCTEN_BF16 = 1, OCTEN_FP8E4M3 = 2 } octen_prec;

/* Shape of one online decomposition (Algorithm 1's REQUIRE line: R, p, Q,
 * shared S; plus the fixed CP-ALS sweep count).  Limits: 1 <= R <= 32,
 * 1 <= S < Q <= 256, 1 <= P <= 65535, 1 <= I, J <= 2^24,
 * Qd = S + P (Q - S) <= 2^20, als_iters >= 1. */
typedef struct {
  int64_t I, J;
  int32_t R, P, Q, S;
  int32_t als_iters;
  int32_t prec; /* octen_prec */
} octen_config;

/* Creates a context and allocates its device state (summaries P x Q^3 fp32,
 * factors, lift operators).  `cuda_stream` is a cudaStream_t or NULL for the
 * legacy default stream.  Returns EINVAL on limits above, ENOMEM on
 * allocation failure.  *out is set only on success.  If the environment
 * variable OCTEN_DEVICE_MEMORY_LIMIT holds a byte count when the context is
 * created, the context never holds more device memory than that (its state,
 * its scratch and the init-time decomposition workspace; the lift operators'
 * transient factorisation workspace at init is not counted): an allocation
 * past the limit fails with ENOMEM like a refused cudaMalloc. */
octen_status octen_create(const octen_config *cfg, void *cuda_stream, octen_ctx **out);

/* Existing summaries and decomposition (Sec. "Problem Formulation" (a)):
 * compresses the existing tensor X_old (t_old x I x J; fp32 for FP32, bf16
 * otherwise) into the P summaries Y_p with U_all, V_all and W_old (t_old x Qd),
 * stores U_all, V_all (rounded per precision), takes A0 (I x R), B0 (J x R),
 * C0 (t_old x R) as the existing factors, forms G_p = W_old,p^T C0 and
 * precomputes the lift operators of Eq. 7.  With C0 == NULL the existing
 * decomposition is computed instead: CP-ALS of X_old (the model
 * X_old[k][i][j] = sum_r A[i][r] B[j][r] C[k][r]) from the starting guesses A0,
 * B0, with the same sweeps as the replica CP (als_iters sweeps: C, A, B, A and
 * B normalised to unit l2, a final C update); it needs a workspace of about
 * 4 t_old (I + J) R bytes and takes t_old <= 65535, t_old I < 2^31 (EINVAL
 * otherwise).  The other arrays are required.  May be called once per context
 * (ESTATE otherwise). */
octen_status octen_init(octen_ctx *ctx, const void *X_old, int64_t t_old,
                        const float *U_all, const float *V_all, const float *W_old,
                        const float *A0, const float *B0, const float *C0);

/* One pass of Algorithm 1's loop for a batch of t >= 1 new slices X_new
 * (t x I x J, element type as in octen_init) with time projections W_new
 * (t x Qd): Y_p += Z_p, CP-ALS of every replica warm-started from U_p^T A,
 * V_p^T B, anchor matching, lift of A and B, t new rows of C.  Limit
 * t <= min(64, 65535 / P) (one mode-1 product per slice and replica).
 * Everything after the batch's mode-2 contraction (mode 1, mode 3, the warm
 * start, the replica CP-ALS, the match, the lift, the new rows of C) is
 * recorded once per batch size as a CUDA graph (on a private stream, at the
 * second append made with the stage timers off) and replayed on the context's
 * stream at every later such append; a reallocated scratch buffer drops the
 * recordings; environment variable OCTEN_GRAPH=0 issues the launches one by
 * one instead.  The first call for
 * each tensor-core GEMM shape times its candidate tile configurations (only
 * ones that give bit-identical results) and keeps the fastest for the process;
 * OCTEN_AUTOTUNE=0 keeps the defaults.  Host slices are copied in pieces on a
 * stream of the library's, each piece's mode-2 contraction starting as it
 * arrives.  Failure: EINVAL, ESTATE and ENOMEM are returned before any state
 * changes (every allocation precedes the first kernel).  After ECUDA,
 * ETIMEOUT or ENUMERIC the update has run in part: the summaries hold the
 * batch, the factors may be partly updated and K is not advanced; discard
 * the context or resume from a checkpoint (octen_save / octen_load).  No
 * work of a failed call is still reading the caller's buffers when it
 * returns. */
octen_status octen_append(octen_ctx *ctx, const void *X_new, int64_t t, const float *W_new);

/* octen_append without waiting for it: the append is enqueued on the
 * context's stream and the call returns at once with a ticket for it (not in
 * the paper: a serving interface, so that the host-to-device copy of the next
 * batch overlaps the update of this one).  Arguments as in octen_append; the
 * caller keeps X_new and W_new unchanged until octen_wait of the ticket has
 * returned.  A_out (I x R), B_out (J x R) and C_new_out (t x R), each may be
 * NULL, receive the factors after this append and its new rows of C once it
 * has run (pinned host memory keeps the copies asynchronous).  Host slices
 * are copied whole into one of two staging buffers used in turn (the copy
 * waits only for the mode-2 contraction of the append two before it, and runs
 * while the appends before it update), then contracted in one piece.  At most 8 appends are in flight: a ninth waits for the oldest
 * first.  K advances when the append is enqueued.  The call does not wait for
 * the device: when C outgrows its buffer (room for 1024 rows, doubled as
 * needed) the rows so far are copied into a larger one on the stream, and the
 * old buffer is freed at the next synchronising call or octen_wait of the
 * latest ticket.  EINVAL, ESTATE and ENOMEM
 * are returned before anything is enqueued, as in octen_append; device-side
 * failures (ENUMERIC, ETIMEOUT) are returned by octen_wait, after which the
 * context is to be discarded or restored from a checkpoint. */
octen_status octen_append_async(octen_ctx *ctx, const void *X_new, int64_t t,
                                const float *W_new, float *A_out, float *B_out,
                                float *C_new_out, int64_t *ticket);

/* Waits until the append of `ticket` (and every one before it) has run and
 * returns its status (OK for a ticket already waited for; EINVAL for a ticket
 * not issued).  Not in the paper (see octen_append_async). */
octen_status octen_wait(octen_ctx *ctx, int64_t ticket);

/* One append on each of n independent decompositions (many streams with
 * uneven shapes, ranks and batch sizes).  Every context is first prepared
 * (arguments checked, every allocation made).  Once each context has recorded
 * the tail of an append of its batch size (from its second append on) and
 * every array is device memory, the whole step is one CUDA graph launch: per
 * context a branch with its head (W rows, quantisation, mode 2), a clone of
 * its recorded tail and the copy of its new C rows, the branches independent;
 * the graph is built once for the contexts and batch sizes and later steps
 * only update its heads and copies.  Otherwise the appends are enqueued one by
 * one, each on its context's stream, before any of them is waited for.  The
 * contexts' CP-ALS GEMMs run on 1 / min(n, 8) of the SMs each (environment
 * variable OCTEN_MANY_CTAS: that many CTAs; 0 all), so that several contexts'
 * GEMMs run side by side.  Arguments per stream as in octen_append.  Every
 * context whose work was enqueued without error is advanced; the first error
 * is returned (details via octen_last_error of that context). */
octen_status octen_append_many(octen_ctx *const *ctxs, int n, const void *const *X_new,
                               const int64_t *t, const float *const *W_new);

/* Copies A (I x R), B (J x R) and C (K x R, K = rows so far) into caller
 * buffers; any pointer may be NULL to skip it.  *K_out (if non-NULL) gets K. */
octen_status octen_get_factors(const octen_ctx *ctx, float *A, float *B, float *C,
                               int64_t *K_out);

/* Number of rows of C so far. */
int64_t octen_rows(const octen_ctx *ctx);

/* Bytes of device memory the context holds now (state and scratch; the
 * figure OCTEN_DEVICE_MEMORY_LIMIT is compared with).  Not in the paper: a
 * read-out for callers that budget device memory.  0 for NULL. */
uint64_t octen_device_bytes(const octen_ctx *ctx);

/* Fitness of the current factors on K slices X_all (K x I x J, element type
 * as in octen_init): 1 - ||X - [[A, B, C]]||_F / ||X||_F (Sec. "Evaluation
 * Measures", as a fraction), with fp64 reductions.  K must equal octen_rows();
 * I <= 65535 * 32 (EINVAL otherwise).  Slices are reduced in chunks of at most
 * 65535 (16 when X_all is host memory, each chunk staged on the stream). */
octen_status octen_fit(octen_ctx *ctx, const void *X_all, int64_t K, double *fit_out);

/* Copies the current summaries Y_p (P x Q x Q x Q, [p][a][b][c]) out. */
octen_status octen_get_replicas(const octen_ctx *ctx, float *Y);

/* Copies the last append's replica factors out, each P x Q x R ([p][q][r]):
 * which = 0 gives the raw CP-ALS output, which = 1 the output of the anchor
 * match (permuted and scaled).  perm (P x R int32, perm[p][s] = matched raw
 * column) and scales (P x 2 x R fp64: d_a then d_b) may be NULL. */
octen_status octen_get_replica_factors(const octen_ctx *ctx, int which, float *At,
                                       float *Bt, float *Ct, int32_t *perm,
                                       double *scales);

/* Stateless compression of one slice batch (Sec. "Parallel Compression and
 * Decomposition"): Z_p = X x1 U_p^T x2 V_p^T x3 W_p^T for every replica,
 * written to Z (P x Q x Q x Q fp32, overwritten).  Same shapes, layouts,
 * precisions and rounding as octen_init / octen_append; scratch space is
 * allocated and freed inside the call.  cuda_stream as in octen_create. */
octen_status octen_compress(const octen_config *cfg, void *cuda_stream, const void *X,
                            int64_t t, const float *U_all, const float *V_all,
                            const float *W_all, float *Z);

/* octen_compress without any device allocation.  The paper has no
 * counterpart: this entry point exists for callers that cannot call
 * cudaMalloc (processes living inside a fixed device-memory budget handed out
 * by a host framework, plugins whose host forbids the CUDA allocator, latency-
 * critical code that must not pay for an allocation).  It computes what
 * octen_compress computes, with the same arguments, but
 *  - every array (X, U_all, V_all, W_all, Z) must already be device memory
 *    (host buffers are rejected with OCTEN_EINVAL: staging them would
 *    allocate);
 *  - all scratch lives in one static device array of 64 MiB that every GPU
 *    loading the library holds until the process exits: the transposed
 *    projections (P*Q*I + Qd*J operand elements) plus, per slice of a pass,
 *    its mode-2 and mode-1 products (P*Q*I operand elements and P*Q*Q fp32;
 *    in fp8 mode also the I*J e4m3 slice and its scale).  Slices are processed
 *    in passes that fit (at most 64 slices and at most 65535 / P per pass); a
 *    shape is rejected with OCTEN_EINVAL and a message on stderr when its
 *    projections plus the scratch of one slice exceed 64 MiB, and so is a
 *    configuration outside octen_create's limits;
 *  - the first call on a device looks up the array's address on that device
 *    (cudaGetSymbolAddress) and caches it: make that first call before any
 *    stream capture;
 *  - the array is shared by all calls and keeps the last call's contents
 *    (each call clears what must start at zero); calls whose GPU work
 *    overlaps (other streams or threads) race on it and must be serialised
 *    by the caller.
 * Returns after the work has finished on `cuda_stream`. */
octen_status octen_compress_noalloc(const octen_config *cfg, void *cuda_stream, const void *X,
                                    int64_t t, const float *U_all, const float *V_all,
                                    const float *W_all, float *Z);

/* Checkpoint and resume (not in the paper; the state is what its complexity
 * analysis says OCTen keeps: summaries, projections, factors).  octen_save
 * writes the full state of an initialised context to a file; octen_load
 * creates a new context on `cuda_stream` from such a file.  A loaded context
 * continues the stream exactly as the saved one would (same results, bit for
 * bit, on the same GPU and library build).  EINVAL on a bad path or file: a
 * missing or short file, another magic, a row count below 1 or above 2^40,
 * or lift-operator layout flags that the configuration's shapes contradict
 * (all checked before any device memory is allocated, except the flags,
 * checked right after the context is created); ENOMEM when the state does
 * not fit.  *out is set only on success. */
octen_status octen_save(const octen_ctx *ctx, const char *path);
octen_status octen_load(const char *path, void *cuda_stream, octen_ctx **out);

/* Releases the context and its device memory (NULL is allowed). */
void octen_destroy(octen_ctx *ctx);

/* Human-readable description of the last error on this context (never NULL). */
const char *octen_last_error(const octen_ctx *ctx);

/* Short name of a status code (never NULL). */
const char *octen_status_name(octen_status s);

/* Number of kernel launches the library has issued in this process, and how
 * many of them were tcgen05 tensor-core contractions (the bf16 / e4m3 paths
 * use them whenever the device is sm_103 and every operand row pitch is a
 * multiple of 16 bytes: J and I multiples of 8 for bf16, J a multiple of 16
 * for e4m3; otherwise the SIMT kernels run). */
uint64_t octen_launch_count(void);
uint64_t octen_tc_launch_count(void);

/* Tensor-core contractions that were wanted (bf16 / e4m3 operands on sm_103)
 * but refused, an operand row pitch off the TMA rules or a resource limit,
 * so that the SIMT kernels ran instead.  The first one in a process is also
 * reported on stderr.  Not in the paper: a guard against a slow path passing
 * unnoticed. */
uint64_t octen_tc_fallback_count(void);

/* Stage timers (measurement aid, not part of the method).  With timing on,
 * every append records CUDA events on the context's stream around each
 * stage: quantize, mode2, mode1, mode3 (the three contractions of the
 * compression), warm_start, als_gemm (the two passes over each replica per
 * sweep: tcgen05 GEMMs in bf16 / e4m3 mode, SIMT kernels in fp32 mode),
 * als_aux (the other CP-ALS data kernels), als_solve (the R x R normal-equation
 * solves), align, lift, c_solve.
 * octen_stage_times fills ms[i] (accumulated milliseconds) and launches[i]
 * (timed intervals) for i < octen_stage_count(); either may be NULL. */
int octen_stage_count(void);
const char *octen_stage_name(int i);
octen_status octen_set_timing(octen_ctx *ctx, int on);
octen_status octen_stage_times(const octen_ctx *ctx, double *ms, uint64_t *launches);
octen_status octen_reset_stage_times(octen_ctx *ctx);

/* ------------------------------------------------------------------------
 * N-mode extension (Sec. "Extending to Higher-Order Tensors"): a tensor with
 * N - 1 non-temporal modes I_1 x ... x I_{N-1} growing in its N-th (time)
 * mode.  Every replica p compresses every non-temporal mode n with its own
 * projection block of U_n,all (I_n x Qd, the same column convention as U_all
 * above: anchors [0, S) shared, replica p's private block after them) and the
 * time mode with W (t x Qd), keeps the N-way summary Y_p (Q^N), decomposes it
 * by CP-ALS (per sweep: the time factor, then each non-temporal factor
 * normalised to unit l2; a final time-factor update), matches the replicas on
 * the anchor rows of every non-temporal mode (similarity: the sum over those
 * modes of |cos|; scales per mode, the time factor scaled by their product)
 * and lifts each non-temporal factor as in Eq. 7 with its own stacked
 * projection; the new rows of the time factor are solved as in the 3-mode
 * update.  With N = 3 this is the 3-mode update in fp32.
 *
 * Precision (prec): OCTEN_FP32 computes everything in fp32.  OCTEN_BF16 takes
 * bf16 slices, rounds every U_all[n] to bf16 once (the rounded values are the
 * matrices from then on), and runs the first contraction of the compression
 * (every slice against all P Q columns of the innermost mode's projection,
 * the one pass that reads the slices) in bf16 with fp32 accumulation, on the
 * tensor cores when I_{N-1} is a multiple of 8; the rest of the update is
 * fp32.  Slices are laid out [k][i_1]...[i_{N-1}] (fp32 or bf16 by prec),
 * summaries [p][q_1]...[q_{N-1}][c].  Pointers may be device or host memory
 * (host inputs are staged on the context's stream).  Same status codes and
 * threading rules as the 3-mode calls.
 * ------------------------------------------------------------------------ */
typedef struct octen_nctx octen_nctx;

#define OCTEN_MAX_MODES 6

/* Limits: 3 <= N <= OCTEN_MAX_MODES, 1 <= R <= 32, 1 <= S < Q <= 256,
 * 1 <= P <= 65535, als_iters >= 1, 1 <= dims[n] <= 2^24 for n < N - 1 (later
 * entries ignored),
 * Q^N <= 2^24 and P Q^N <= 2^28, and the replica CP state of one summary must
 * fit one thread block's shared memory (N Q R-ish floats; X_p itself is read
 * from global memory when it does not fit). */
typedef struct {
  int32_t N;
  int32_t R, P, Q, S;
  int32_t als_iters;
  int64_t dims[OCTEN_MAX_MODES - 1];
  int32_t prec; /* OCTEN_FP32 or OCTEN_BF16 */
} octen_nconfig;

/* Creates a context (summaries, projections, factors, scratch on the device).
 * EINVAL on the limits above, ENOMEM on allocation failure. */
octen_status octen_n_create(const octen_nconfig *cfg, void *cuda_stream, octen_nctx **out);

/* Existing summaries and decomposition: compresses X_old (t_old slices, element
 * type by prec) with U_all[n] (n < N - 1, each I_n x Qd) and W_old
 * (t_old x Qd), takes A0[n] (I_n x R) and C0 (t_old x R) as the existing
 * factors, forms G_p = W_old,p^T C0 and the lift operators of every
 * non-temporal mode.  With C0 == NULL the existing decomposition is computed
 * instead: the N-way CP-ALS of X_old (model X_old[k][i_1]..[i_{N-1}] =
 * sum_r prod_n A_n[i_n][r] C[k][r]) from the starting guesses A0, with the
 * sweeps of the replica CP (als_iters sweeps: the time factor, then every
 * non-temporal factor normalised to unit l2, a final time-factor update); it
 * needs a workspace of about 4 R (t_old + sum_n I_n) bytes plus 4 MB.  The
 * other arrays are required.  Once per context (ESTATE otherwise). */
octen_status octen_n_init(octen_nctx *ctx, const void *X_old, int64_t t_old,
                          const float *const *U_all, const float *W_old,
                          const float *const *A0, const float *C0);

/* One update with t new slices (1 <= t <= 64, element type by prec) and their
 * time projections W_new (t x Qd). */
octen_status octen_n_append(octen_nctx *ctx, const void *X_new, int64_t t,
                            const float *W_new);

/* Copies A[n] (I_n x R, n < N - 1) and C (K x R); A, any A[n] and C may be
 * NULL.  *K_out (if non-NULL) gets K. */
octen_status octen_n_get_factors(const octen_nctx *ctx, float *const *A, float *C,
                                 int64_t *K_out);

/* Copies the summaries Y (P x Q^N, [p][q_1]...[q_{N-1}][c]) out. */
octen_status octen_n_get_replicas(const octen_nctx *ctx, float *Y);

/* The last update's replica factors, F[n] (P x Q x R) for n < N - 1 and the
 * time factor F[N - 1]: which = 0 the raw CP-ALS output, 1 the matched ones.
 * perm (P x R int32) and scales (P x (N - 1) x R fp64, the per-mode anchor
 * scales) may be NULL, as may F and any F[n]. */
octen_status octen_n_get_replica_factors(const octen_nctx *ctx, int which, float *const *F,
                                         int32_t *perm, double *scales);

/* Rows of the time factor so far. */
int64_t octen_n_rows(const octen_nctx *ctx);

/* Fitness of the current factors on the K = octen_n_rows() slices X_all
 * (K x I_1 x ... x I_{N-1}, element type by prec, device or host):
 * 1 - ||X - [[A_1, ..., A_{N-1}, C]]||_F / ||X||_F (Sec. "Evaluation
 * Measures"), the residual formed element by element with fp64 sums. */
octen_status octen_n_fit(octen_nctx *ctx, const void *X_all, int64_t K, double *fit_out);

/* Checkpoint and resume of an N-mode context (as octen_save / octen_load:
 * the projections, lift operators, factors, summaries and G_p; a loaded
 * context continues the stream bit for bit on the same GPU and build). */
octen_status octen_n_save(const octen_nctx *ctx, const char *path);
octen_status octen_n_load(const char *path, void *cuda_stream, octen_nctx **out);

/* Stage timers of the N-mode update (measurement aid): with timing on, every
 * append records CUDA events around compress, warm_start, als, align, lift
 * and c_solve; same conventions as octen_stage_times. */
int octen_n_stage_count(void);
const char *octen_n_stage_name(int i);
octen_status octen_n_set_timing(octen_nctx *ctx, int on);
octen_status octen_n_stage_times(const octen_nctx *ctx, double *ms, uint64_t *launches);

void octen_n_destroy(octen_nctx *ctx);
const char *octen_n_last_error(const octen_nctx *ctx);

#ifdef __cplusplus
}
#endif

#endif /* OCTEN_H */
