// C ABI of the N-mode extension (octen_n_* in include/octen.h): the state of
// one online CP decomposition of a tensor with N - 1 non-temporal modes growing
// in its time mode, and the order of the stages of one update (Sec. "Extending
// to Higher-Order Tensors" applied to Algorithm 1's loop body): compress the
// batch into every replica's N-way summary, CP of every summary warm-started
// from the projected previous factors, anchor match in every non-temporal
// mode, lift of every non-temporal factor (Eq. 7) and the new rows of the time
// factor.  fp32, or bf16 slices and projections with the slice-reading first
// contraction of the compression in bf16 (fp32 accumulation).
#include <cmath>
#include <cstdarg>
#include <cstring>
#include <string>
#include <vector>

#include "octen_internal.cuh"

using namespace octen;

namespace {

int nround_rt(int R) { return R <= 8 ? 8 : (R <= 16 ? 16 : 32); }

// bounds of one compression pass (rows of a GEMM stay within the SIMT
// kernels' grid limits, the two intermediate buffers within 1 GiB each)
constexpr int64_t kNRowsMax = 4000000;
constexpr int64_t kNBufFloatsMax = int64_t(1) << 28;
constexpr int64_t kNBatchMax = 64;

// stages timed with CUDA events when timing is on
enum NStage : int { kNCompress = 0, kNWarm, kNAls, kNAlign, kNLift, kNCsolve, kNStages };
const char *const kNStageNames[kNStages] = {"compress", "warm_start", "als", "align", "lift",
                                            "c_solve"};

}  // namespace

struct octen_nctx {
  octen_nconfig cfg{};
  int nm = 0, NN = 0, Qd = 0, RT = 8;
  int64_t dims[kMaxNModes] = {};
  int64_t slice = 1;      // elements per slice
  Elem xin = Elem::F32;   // slice element type (OCTEN_FP32 or OCTEN_BF16)
  void *Ut16 = nullptr;   // bf16 replica transpose of the innermost mode (bf16 mode)
  int64_t tchunk = 1;     // slices per compression pass
  cudaStream_t st = nullptr;
  bool initialized = false;
  std::string err;
  int64_t K = 0, Kcap = 0;
  std::vector<void *> owned;

  float *U32[kMaxNModes] = {}, *Ut[kMaxNModes] = {}, *L[kMaxNModes] = {};
  float *A[kMaxNModes] = {}, *PF[kMaxNModes] = {}, *Gw[kMaxNModes] = {};
  float *Ft[kMaxNModes] = {}, *Fh[kMaxNModes] = {};
  int over[kMaxNModes] = {};
  float *Y = nullptr, *G = nullptr, *C = nullptr, *e = nullptr;
  float *bufA = nullptr, *bufB = nullptr, *Wt = nullptr, *csolve = nullptr, *splitk = nullptr;
  int *perm = nullptr, *dstatus = nullptr;
  double *scales = nullptr;
  static constexpr size_t kSplitkFloats = size_t(4) << 20;
  // staging of host inputs
  void *stg[2] = {nullptr, nullptr};
  size_t stg_bytes[2] = {0, 0};

  // stage timers
  bool timing = false;
  std::vector<cudaEvent_t> evpool;
  size_t evused = 0;
  cudaEvent_t open_ev = nullptr;
  struct Pending { int stage; cudaEvent_t a, b; };
  std::vector<Pending> pending;
  double stage_ms[kNStages] = {};
  uint64_t stage_n[kNStages] = {};

  void mark(int stage, int begin) {
    if (!timing) return;
    if (evused == evpool.size()) {
      cudaEvent_t e;
      if (cudaEventCreate(&e) != cudaSuccess) return;
      evpool.push_back(e);
    }
    cudaEvent_t e = evpool[evused++];
    cudaEventRecord(e, st);
    if (begin) open_ev = e;
    else if (open_ev) pending.push_back({stage, open_ev, e});
  }
  void flush_timers() {
    for (const Pending &q : pending) {
      float ms = 0.f;
      if (cudaEventElapsedTime(&ms, q.a, q.b) == cudaSuccess) {
        stage_ms[q.stage] += ms;
        stage_n[q.stage] += 1;
      } else {
        cudaGetLastError();
      }
    }
    pending.clear();
    evused = 0;
  }

  ~octen_nctx() {
    cudaStreamSynchronize(st);
    for (cudaEvent_t e : evpool) cudaEventDestroy(e);
    for (void *p : owned) cudaFree(p);
    if (C) cudaFree(C);
    for (void *p : stg) cudaFree(p);
  }

  octen_status fail(octen_status s, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    err = buf;
    return s;
  }

  template <class T>
  bool alloc(T *&ptr, size_t count) {
    void *p = nullptr;
    if (cudaMalloc(&p, count * sizeof(T) + 16) != cudaSuccess) {
      cudaGetLastError();
      return false;
    }
    owned.push_back(p);
    ptr = static_cast<T *>(p);
    return true;
  }

  // device view of a caller buffer (copied into staging slot `slot` if host)
  template <class T>
  const T *stage_in(const T *p, size_t bytes, int slot) {
    if (is_device_pointer(p)) return p;
    if (stg_bytes[slot] < bytes) {
      cudaStreamSynchronize(st);
      cudaFree(stg[slot]);
      stg[slot] = nullptr;
      stg_bytes[slot] = 0;
      if (cudaMalloc(&stg[slot], bytes) != cudaSuccess) {
        cudaGetLastError();
        stg[slot] = nullptr;
        return nullptr;
      }
      stg_bytes[slot] = bytes;
    }
    if (cudaMemcpyAsync(stg[slot], p, bytes, cudaMemcpyHostToDevice, st) != cudaSuccess)
      return nullptr;
    return static_cast<const T *>(stg[slot]);
  }

  octen_status sync_check(const char *what) {
    cudaError_t e = cudaStreamSynchronize(st);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e != cudaSuccess) return fail(OCTEN_ECUDA, "%s: %s", what, cudaGetErrorString(e));
    if (!pending.empty()) flush_timers();
    int flags = 0;
    cudaMemcpy(&flags, dstatus, sizeof(int), cudaMemcpyDeviceToHost);
    if (flags) {
      cudaMemsetAsync(dstatus, 0, sizeof(int), st);
      cudaStreamSynchronize(st);
      if (flags & kDevTimeout) return fail(OCTEN_ETIMEOUT, "%s: a device wait ran out", what);
      return fail(OCTEN_ENUMERIC, "%s: a Cholesky pivot was not positive", what);
    }
    return OCTEN_OK;
  }

  LiftEnv lift_env() {
    return LiftEnv{Qd, cfg.P, cfg.Q, cfg.S, cfg.R, RT, st, dstatus, e, splitk, kSplitkFloats};
  }

  bool ensure_c(int64_t rows) {
    if (rows <= Kcap) return true;
    if (rows > kCRowsMax) return false;
    int64_t cap = Kcap > 0 ? Kcap : 64;
    while (cap < rows) cap *= 2;
    float *nc = nullptr;
    if (cudaMalloc(&nc, (size_t)cap * cfg.R * sizeof(float)) != cudaSuccess) {
      cudaGetLastError();
      return false;
    }
    if (C) {
      cudaMemcpyAsync(nc, C, (size_t)K * cfg.R * sizeof(float), cudaMemcpyDeviceToDevice, st);
      cudaStreamSynchronize(st);
      cudaFree(C);
    }
    C = nc;
    Kcap = cap;
    return true;
  }

  // Y_p += compression of t slices (device X, device W rows t x Qd)
  size_t slice_bytes() const { return (size_t)slice * elem_size(xin); }
  const void *slice_at(const void *X, int64_t k) const {
    return static_cast<const char *>(X) + k * slice_bytes();
  }

  void compress(const void *X, int64_t t, const float *W) {
    NCompressInput c{nm, cfg.P, cfg.Q, dims, Ut, bufA, bufB};
    for (int64_t k0 = 0; k0 < t; k0 += tchunk) {
      const int64_t n = t - k0 < tchunk ? t - k0 : tchunk;
      make_replica_transpose(W + k0 * Qd, n, cfg.P, cfg.Q, cfg.S, Qd, Wt, Elem::F32, st);
      ncompress_chunk(c, slice_at(X, k0), xin, n, Wt, Y, st, Ut16, dstatus);
    }
  }

  // PF = U_all^T F (Qd x R) for non-temporal mode n
  void project(int n) {
    GemmArgs g{};
    g.A = U32[n]; g.ta = Elem::F32; g.sAm = 1; g.sAk = Qd;
    g.B = A[n]; g.tb = Elem::F32; g.sBn = 1; g.sBk = cfg.R;
    g.D = PF[n]; g.sDm = cfg.R; g.sDn = 1;
    g.M = Qd; g.N = cfg.R; g.K = (int)dims[n]; g.batch = 1; g.alpha = 1.f; g.beta = 0.f;
    g.split_scratch = splitk; g.split_scratch_floats = kSplitkFloats;
    gemm_strided(g, st);
  }
};

namespace {

octen_status nvalidate(const octen_nconfig *c, std::string &why) {
  char buf[320];
  if (!c) { why = "config is NULL"; return OCTEN_EINVAL; }
  if (c->N < 3 || c->N > kMaxNModes || c->R < 1 || c->R > 32 || c->P < 1 ||
      c->P > kGridYZMax || c->Q < 2 || c->Q > 256 || c->S < 1 || c->S >= c->Q ||
      c->als_iters < 1 || (c->prec != OCTEN_FP32 && c->prec != OCTEN_BF16)) {
    snprintf(buf, sizeof buf,
             "unsupported config N=%d R=%d P=%d Q=%d S=%d iters=%d prec=%d (limits: "
             "3<=N<=%d, 1<=R<=32, 1<=S<Q<=256, 1<=P<=65535, iters>=1, prec fp32 or bf16)",
             c->N, c->R, c->P, c->Q, c->S, c->als_iters, c->prec, kMaxNModes);
    why = buf;
    return OCTEN_EINVAL;
  }
  int64_t slice = 1;
  for (int n = 0; n < c->N - 1; ++n) {
    if (c->dims[n] < 1 || c->dims[n] > (1 << 24)) {
      snprintf(buf, sizeof buf, "dims[%d]=%lld out of [1, 2^24]", n, (long long)c->dims[n]);
      why = buf;
      return OCTEN_EINVAL;
    }
    slice *= c->dims[n];
    if (slice > (int64_t(1) << 31)) { why = "a slice holds more than 2^31 elements"; return OCTEN_EINVAL; }
  }
  int64_t qn = 1;
  for (int n = 0; n < c->N; ++n) qn *= c->Q;
  if (qn > (int64_t(1) << 24) || qn * c->P > (int64_t(1) << 28)) {
    why = "summaries too large (Q^N <= 2^24 and P Q^N <= 2^28)";
    return OCTEN_EINVAL;
  }
  const int64_t Qd = (int64_t)c->S + (int64_t)c->P * (c->Q - c->S);
  if (Qd > (1 << 20)) { why = "S + P (Q - S) above 2^20"; return OCTEN_EINVAL; }
  const int nm = c->N - 1;
  if (ncompress_rows_max(nm, c->dims, c->Q, 1) > kNRowsMax ||
      ncompress_buf_floats(nm, c->dims, c->P, c->Q, 1) > kNBufFloatsMax) {
    why = "one slice's compression intermediates exceed the pass limits";
    return OCTEN_EINVAL;
  }
  if (!nals_fits(c->N, c->Q, nround_rt(c->R))) {
    why = "replica CP-ALS: Q too large for one CTA per replica";
    return OCTEN_EINVAL;
  }
  return OCTEN_OK;
}

}  // namespace

extern "C" {

octen_status octen_n_create(const octen_nconfig *cfg, void *cuda_stream, octen_nctx **out) {
  if (!out) return OCTEN_EINVAL;
  std::string why;
  if (nvalidate(cfg, why) != OCTEN_OK) {
    fprintf(stderr, "octen_n_create: %s\n", why.c_str());
    return OCTEN_EINVAL;
  }
  octen_nctx *x = new octen_nctx();
  x->cfg = *cfg;
  x->NN = cfg->N;
  x->nm = cfg->N - 1;
  for (int n = 0; n < x->nm; ++n) {
    x->dims[n] = cfg->dims[n];
    x->slice *= cfg->dims[n];
  }
  x->Qd = cfg->S + cfg->P * (cfg->Q - cfg->S);
  x->RT = nround_rt(cfg->R);
  x->xin = cfg->prec == OCTEN_BF16 ? Elem::BF16 : Elem::F32;
  x->st = static_cast<cudaStream_t>(cuda_stream);
  const int64_t r1 = ncompress_rows_max(x->nm, x->dims, cfg->Q, 1);
  const int64_t b1 = ncompress_buf_floats(x->nm, x->dims, cfg->P, cfg->Q, 1);
  int64_t tc = kNBatchMax;
  if (tc * r1 > kNRowsMax) tc = kNRowsMax / r1;
  if (tc * b1 > kNBufFloatsMax) tc = kNBufFloatsMax / b1;
  x->tchunk = tc < 1 ? 1 : tc;
  const octen_nconfig &c = x->cfg;
  const size_t P = c.P, Q = c.Q, RT = x->RT, Qd = x->Qd;
  size_t qn = 1;
  for (int n = 0; n < x->NN; ++n) qn *= Q;
  bool ok = true;
  for (int n = 0; n < x->nm && ok; ++n) {
    const size_t I = (size_t)x->dims[n];
    ok = x->alloc(x->U32[n], I * Qd) && x->alloc(x->Ut[n], P * Q * I) &&
         x->alloc(x->L[n], I * Qd) && x->alloc(x->A[n], I * c.R) &&
         x->alloc(x->PF[n], Qd * c.R) && x->alloc(x->Gw[n], P * RT * RT);
  }
  for (int n = 0; n <= x->nm && ok; ++n)
    ok = x->alloc(x->Ft[n], P * Q * RT) && x->alloc(x->Fh[n], P * Q * RT);
  const size_t buf = (size_t)ncompress_buf_floats(x->nm, x->dims, c.P, c.Q, x->tchunk);
  ok = ok && x->alloc(x->Y, P * qn) && x->alloc(x->G, P * Q * c.R) &&
       x->alloc(x->e, Qd * c.R) && x->alloc(x->bufA, buf) && x->alloc(x->bufB, buf) &&
       x->alloc(x->Wt, P * Q * (size_t)x->tchunk) &&
       x->alloc(x->csolve, c_solve_scratch_floats(kNBatchMax, Qd, c.R)) &&
       x->alloc(x->splitk, octen_nctx::kSplitkFloats) && x->alloc(x->perm, P * c.R) &&
       x->alloc(x->scales, P * x->nm * c.R) && x->alloc(x->dstatus, 1);
  if (ok && x->xin == Elem::BF16) {
    __nv_bfloat16 *u16 = nullptr;
    ok = x->alloc(u16, P * Q * (size_t)x->dims[x->nm - 1]);
    x->Ut16 = u16;
  }
  if (!ok) {
    cudaGetLastError();
    delete x;
    return OCTEN_ENOMEM;
  }
  cudaMemsetAsync(x->Y, 0, P * qn * sizeof(float), x->st);
  cudaMemsetAsync(x->G, 0, P * Q * c.R * sizeof(float), x->st);
  cudaMemsetAsync(x->dstatus, 0, sizeof(int), x->st);
  if (x->sync_check("create") != OCTEN_OK) {
    delete x;
    return OCTEN_ECUDA;
  }
  *out = x;
  return OCTEN_OK;
}

octen_status octen_n_init(octen_nctx *x, const void *X_old, int64_t t_old,
                          const float *const *U_all, const float *W_old,
                          const float *const *A0, const float *C0) {
  if (!x) return OCTEN_EINVAL;
  if (x->initialized) return x->fail(OCTEN_ESTATE, "octen_n_init called twice");
  if (!X_old || !U_all || !W_old || !A0 || t_old < 1)
    return x->fail(OCTEN_EINVAL, "octen_n_init: X_old, U_all, W_old, A0 are required, t_old >= 1");
  if (!C0 && t_old > (int64_t)1 << 31)
    return x->fail(OCTEN_EINVAL, "octen_n_init: decomposing X_old takes t_old < 2^31");
  for (int n = 0; n < x->nm; ++n)
    if (!U_all[n] || !A0[n]) return x->fail(OCTEN_EINVAL, "octen_n_init: U_all[%d] or A0[%d] is NULL", n, n);
  const octen_nconfig &c = x->cfg;
  const int Qd = x->Qd;
  for (int n = 0; n < x->nm; ++n) {
    // bf16 mode: the projections are rounded to bf16 once (through L[n],
    // free until the lift operators are built); the rounded values are the
    // matrices from then on
    if (x->xin == Elem::BF16) {
      cudaMemcpyAsync(x->L[n], U_all[n], (size_t)x->dims[n] * Qd * 4, cudaMemcpyDefault, x->st);
      round_copy(x->L[n], x->U32[n], x->dims[n] * Qd, Elem::BF16, x->st);
    } else {
      cudaMemcpyAsync(x->U32[n], U_all[n], (size_t)x->dims[n] * Qd * 4, cudaMemcpyDefault,
                      x->st);
    }
    make_replica_transpose(x->U32[n], x->dims[n], c.P, c.Q, c.S, Qd, x->Ut[n], Elem::F32, x->st);
    if (x->xin == Elem::BF16 && n == x->nm - 1)
      make_replica_transpose(x->U32[n], x->dims[n], c.P, c.Q, c.S, Qd, x->Ut16, Elem::BF16,
                             x->st);
    cudaMemcpyAsync(x->A[n], A0[n], (size_t)x->dims[n] * c.R * 4, cudaMemcpyDefault, x->st);
  }
  octen_status s = x->sync_check("projection setup");
  if (s != OCTEN_OK) return s;
  const float *Wd = x->stage_in(W_old, (size_t)t_old * Qd * 4, 1);
  if (!Wd) return x->fail(OCTEN_ENOMEM, "staging W_old");
  const bool xdev = is_device_pointer(X_old);
  for (int64_t k0 = 0; k0 < t_old; k0 += x->tchunk) {
    const int64_t n = t_old - k0 < x->tchunk ? t_old - k0 : x->tchunk;
    const void *Xd = xdev ? x->slice_at(X_old, k0)
                          : x->stage_in(x->slice_at(X_old, k0), n * x->slice_bytes(), 0);
    if (!Xd) return x->fail(OCTEN_ENOMEM, "staging X_old");
    x->compress(Xd, n, Wd + k0 * Qd);
    if (!xdev) cudaStreamSynchronize(x->st);   // the staging slot is reused
  }
  if (!x->ensure_c(t_old)) return x->fail(OCTEN_ENOMEM, "C");
  if (C0) {
    cudaMemcpyAsync(x->C, C0, (size_t)t_old * c.R * 4, cudaMemcpyDefault, x->st);
  } else {
    // the existing decomposition: N-way CP-ALS of X_old from the guesses A0
    // (already in x->A), results into x->A and x->C
    s = x->sync_check("init summaries");
    if (s != OCTEN_OK) return s;
    const void *Xd = xdev ? X_old : x->stage_in(X_old, t_old * x->slice_bytes(), 0);
    if (!Xd) return x->fail(OCTEN_ENOMEM, "staging X_old");
    int64_t dims[kMaxNModes];
    dims[0] = t_old;
    for (int n = 0; n < x->nm; ++n) dims[n + 1] = x->dims[n];
    const size_t wf = dense_cp_n_work_floats(x->NN, dims, x->RT);
    float *work = nullptr;
    if (cudaMalloc(&work, wf * sizeof(float)) != cudaSuccess) {
      cudaGetLastError();
      return x->fail(OCTEN_ENOMEM, "N-way CP-ALS workspace (%zu bytes)", wf * sizeof(float));
    }
    const float *a0[kMaxNModes];
    float *aout[kMaxNModes];
    for (int n = 0; n < x->nm; ++n) {
      a0[n] = x->A[n];
      aout[n] = x->A[n];
    }
    DenseCpNArgs a{};
    a.X = Xd; a.xt = x->xin; a.NN = x->NN; a.dims = dims; a.R = c.R; a.iters = c.als_iters;
    a.A0 = a0; a.A_out = aout; a.C_out = x->C; a.work = work; a.status = x->dstatus;
    a.st = x->st;
    dense_cp_n(a, x->RT);
    s = x->sync_check("init decomposition");
    cudaFree(work);
    if (s != OCTEN_OK) return s;
  }
  update_g(Wd, x->C, t_old, c.P, c.Q, c.S, Qd, c.R, x->G, x->st);
  s = x->sync_check("init summaries");
  if (s != OCTEN_OK) return s;
  x->K = t_old;
  for (int n = 0; n < x->nm; ++n) {
    if (!lift_build(x->lift_env(), x->U32[n], x->dims[n], x->L[n], x->over[n]))
      return x->fail(OCTEN_ENOMEM, "lift operator of mode %d", n);
    s = x->sync_check("lift operator");
    if (s != OCTEN_OK) return s;
  }
  x->initialized = true;
  return OCTEN_OK;
}

octen_status octen_n_append(octen_nctx *x, const void *X_new, int64_t t, const float *W_new) {
  if (!x) return OCTEN_EINVAL;
  if (!x->initialized) return x->fail(OCTEN_ESTATE, "octen_n_append before octen_n_init");
  if (!X_new || !W_new || t < 1 || t > kNBatchMax)
    return x->fail(OCTEN_EINVAL, "octen_n_append: need X_new, W_new and 1 <= t <= %d",
                   (int)kNBatchMax);
  const octen_nconfig &c = x->cfg;
  const int Qd = x->Qd, RT = x->RT, nm = x->nm;
  if (!x->ensure_c(x->K + t)) return x->fail(OCTEN_ENOMEM, "C");
  const void *Xd = x->stage_in(X_new, t * x->slice_bytes(), 0);
  const float *Wd = x->stage_in(W_new, (size_t)t * Qd * 4, 1);
  if (!Xd || !Wd) return x->fail(OCTEN_ENOMEM, "staging the batch");
  // 1. compress the batch into the summaries
  x->mark(kNCompress, 1);
  x->compress(Xd, t, Wd);
  x->mark(kNCompress, 0);
  // 2. CP of every summary, warm-started from U_n,p^T A_n
  x->mark(kNWarm, 1);
  for (int n = 0; n < nm; ++n) {
    x->project(n);
    warm_start(x->PF[n], c.P, c.Q, c.S, c.R, RT, x->Ft[n], x->Gw[n], x->st);
  }
  x->mark(kNWarm, 0);
  NAlsInput ai{};
  ai.Y = x->Y;
  for (int n = 0; n <= nm; ++n) ai.F[n] = x->Ft[n];
  for (int n = 0; n < nm; ++n) ai.G0[n] = x->Gw[n];
  ai.NN = x->NN; ai.P = c.P; ai.Q = c.Q; ai.R = c.R; ai.RT = RT; ai.iters = c.als_iters;
  ai.status = x->dstatus;
  x->mark(kNAls, 1);
  if (!nals_run(ai, x->st)) return x->fail(OCTEN_ECUDA, "replica CP-ALS launch failed");
  x->mark(kNAls, 0);
  // 3. anchor match in every non-temporal mode
  NAlignInput mi{};
  for (int n = 0; n <= nm; ++n) {
    mi.F[n] = x->Ft[n];
    mi.Fh[n] = x->Fh[n];
  }
  for (int n = 0; n < nm; ++n) mi.PF[n] = x->PF[n];
  mi.nm = nm; mi.P = c.P; mi.Q = c.Q; mi.S = c.S; mi.R = c.R; mi.RT = RT;
  mi.perm = x->perm; mi.scales = x->scales;
  x->mark(kNAlign, 1);
  n_align(mi, x->st);
  x->mark(kNAlign, 0);
  // 4. lift every non-temporal factor, solve the new rows of the time factor
  x->mark(kNLift, 1);
  for (int n = 0; n < nm; ++n)
    lift_apply(x->lift_env(), x->Fh[n], x->PF[n], x->L[n], x->over[n], x->dims[n], x->A[n]);
  x->mark(kNLift, 0);
  float *C_new = x->C + x->K * c.R;
  x->mark(kNCsolve, 1);
  solve_c_new(Wd, x->Fh[nm], x->G, t, c.P, c.Q, c.S, Qd, c.R, RT, x->csolve, C_new, x->dstatus,
              x->st);
  update_g(Wd, C_new, t, c.P, c.Q, c.S, Qd, c.R, x->G, x->st);
  x->mark(kNCsolve, 0);
  const octen_status s = x->sync_check("append");
  if (s != OCTEN_OK) return s;
  x->K += t;
  return OCTEN_OK;
}

octen_status octen_n_get_factors(const octen_nctx *cx, float *const *A, float *C,
                                 int64_t *K_out) {
  octen_nctx *x = const_cast<octen_nctx *>(cx);
  if (!x) return OCTEN_EINVAL;
  if (!x->initialized) return x->fail(OCTEN_ESTATE, "no factors before octen_n_init");
  const octen_nconfig &c = x->cfg;
  if (A)
    for (int n = 0; n < x->nm; ++n)
      if (A[n])
        cudaMemcpyAsync(A[n], x->A[n], (size_t)x->dims[n] * c.R * 4, cudaMemcpyDefault, x->st);
  if (C) cudaMemcpyAsync(C, x->C, (size_t)x->K * c.R * 4, cudaMemcpyDefault, x->st);
  if (K_out) *K_out = x->K;
  return x->sync_check("get_factors");
}

octen_status octen_n_get_replicas(const octen_nctx *cx, float *Y) {
  octen_nctx *x = const_cast<octen_nctx *>(cx);
  if (!x || !Y) return OCTEN_EINVAL;
  size_t n = (size_t)x->cfg.P;
  for (int m = 0; m < x->NN; ++m) n *= (size_t)x->cfg.Q;
  cudaMemcpyAsync(Y, x->Y, n * 4, cudaMemcpyDefault, x->st);
  return x->sync_check("get_replicas");
}

octen_status octen_n_get_replica_factors(const octen_nctx *cx, int which, float *const *F,
                                         int32_t *perm, double *scales) {
  octen_nctx *x = const_cast<octen_nctx *>(cx);
  if (!x || (which != 0 && which != 1)) return OCTEN_EINVAL;
  const octen_nconfig &c = x->cfg;
  if (F)
    for (int n = 0; n <= x->nm; ++n) {
      if (!F[n]) continue;
      cudaMemcpy2DAsync(F[n], c.R * 4, which ? x->Fh[n] : x->Ft[n], x->RT * 4, c.R * 4,
                        (size_t)c.P * c.Q, cudaMemcpyDefault, x->st);
    }
  if (perm) cudaMemcpyAsync(perm, x->perm, (size_t)c.P * c.R * 4, cudaMemcpyDefault, x->st);
  if (scales)
    cudaMemcpyAsync(scales, x->scales, (size_t)c.P * x->nm * c.R * 8, cudaMemcpyDefault, x->st);
  return x->sync_check("get_replica_factors");
}

int64_t octen_n_rows(const octen_nctx *x) { return x ? x->K : 0; }

}  // extern "C"

namespace {

// Device arrays that make up the state of an initialised N-mode context, in
// file order: per non-temporal mode the rounded projection, its replica
// transpose, its lift operator and the factor; the summaries, G_p and C.
struct NStateArray {
  void *p;
  size_t bytes;
};

std::vector<NStateArray> nstate_arrays(octen_nctx *x) {
  const octen_nconfig &c = x->cfg;
  const size_t P = c.P, Q = c.Q, Qd = x->Qd;
  std::vector<NStateArray> v;
  for (int n = 0; n < x->nm; ++n) {
    const size_t I = (size_t)x->dims[n];
    v.push_back({x->U32[n], I * Qd * 4});
    v.push_back({x->Ut[n], P * Q * I * 4});
    v.push_back({x->L[n], I * Qd * 4});
    v.push_back({x->A[n], I * c.R * 4});
  }
  if (x->Ut16)
    v.push_back({x->Ut16, P * Q * (size_t)x->dims[x->nm - 1] * sizeof(__nv_bfloat16)});
  size_t qn = 1;
  for (int n = 0; n < x->NN; ++n) qn *= Q;
  v.push_back({x->Y, P * qn * 4});
  v.push_back({x->G, P * Q * c.R * 4});
  v.push_back({x->C, (size_t)x->K * c.R * 4});
  return v;
}

const char kNMagic[8] = {'O', 'C', 'T', 'E', 'N', 'N', 'M', '1'};

}  // namespace

extern "C" {

octen_status octen_n_save(const octen_nctx *cx, const char *path) {
  octen_nctx *x = const_cast<octen_nctx *>(cx);
  if (!x || !path) return OCTEN_EINVAL;
  if (!x->initialized) return x->fail(OCTEN_ESTATE, "octen_n_save before octen_n_init");
  if (x->sync_check("save") != OCTEN_OK) return OCTEN_ECUDA;
  FILE *f = fopen(path, "wb");
  if (!f) return x->fail(OCTEN_EINVAL, "octen_n_save: cannot open %s", path);
  int64_t hdr[2 + kMaxNModes] = {x->K, 0};
  for (int n = 0; n < x->nm; ++n) hdr[2 + n] = x->over[n];
  bool ok = fwrite(kNMagic, 1, 8, f) == 8 && fwrite(&x->cfg, sizeof x->cfg, 1, f) == 1 &&
            fwrite(hdr, sizeof hdr, 1, f) == 1;
  std::vector<char> host;
  for (const NStateArray &a : nstate_arrays(x)) {
    if (!ok) break;
    host.resize(a.bytes);
    ok = cudaMemcpy(host.data(), a.p, a.bytes, cudaMemcpyDeviceToHost) == cudaSuccess &&
         fwrite(host.data(), 1, a.bytes, f) == a.bytes;
  }
  ok = (fclose(f) == 0) && ok;
  return ok ? OCTEN_OK : x->fail(OCTEN_ECUDA, "octen_n_save: writing %s failed", path);
}

octen_status octen_n_load(const char *path, void *cuda_stream, octen_nctx **out) {
  if (!path || !out) return OCTEN_EINVAL;
  FILE *f = fopen(path, "rb");
  if (!f) return OCTEN_EINVAL;
  char magic[8];
  octen_nconfig cfg{};
  int64_t hdr[2 + kMaxNModes];
  if (fread(magic, 1, 8, f) != 8 || memcmp(magic, kNMagic, 8) != 0 ||
      fread(&cfg, sizeof cfg, 1, f) != 1 || fread(hdr, sizeof hdr, 1, f) != 1 || hdr[0] < 1 ||
      hdr[0] > kCRowsMax) {
    fclose(f);
    return OCTEN_EINVAL;
  }
  octen_nctx *x = nullptr;
  octen_status s = octen_n_create(&cfg, cuda_stream, &x);
  if (s != OCTEN_OK) {
    fclose(f);
    return s;
  }
  // the lift operators' layouts follow from the shapes
  for (int n = 0; n < x->nm; ++n) {
    if (hdr[2 + n] != (x->Qd > x->dims[n] ? 1 : 0)) {
      fclose(f);
      delete x;
      return OCTEN_EINVAL;
    }
  }
  if (!x->ensure_c(hdr[0])) {
    fclose(f);
    delete x;
    return OCTEN_ENOMEM;
  }
  x->K = hdr[0];
  for (int n = 0; n < x->nm; ++n) x->over[n] = (int)hdr[2 + n];
  bool ok = true;
  std::vector<char> host;
  for (const NStateArray &a : nstate_arrays(x)) {
    host.resize(a.bytes);
    ok = fread(host.data(), 1, a.bytes, f) == a.bytes &&
         cudaMemcpy(a.p, host.data(), a.bytes, cudaMemcpyHostToDevice) == cudaSuccess;
    if (!ok) break;
  }
  fclose(f);
  if (!ok) {
    delete x;
    return OCTEN_EINVAL;
  }
  x->initialized = true;
  *out = x;
  return OCTEN_OK;
}

octen_status octen_n_fit(octen_nctx *x, const void *X_all, int64_t K, double *fit_out) {
  if (!x || !X_all || !fit_out) return OCTEN_EINVAL;
  if (!x->initialized) return x->fail(OCTEN_ESTATE, "octen_n_fit before octen_n_init");
  if (K != x->K)
    return x->fail(OCTEN_EINVAL, "octen_n_fit: K=%lld, rows=%lld", (long long)K, (long long)x->K);
  const int nb = n_fit_blocks(x->slice);
  const bool dev = is_device_pointer(X_all);
  // host slices are staged chunk by chunk; device slices are taken in chunks
  // of at most kFitSlicesMax
  const int64_t chunk = dev ? (K < kFitSlicesMax ? K : kFitSlicesMax) : 16;
  double *part = nullptr;
  if (cudaMalloc(&part, (size_t)chunk * nb * 2 * sizeof(double)) != cudaSuccess) {
    cudaGetLastError();
    return x->fail(OCTEN_ENOMEM, "fit scratch");
  }
  std::vector<double> h((size_t)chunk * nb * 2);
  double t0 = 0.0, t1 = 0.0;
  octen_status s = OCTEN_OK;
  for (int64_t k0 = 0; k0 < K && s == OCTEN_OK; k0 += chunk) {
    const int64_t n = K - k0 < chunk ? K - k0 : chunk;
    const void *Xd = dev ? x->slice_at(X_all, k0)
                         : x->stage_in(x->slice_at(X_all, k0), n * x->slice_bytes(), 0);
    if (!Xd) {
      s = x->fail(OCTEN_ENOMEM, "staging X_all");
      break;
    }
    n_fit_sums(Xd, x->xin, n, x->A, x->C + k0 * x->cfg.R, x->dims, x->nm, x->cfg.R, part,
               x->st);
    cudaMemcpyAsync(h.data(), part, (size_t)n * nb * 2 * sizeof(double), cudaMemcpyDeviceToHost,
                    x->st);
    s = x->sync_check("fit");
    for (int64_t i = 0; i < n * nb && s == OCTEN_OK; ++i) {
      t0 += h[2 * i];
      t1 += h[2 * i + 1];
    }
  }
  cudaFree(part);
  if (s != OCTEN_OK) return s;
  *fit_out = t0 > 0.0 ? 1.0 - sqrt(t1) / sqrt(t0) : 0.0;
  return OCTEN_OK;
}

int octen_n_stage_count(void) { return kNStages; }

const char *octen_n_stage_name(int i) { return i >= 0 && i < kNStages ? kNStageNames[i] : ""; }

octen_status octen_n_set_timing(octen_nctx *x, int on) {
  if (!x) return OCTEN_EINVAL;
  x->timing = on != 0;
  return OCTEN_OK;
}

octen_status octen_n_stage_times(const octen_nctx *cx, double *ms, uint64_t *launches) {
  octen_nctx *x = const_cast<octen_nctx *>(cx);
  if (!x) return OCTEN_EINVAL;
  for (int i = 0; i < kNStages; ++i) {
    if (ms) ms[i] = x->stage_ms[i];
    if (launches) launches[i] = x->stage_n[i];
  }
  return OCTEN_OK;
}

void octen_n_destroy(octen_nctx *x) { delete x; }

const char *octen_n_last_error(const octen_nctx *x) {
  if (!x) return "NULL context";
  return x->err.c_str();
}

}  // extern "C"
