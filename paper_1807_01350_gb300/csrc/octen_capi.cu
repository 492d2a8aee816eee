// C ABI of the library (include/octen.h): the context, its device state, and
// the order of the stages of one online update (the loop body of the paper's
// Algorithm 1: compress, X_p = Y_p + Z_p, CP of every replica, factor match,
// lift of A, B and the new rows of C).
#include <algorithm>
#include <atomic>
#include <cstdarg>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "octen_internal.cuh"

using namespace octen;

namespace octen {
static std::atomic<uint64_t> g_launches{0};
static std::atomic<uint64_t> g_tc_launches{0};
static std::atomic<uint64_t> g_tc_fallbacks{0};
void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
void count_tc_launch() { g_tc_launches.fetch_add(1, std::memory_order_relaxed); }
// A tensor-core contraction that was wanted (bf16 / e4m3 operands on sm_103)
// but refused (an operand pitch off the TMA rules, a resource limit): the
// SIMT kernels run instead.  Counted, and reported once per process on stderr
// so that a slow path does not pass unnoticed.
void count_tc_fallback(const char *what) {
  if (g_tc_fallbacks.fetch_add(1, std::memory_order_relaxed) == 0)
    fprintf(stderr,
            "octen: a tensor-core launch (%s) was refused; the SIMT kernels run instead "
            "(octen_tc_fallback_count() counts these)\n",
            what);
}
bool is_device_pointer(const void *p) {
  if (p == nullptr) return false;
  cudaPointerAttributes a{};
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}
// launches recorded into a graph are counted when the graph runs, not when
// captured; the autotuner's timing launches are not counted
void adjust_launch_counts(int64_t n, int64_t ntc) {
  g_launches.fetch_add(static_cast<uint64_t>(n), std::memory_order_relaxed);
  g_tc_launches.fetch_add(static_cast<uint64_t>(ntc), std::memory_order_relaxed);
}
}  // namespace octen

namespace {

// Device buffer owned by a context (freed in the destructor).
struct DevBuf {
  void *p = nullptr;
  size_t bytes = 0;
};

bool is_device_ptr(const void *p) { return is_device_pointer(p); }

int round_rt(int R) { return R <= 8 ? 8 : (R <= 16 ? 16 : 32); }

}  // namespace

struct octen_ctx {
  octen_config cfg{};
  int Qd = 0, RT = 8;
  Elem xin = Elem::F32;    // slice element type at the boundary
  Elem tu = Elem::F32;     // U rounding / mode-1 operand type
  Elem tv = Elem::F32;     // V rounding / mode-2 operand type
  Elem tmid = Elem::F32;   // mode-2 output (T_rep) type
  cudaStream_t st = nullptr;
  bool initialized = false;
  bool use_tc = true;      // tcgen05 contractions for bf16 / e4m3 operands
  std::string err;
  int64_t K = 0, Kcap = 0;
  int a_over = 0, b_over = 0;
  std::vector<DevBuf> owned;

  // persistent state
  float *U32 = nullptr, *V32 = nullptr;   // rounded projections [rows][Qd]
  void *Ut_rep = nullptr, *Vt = nullptr;  // contraction operands
  float *La = nullptr, *Lb = nullptr;     // lift operators
  float *Y = nullptr, *A = nullptr, *B = nullptr, *C = nullptr, *G = nullptr;
  float *PA = nullptr, *PB = nullptr, *e = nullptr;
  float *At = nullptr, *Bt = nullptr, *Ct = nullptr, *Ah = nullptr, *Bh = nullptr, *Ch = nullptr;
  float *M = nullptr, *H = nullptr, *csolve = nullptr;
  float *GA = nullptr, *GB = nullptr, *GC = nullptr;
  float *splitk = nullptr;                 // split-K partials of the small GEMMs
  // the B-side halves of the warm start and the lift run on als_side beside
  // the A-side halves, with their own split-K and right-hand-side scratch
  float *splitk2 = nullptr, *e2 = nullptr;
  cudaEvent_t pair_fork = nullptr, pair_join = nullptr;
  static constexpr size_t kSplitkFloats = size_t(4) << 20;
  // tensor-core ALS (bf16 / e4m3 modes with Q % 8 == 0, or Q >= 32 zero-padded
  // to als_qp, the next multiple of 8, with factors Apad, Bpad, Cpad)
  bool als_tc = false;
  int als_ks = 1;
  int als_qp = 0;
  float *Apad = nullptr, *Bpad = nullptr, *Cpad = nullptr;
  // CTAs of the replica-ALS GEMMs (0: one per SM).  octen_append_many gives
  // each of its contexts a share of the SMs, so that the GEMMs of several
  // contexts run side by side instead of one after another.
  int als_ctas = 0;
  __nv_bfloat16 *Xa = nullptr, *Xc = nullptr, *KR = nullptr, *Ctb = nullptr, *Btb = nullptr;
  float *Mparts = nullptr;
  // replica CP-ALS: the factor of each update runs on als_side beside its MTTKRP
  cudaStream_t als_side = nullptr;
  cudaEvent_t als_fork = nullptr, als_join = nullptr;
  // replica groups of the tensor-core CP-ALS (see AlsBuffers::groups): group
  // g > 0 runs on grp_st[g] with its factor kernels on grp_side[g]
  int als_groups = 1;
  cudaStream_t grp_st[kMaxAlsGroups] = {}, grp_side[kMaxAlsGroups] = {};
  cudaEvent_t grp_fork[kMaxAlsGroups] = {}, grp_join[kMaxAlsGroups] = {};
  cudaEvent_t grp_split = nullptr, grp_done[kMaxAlsGroups] = {}, grp_first[kMaxAlsGroups] = {};
  float *Lfac = nullptr;
  bool layouts_ready = false;   // Xa / Xc hold bf16(Y) from the last mode-3 pass
  int *perm = nullptr;
  double *scales = nullptr, *align_scratch = nullptr;
  int *dstatus = nullptr;
  double *dfit = nullptr;

  // Everything of an append after its mode-2 contraction (mode 1, mode 3, the
  // warm start, the replica CP-ALS, the match, the lift, the new rows of C and
  // the G_p update: about 200 launches on fixed buffers) runs as one CUDA
  // graph, recorded on a private stream per batch size (the first append runs
  // eagerly, so that the GEMM autotuner has timed its shapes) and replayed on
  // the context's stream.  The batch's W rows reach it through Wfix and the
  // new C rows leave it through Cnew_fix.  A graph is valid for the scratch
  // buffers it was recorded with: any reallocation bumps `gen` and drops the
  // graphs.  OCTEN_GRAPH=0 keeps the launches eager.
  struct TailGraph {
    int64_t t = 0;
    cudaGraph_t graph = nullptr;     // kept: octen_append_many's step graph clones it
    cudaGraphExec_t exec = nullptr;
    int64_t launches = 0, tc = 0;
  };
  static constexpr int kTailGraphs = 4;     // batch sizes kept at once
  static constexpr int kMaxCaptures = 16;   // recordings per generation of buffers
  bool use_graph = true;
  cudaStream_t cap_st = nullptr;
  TailGraph tails[kTailGraphs];
  int next_tail = 0, captures = 0;
  uint64_t gen = 0;                 // bumped whenever a scratch buffer is reallocated
  float *Wfix = nullptr;            // chunk_slices x Qd: the batch's W rows
  float *Cnew_fix = nullptr;        // chunk_slices x R: the batch's new C rows
  int64_t appends = 0;              // appends enqueued so far

  void drop_graphs() {
    for (TailGraph &g : tails) {
      if (g.exec) cudaGraphExecDestroy(g.exec);
      if (g.graph) cudaGraphDestroy(g.graph);
      g = TailGraph{};
    }
    captures = 0;
  }

  // One step of octen_append_many led by this context (the first of the
  // call) as one graph: per context a child graph with its head (W rows into
  // Wfix, quantisation, mode 2), a clone of its tail graph and the copy of
  // the new C rows.  The graph is built for the contexts' ids, buffer
  // generations and batch sizes; later steps with the same key only update
  // the heads (new slices) and the C copies (new row offsets).
  struct StepGraph {
    std::vector<int64_t> key;
    cudaGraph_t graph = nullptr;     // kept: its nodes name the ones updated per step
    cudaGraphExec_t exec = nullptr;
    std::vector<cudaGraphNode_t> head, cmem;
    int64_t launches = 0, tc = 0;   // kernels of the tails, counted per launch
  } step;
  uint64_t id = 0;                  // unique per context in the process
  cudaEvent_t step_ev = nullptr;    // this context's stream reached the step
  cudaEvent_t step_done = nullptr;  // the step graph this context led has run
  void drop_step() {
    if (step.exec) cudaGraphExecDestroy(step.exec);
    if (step.graph) cudaGraphDestroy(step.graph);
    step = StepGraph{};
  }

  // per-batch scratch, grown on demand
  DevBuf Tbuf, T2buf, Wbuf, X8buf, xscale, stage[4], fitpart;

  // host slices of an append are copied in chunks on copy_st, so that the
  // mode-2 contraction of one chunk runs while the next is in flight.  Two
  // staging slots are used in turn, each free again once the mode-2
  // contraction of the append that filled it has run (xslot_free), so that
  // the copy of a batch need not wait for the rest of the previous append.
  static constexpr int kCopyChunks = 8;
  cudaStream_t copy_st = nullptr;
  cudaEvent_t copy_ev[kCopyChunks] = {}, copy_ready = nullptr;
  DevBuf xstage[2];
  cudaEvent_t xslot_free[2] = {};
  int xslot = 0;

  // appends enqueued without waiting (octen_append_async / octen_wait): a
  // ring of tickets, each with the event recorded after its append and the
  // device status word copied to pinned host memory just before it
  static constexpr int kTickets = 8;
  cudaEvent_t ticket_ev[kTickets] = {};
  int *ticket_status = nullptr;              // pinned, kTickets
  int64_t next_ticket = 0, done_ticket = 0;  // issued; known complete

  // stage timers (CUDA events on the context's stream)
  bool timing = false;
  std::vector<cudaEvent_t> evpool;
  size_t evused = 0;
  cudaEvent_t open_ev[kNumStages] = {};
  struct Pending { int stage; cudaEvent_t a, b; };
  std::vector<Pending> pending;
  double stage_ms[kNumStages] = {};
  uint64_t stage_n[kNumStages] = {};

  cudaEvent_t next_event() {
    if (evused == evpool.size()) {
      cudaEvent_t e;
      if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
      evpool.push_back(e);
    }
    return evpool[evused++];
  }
  void mark(int stage, int begin) {
    if (!timing) return;
    cudaEvent_t e = next_event();
    if (!e) return;
    cudaEventRecord(e, st);
    if (begin) open_ev[stage] = e;
    else if (open_ev[stage]) pending.push_back({stage, open_ev[stage], e});
  }
  static void mark_cb(void *self, int stage, int begin) {
    static_cast<octen_ctx *>(self)->mark(stage, begin);
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

  ~octen_ctx() {
    cudaStreamSynchronize(st);
    drop_graphs();
    drop_step();
    if (step_ev) cudaEventDestroy(step_ev);
    if (step_done) cudaEventDestroy(step_done);
    if (cap_st) cudaStreamDestroy(cap_st);
    if (als_side) {
      cudaStreamSynchronize(als_side);
      cudaStreamDestroy(als_side);
    }
    if (als_fork) cudaEventDestroy(als_fork);
    if (als_join) cudaEventDestroy(als_join);
    if (pair_fork) cudaEventDestroy(pair_fork);
    if (pair_join) cudaEventDestroy(pair_join);
    for (int g = 0; g < kMaxAlsGroups; ++g) {
      for (cudaStream_t s2 : {grp_st[g], grp_side[g]})
        if (s2) {
          cudaStreamSynchronize(s2);
          cudaStreamDestroy(s2);
        }
      for (cudaEvent_t e : {grp_fork[g], grp_join[g], grp_done[g], grp_first[g]})
        if (e) cudaEventDestroy(e);
    }
    if (grp_split) cudaEventDestroy(grp_split);
    for (cudaEvent_t e : evpool) cudaEventDestroy(e);
    if (copy_st) {
      cudaStreamSynchronize(copy_st);
      cudaStreamDestroy(copy_st);
    }
    for (cudaEvent_t e : copy_ev)
      if (e) cudaEventDestroy(e);
    if (copy_ready) cudaEventDestroy(copy_ready);
    for (auto &b : owned) cudaFree(b.p);
    for (auto &r : retired) cudaFree(r.first);
    DevBuf *extra[] = {&Tbuf, &T2buf, &Wbuf, &X8buf, &xscale, &stage[0], &stage[1], &stage[2],
                       &stage[3], &fitpart, &xstage[0], &xstage[1]};
    for (DevBuf *b : extra) cudaFree(b->p);
    for (cudaEvent_t e : xslot_free)
      if (e) cudaEventDestroy(e);
    for (cudaEvent_t e : ticket_ev)
      if (e) cudaEventDestroy(e);
    if (ticket_status) cudaFreeHost(ticket_status);
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

  // Device memory the context holds (its state and scratch buffers), and the
  // most it may hold: OCTEN_DEVICE_MEMORY_LIMIT bytes when that is set at
  // create, else unbounded.  An allocation past the limit fails like a
  // refused cudaMalloc (ENOMEM).
  size_t held = 0;
  size_t limit = SIZE_MAX;

  bool dev_malloc(void **p, size_t bytes) {
    *p = nullptr;
    if (bytes > limit || held > limit - bytes) return false;
    if (cudaMalloc(p, bytes) != cudaSuccess) {
      cudaGetLastError();
      *p = nullptr;
      return false;
    }
    held += bytes;
    return true;
  }
  void dev_free(void *p, size_t bytes) {
    if (!p) return;
    cudaFree(p);
    held -= bytes;
  }
  // Buffers replaced while enqueued work may still read them (the old C after
  // it grows): held until the context's streams are next known to be idle,
  // then freed (cudaFree would wait for the device).
  std::vector<std::pair<void *, size_t>> retired;
  void free_retired() {
    for (auto &r : retired) dev_free(r.first, r.second);
    retired.clear();
  }

  template <class T>
  bool alloc(T *&ptr, size_t count) {
    void *p = nullptr;
    if (!dev_malloc(&p, count * sizeof(T) + 16)) return false;
    owned.push_back({p, count * sizeof(T) + 16});
    ptr = static_cast<T *>(p);
    return true;
  }

  // Scratch of at least `bytes` in b; a refused allocation (device or limit)
  // is detected before the smaller buffer is released.
  bool grow(DevBuf &b, size_t bytes) {
    if (b.bytes >= bytes) return true;
    const size_t old = b.p ? b.bytes + 16 : 0;
    const size_t want = bytes + 16;
    if (want > limit || held - old > limit - want) return false;
    cudaStreamSynchronize(st);
    if (b.p) {
      drop_graphs();   // recorded with the old address
      ++gen;
    }
    dev_free(b.p, old);
    b.p = nullptr;
    b.bytes = 0;
    if (!dev_malloc(&b.p, want)) return false;
    b.bytes = bytes;
    return true;
  }

  // Device view of a caller buffer: the pointer itself if it is device
  // memory, else a copy in staging slot `slot`.
  const void *stage_in(const void *p, size_t bytes, int slot) {
    if (is_device_ptr(p)) return p;
    if (!grow(stage[slot], bytes)) return nullptr;
    if (cudaMemcpyAsync(stage[slot].p, p, bytes, cudaMemcpyHostToDevice, st) != cudaSuccess)
      return nullptr;
    return stage[slot].p;
  }

  octen_status sync_check(const char *what) {
    cudaError_t e = cudaStreamSynchronize(st);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e == cudaSuccess) free_retired();
    if (e == cudaSuccess && !pending.empty()) flush_timers();
    if (e != cudaSuccess) return fail(OCTEN_ECUDA, "%s: %s", what, cudaGetErrorString(e));
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
};

namespace octen {

octen_status validate_config(const octen_config *c, std::string &why) {
  char buf[256];
  if (!c) { why = "config is NULL"; return OCTEN_EINVAL; }
  if (c->I < 1 || c->J < 1 || c->R < 1 || c->R > 32 || c->P < 1 || c->P > kGridYZMax ||
      c->Q < 2 || c->Q > 256 || c->S < 1 || c->S >= c->Q || c->als_iters < 1 || c->prec < 0 ||
      c->prec > 2) {
    snprintf(buf, sizeof buf,
             "unsupported config I=%lld J=%lld R=%d P=%d Q=%d S=%d iters=%d prec=%d (limits: "
             "1<=R<=32, 1<=S<Q<=256, 1<=P<=65535, iters>=1)",
             (long long)c->I, (long long)c->J, c->R, c->P, c->Q, c->S, c->als_iters, c->prec);
    why = buf;
    return OCTEN_EINVAL;
  }
  const int64_t Qd = (int64_t)c->S + (int64_t)c->P * (c->Q - c->S);
  if (Qd > (1 << 20) || c->I > (1 << 24) || c->J > (1 << 24)) {
    why = "dimensions too large";
    return OCTEN_EINVAL;
  }
  return OCTEN_OK;
}

}  // namespace octen

namespace {

// OCTEN_DEVICE_MEMORY_LIMIT: bytes of device memory a context created now may
// hold (unset, empty or not a number: no limit).
size_t device_memory_limit() {
  const char *v = getenv("OCTEN_DEVICE_MEMORY_LIMIT");
  if (!v || !*v) return SIZE_MAX;
  char *end = nullptr;
  const unsigned long long n = strtoull(v, &end, 10);
  return end == v ? SIZE_MAX : (size_t)n;
}

// Replica groups of the tensor-core CP-ALS: OCTEN_ALS_GROUPS (1 to
// kMaxAlsGroups, at most P), else 1.
int als_groups_wanted(int P) {
  int g = 1;
  const char *v = getenv("OCTEN_ALS_GROUPS");
  if (v && *v) g = atoi(v);
  if (g < 1) g = 1;
  if (g > kMaxAlsGroups) g = kMaxAlsGroups;
  return g > P ? P : g;
}

// The replica CP-ALS chain as programmatic dependent launches: OCTEN_PDL=1
// (off by default: at 4000^2 it measured 1435 against 1642 slices/s, the
// early-launched kernels waiting resident on the SMs beside the running ones).
bool pdl_wanted() {
  const char *v = getenv("OCTEN_PDL");
  return v && v[0] == '1';
}

// OCTEN_GEMM=simt keeps the large contractions on the SIMT kernels (used to
// cross-check the tensor-core kernels against an independent implementation).
bool tc_wanted() {
  const char *v = getenv("OCTEN_GEMM");
  return !(v && strcmp(v, "simt") == 0) && tc_supported();
}

void set_types(octen_ctx *x) {
  x->use_tc = x->cfg.prec != OCTEN_FP32 && tc_wanted();
  const char *g = getenv("OCTEN_GRAPH");
  x->use_graph = !(g && strcmp(g, "0") == 0);
  switch (x->cfg.prec) {
    case OCTEN_FP32:
      x->xin = Elem::F32; x->tu = Elem::F32; x->tv = Elem::F32; x->tmid = Elem::F32; break;
    case OCTEN_BF16:
      x->xin = Elem::BF16; x->tu = Elem::BF16; x->tv = Elem::BF16; x->tmid = Elem::BF16; break;
    default:
      x->xin = Elem::BF16; x->tu = Elem::BF16; x->tv = Elem::E4M3; x->tmid = Elem::BF16; break;
  }
}

constexpr int64_t kChunk = 64;  // slices per compression pass

// Slices per compression pass for this context: kChunk, fewer when the
// batched mode-1 contraction (one product per slice and replica, the batch a
// grid dimension) would exceed kGridYZMax products.
int64_t chunk_slices(const octen_ctx *x) {
  const int64_t m = kGridYZMax / x->cfg.P;
  return m < kChunk ? m : kChunk;
}

// Scratch of one compression pass of t slices.
octen_status compress_scratch(octen_ctx *x, int64_t t) {
  const octen_config &c = x->cfg;
  const size_t tb = (size_t)t * c.P * c.Q * c.I * elem_size(x->tmid);
  if (!x->grow(x->Tbuf, tb)) return x->fail(OCTEN_ENOMEM, "scratch T (%zu bytes)", tb);
  const size_t t2b = (size_t)t * c.P * c.Q * c.Q * sizeof(float);
  if (!x->grow(x->T2buf, t2b)) return x->fail(OCTEN_ENOMEM, "scratch T2 (%zu bytes)", t2b);
  if (c.prec == OCTEN_FP8E4M3) {
    const size_t xb = (size_t)t * c.I * c.J;
    if (!x->grow(x->X8buf, xb) || !x->grow(x->xscale, (size_t)t * sizeof(float)))
      return x->fail(OCTEN_ENOMEM, "scratch for e4m3 slices");
  }
  return OCTEN_OK;
}

// Quantisation (fp8) and mode-2 contraction of slices [k0, k0 + n) of a pass
// whose slices start at Xd (device).
void compress_mode2(octen_ctx *x, const void *Xd, int64_t k0, int64_t n) {
  const octen_config &c = x->cfg;
  const size_t slice = (size_t)c.I * c.J * elem_size(x->xin);
  Mode2Args m2{};
  m2.X = static_cast<const char *>(Xd) + k0 * slice; m2.tx = x->xin; m2.Vt = x->Vt;
  m2.tv = x->tv; m2.slice_scale = nullptr;
  m2.T = static_cast<char *>(x->Tbuf.p) + (size_t)k0 * c.P * c.Q * c.I * elem_size(x->tmid);
  m2.tt = x->tmid; m2.t = n; m2.I = c.I; m2.J = c.J;
  m2.P = c.P; m2.Q = c.Q; m2.S = c.S; m2.Qd = x->Qd;
  if (c.prec == OCTEN_FP8E4M3) {
    const int64_t IJ = c.I * c.J;
    __nv_fp8_e4m3 *x8 = static_cast<__nv_fp8_e4m3 *>(x->X8buf.p) + k0 * IJ;
    float *sc = static_cast<float *>(x->xscale.p) + k0;
    x->mark(kStQuant, 1);
    quantize_e4m3(static_cast<const __nv_bfloat16 *>(m2.X), n, IJ, x8, sc, x->st);
    x->mark(kStQuant, 0);
    m2.X = x8; m2.tx = Elem::E4M3; m2.slice_scale = sc;
  }
  x->mark(kStMode2, 1);
  if (!(x->use_tc && mode2_tc(m2, x->dstatus, x->st))) {
    cudaGetLastError();
    if (x->use_tc) count_tc_fallback("mode-2 contraction");
    mode2_simt(m2, x->st);
  }
  x->mark(kStMode2, 0);
}

// Mode-1 and mode-3 contractions of a pass of t slices (after its mode 2):
// Z_p (+)= into Yacc.  With `layouts` the mode-3 pass may also leave the bf16
// copies of Yacc for the tensor-core CP-ALS in x->Xa / x->Xc
// (x->layouts_ready says whether it did).
void compress_finish(octen_ctx *x, int64_t t, const float *Wd, float *Yacc, bool layouts) {
  const octen_config &c = x->cfg;
  Mode1Args m1{};
  m1.Ut = x->Ut_rep; m1.T = x->Tbuf.p; m1.te = x->tmid; m1.T2 = static_cast<float *>(x->T2buf.p);
  m1.t = t; m1.I = c.I; m1.P = c.P; m1.Q = c.Q;
  x->mark(kStMode1, 1);
  if (!(x->use_tc && mode1_tc(m1, x->dstatus, x->st))) {
    cudaGetLastError();
    if (x->use_tc) count_tc_fallback("mode-1 contraction");
    mode1_simt(m1, x->st);
  }
  x->mark(kStMode1, 0);
  x->mark(kStMode3, 1);
  // (the padded ALS builds its own zero-padded copies)
  const bool want = layouts && x->als_tc && x->als_qp == 0;
  x->layouts_ready =
      mode3_accumulate(static_cast<float *>(x->T2buf.p), Wd, Yacc, t, c.P, c.Q, c.S, x->Qd, x->st,
                       want ? x->Xa : nullptr, want ? x->Xc : nullptr);
  x->mark(kStMode3, 0);
}

// Z_p (+)= compression of t slices (t <= chunk_slices(x), device) into Yacc.
octen_status compress_chunk(octen_ctx *x, const void *Xd, int64_t t, const float *Wd,
                            float *Yacc, bool layouts = false) {
  octen_status s = compress_scratch(x, t);
  if (s != OCTEN_OK) return s;
  compress_mode2(x, Xd, 0, t);
  compress_finish(x, t, Wd, Yacc, layouts);
  return OCTEN_OK;
}

// Quantisation and mode-2 contraction of t host slices: they are copied into
// staging slot 2 (already sized by the caller) in up to `pieces` pieces on
// copy_st, and the contraction of each piece starts as soon as it has arrived
// (one piece: one contraction of the whole batch once it has all arrived).
// The caller ensures 16-byte aligned piece offsets (I J a multiple of 16),
// which the tensor-map operands need.
octen_status compress_mode2_host(octen_ctx *x, const void *Xh, int64_t t, int pieces) {
  const octen_config &c = x->cfg;
  const size_t slice = (size_t)c.I * c.J * elem_size(x->xin);
  // the slot is free once the mode-2 contraction of its previous batch has run
  DevBuf &stg = x->xstage[x->xslot];
  cudaStreamWaitEvent(x->copy_st, x->xslot_free[x->xslot], 0);
  const int np = pieces < 1 ? 1 : (pieces > octen_ctx::kCopyChunks ? octen_ctx::kCopyChunks : pieces);
  const int64_t per = (t + np - 1) / np;
  const int64_t step = per < 2 ? 2 : per;
  int nc = 0;
  for (int64_t k0 = 0; k0 < t; k0 += step, ++nc) {
    const int64_t n = t - k0 < step ? t - k0 : step;
    if (cudaMemcpyAsync(static_cast<char *>(stg.p) + k0 * slice,
                        static_cast<const char *>(Xh) + k0 * slice, n * slice,
                        cudaMemcpyHostToDevice, x->copy_st) != cudaSuccess) {
      cudaStreamSynchronize(x->copy_st);   // no copy of the caller's buffer stays in flight
      return x->fail(OCTEN_ECUDA, "copying the batch");
    }
    cudaEventRecord(x->copy_ev[nc], x->copy_st);
  }
  nc = 0;
  for (int64_t k0 = 0; k0 < t; k0 += step, ++nc) {
    const int64_t n = t - k0 < step ? t - k0 : step;
    cudaStreamWaitEvent(x->st, x->copy_ev[nc], 0);
    compress_mode2(x, stg.p, k0, n);
  }
  cudaEventRecord(x->xslot_free[x->xslot], x->st);
  x->xslot ^= 1;
  return OCTEN_OK;
}

octen_status compress_all(octen_ctx *x, const void *Xd, int64_t t, const float *Wd, float *Yacc) {
  const size_t slice = (size_t)x->cfg.I * x->cfg.J * elem_size(x->xin);
  const int64_t ck = chunk_slices(x);
  for (int64_t k0 = 0; k0 < t; k0 += ck) {
    const int64_t n = t - k0 < ck ? t - k0 : ck;
    octen_status s = compress_chunk(x, static_cast<const char *>(Xd) + k0 * slice, n,
                                    Wd + k0 * x->Qd, Yacc);
    if (s != OCTEN_OK) return s;
  }
  return OCTEN_OK;
}

// Lift operator of one mode (Eq. 7 with P^-1 the pseudo-inverse).  With
// Qd > rows the stack has full column rank: L = (U Omega U^T)^-1 U, shape
// rows x Qd (Omega weights the anchor columns by P).  Otherwise the distinct
// rows have full row rank: L = U (U^T U)^-1, stored transposed (Qd x rows).
LiftEnv lift_env(octen_ctx *x, bool side = false) {
  const octen_config &c = x->cfg;
  return LiftEnv{x->Qd, c.P, c.Q, c.S, c.R, x->RT, side ? x->als_side : x->st, x->dstatus,
                 side ? x->e2 : x->e, side ? x->splitk2 : x->splitk, octen_ctx::kSplitkFloats};
}

octen_status build_lift(octen_ctx *x, const float *Ur, int64_t rows, float *L, int &over) {
  if (!lift_build(lift_env(x), Ur, rows, L, over))
    return x->fail(OCTEN_ENOMEM, "lift operator (%lld rows)", (long long)rows);
  return x->sync_check("lift operator");
}

// Delta of one global factor: F += Lift * e (Qd x R rhs built from the
// aligned replica blocks and the projected previous factor PF).
void lift_mode(octen_ctx *x, const float *Fh, const float *PF, const float *L, int over,
               int64_t rows, float *F, bool side) {
  lift_apply(lift_env(x, side), Fh, PF, L, over, rows, F);
}

// The A- and B-side halves of the warm start and of the lift are independent:
// the B side goes to als_side between pair_fork and pair_join.
void pair_fork(octen_ctx *x) {
  cudaEventRecord(x->pair_fork, x->st);
  cudaStreamWaitEvent(x->als_side, x->pair_fork, 0);
}
void pair_join(octen_ctx *x) {
  cudaEventRecord(x->pair_join, x->als_side);
  cudaStreamWaitEvent(x->st, x->pair_join, 0);
}

// PF = U_all^T F (Qd x R) on stream st with split-K scratch splitk
void project(octen_ctx *x, const float *Ur, int64_t rows, const float *F, float *PF,
             cudaStream_t st, float *splitk) {
  const octen_config &c = x->cfg;
  GemmArgs g{};
  g.A = Ur; g.ta = Elem::F32; g.sAm = 1; g.sAk = x->Qd;
  g.B = F; g.tb = Elem::F32; g.sBn = 1; g.sBk = c.R;
  g.D = PF; g.sDm = c.R; g.sDn = 1;
  g.M = x->Qd; g.N = c.R; g.K = (int)rows; g.batch = 1; g.alpha = 1.f; g.beta = 0.f;
  g.split_scratch = splitk; g.split_scratch_floats = octen_ctx::kSplitkFloats;
  gemm_strided(g, st);
}

// Room for `rows` rows of C (capacity doubling from 1024 rows).  Growing
// enqueues the copy of the rows so far on x->st and retires the old buffer
// rather than synchronising: appends already enqueued write their rows into
// the old C before the copy runs, and the next append's rows go to the new one.
bool ensure_c_capacity(octen_ctx *x, int64_t rows) {
  if (rows <= x->Kcap) return true;
  if (rows > kCRowsMax) return false;
  int64_t cap = x->Kcap > 0 ? x->Kcap : 1024;
  while (cap < rows) cap *= 2;
  float *nc = nullptr;
  const size_t bytes = (size_t)cap * x->cfg.R * sizeof(float);
  if (!x->dev_malloc(reinterpret_cast<void **>(&nc), bytes)) return false;
  if (x->C) {
    cudaMemcpyAsync(nc, x->C, (size_t)x->K * x->cfg.R * sizeof(float), cudaMemcpyDeviceToDevice,
                    x->st);
    for (auto &b : x->owned)
      if (b.p == x->C) {
        x->retired.push_back({b.p, b.bytes});
        b.p = nc;
        b.bytes = bytes;
      }
  } else {
    x->owned.push_back({nc, bytes});
  }
  x->C = nc;
  x->Kcap = cap;
  return true;
}

}  // namespace

extern "C" {

octen_status octen_create(const octen_config *cfg, void *cuda_stream, octen_ctx **out) {
  if (!out) return OCTEN_EINVAL;
  std::string why;
  octen_status s = validate_config(cfg, why);
  if (s != OCTEN_OK) {
    fprintf(stderr, "octen_create: %s\n", why.c_str());
    return s;
  }
  octen_ctx *x = new octen_ctx();
  static std::atomic<uint64_t> ids{0};
  x->id = ++ids;
  x->limit = device_memory_limit();
  x->cfg = *cfg;
  x->Qd = cfg->S + cfg->P * (cfg->Q - cfg->S);
  x->RT = round_rt(cfg->R);
  x->st = static_cast<cudaStream_t>(cuda_stream);
  set_types(x);
  const octen_config &c = x->cfg;
  const size_t P = c.P, Q = c.Q, RT = x->RT, Qd = x->Qd;
  bool ok = x->alloc(x->U32, (size_t)c.I * Qd) && x->alloc(x->V32, (size_t)c.J * Qd) &&
            x->alloc(x->La, (size_t)c.I * Qd) && x->alloc(x->Lb, (size_t)c.J * Qd) &&
            x->alloc(x->Y, P * Q * Q * Q) && x->alloc(x->A, (size_t)c.I * c.R) &&
            x->alloc(x->B, (size_t)c.J * c.R) && x->alloc(x->G, P * Q * c.R) &&
            x->alloc(x->PA, Qd * c.R) && x->alloc(x->PB, Qd * c.R) && x->alloc(x->e, Qd * c.R) &&
            x->alloc(x->At, P * Q * RT) && x->alloc(x->Bt, P * Q * RT) &&
            x->alloc(x->Ct, P * Q * RT) && x->alloc(x->Ah, P * Q * RT) &&
            x->alloc(x->Bh, P * Q * RT) && x->alloc(x->Ch, P * Q * RT) &&
            x->alloc(x->M, P * ((Q + 7) / 8 * 8) * RT) && x->alloc(x->H, P * Q * Q * RT) &&
            x->alloc(x->perm, P * c.R) && x->alloc(x->scales, P * 2 * c.R) &&
            x->alloc(x->align_scratch, align_scratch_doubles(c.P, x->RT)) &&
            x->alloc(x->dstatus, 1) && x->alloc(x->dfit, 2) && x->alloc(x->GA, P * RT * RT) &&
            x->alloc(x->GB, P * RT * RT) && x->alloc(x->GC, P * RT * RT) &&
            x->alloc(x->Lfac, P * (size_t)als_factor_floats(x->RT)) &&
            x->alloc(x->splitk, octen_ctx::kSplitkFloats) &&
            x->alloc(x->splitk2, octen_ctx::kSplitkFloats) && x->alloc(x->e2, Qd * c.R) &&
            x->alloc(x->Wfix, (size_t)chunk_slices(x) * Qd) &&
            x->alloc(x->Cnew_fix, (size_t)chunk_slices(x) * c.R);
  if (ok && x->use_tc && als_tc_eligible(c.Q)) {
    // Q not a multiple of 8: the tensor-core passes run on X_p zero-padded to Qp
    const size_t Qp = (Q + 7) / 8 * 8;
    x->als_qp = Qp == Q ? 0 : (int)Qp;
    const int mt = (c.Q + 127) / 128;
    const int want = (4 * 152 + mt * c.P - 1) / (mt * c.P);
    x->als_ks = als_tc_splits(c.P, c.Q, want < 1 ? 1 : want);
    const size_t nparts = (size_t)(x->als_ks > (int)(Qp / 32) ? x->als_ks : (int)(Qp / 32));
    // the Khatri-Rao operand of the M3 pass exists only below Q = 32 (from 32
    // on, the M3 GEMM contracts b against B^T and reduces a in its epilogue)
    ok = x->alloc(x->Xa, P * Qp * Qp * Qp) && x->alloc(x->Xc, P * Qp * Qp * Qp) &&
         (c.Q >= 32 || x->alloc(x->KR, P * kAlsNP * Q * Q)) &&
         x->alloc(x->Ctb, P * kAlsNP * Qp) && x->alloc(x->Btb, P * kAlsNP * Qp) &&
         x->alloc(x->Mparts, std::max(nparts * Qp, 2 * ((Qp * Qp + 31) / 32)) * P * RT) &&
         (Qp == Q || (x->alloc(x->Apad, P * Qp * RT) && x->alloc(x->Bpad, P * Qp * RT) &&
                      x->alloc(x->Cpad, P * Qp * RT)));
    x->als_tc = ok;
  }
  void *ut = nullptr, *vt = nullptr;
  if (ok) {
    const size_t ub = P * Q * c.I * elem_size(x->tu), vb = Qd * c.J * elem_size(x->tv);
    ok = x->dev_malloc(&ut, ub) && x->dev_malloc(&vt, vb);
    if (ut) x->owned.push_back({ut, ub});
    if (vt) x->owned.push_back({vt, vb});
    x->Ut_rep = ut;
    x->Vt = vt;
  }
  if (ok) {
    ok = cudaStreamCreateWithFlags(&x->copy_st, cudaStreamNonBlocking) == cudaSuccess &&
         cudaEventCreateWithFlags(&x->copy_ready, cudaEventDisableTiming) == cudaSuccess;
    for (cudaEvent_t &e : x->copy_ev)
      ok = ok && cudaEventCreateWithFlags(&e, cudaEventDisableTiming) == cudaSuccess;
    for (cudaEvent_t &e : x->xslot_free)
      ok = ok && cudaEventCreateWithFlags(&e, cudaEventDisableTiming) == cudaSuccess;
    for (cudaEvent_t &e : x->ticket_ev)
      ok = ok && cudaEventCreateWithFlags(&e, cudaEventDisableTiming) == cudaSuccess;
    ok = ok && cudaHostAlloc(reinterpret_cast<void **>(&x->ticket_status),
                             octen_ctx::kTickets * sizeof(int), cudaHostAllocDefault) ==
                   cudaSuccess;
  }
  if (ok) {
    ok = cudaStreamCreateWithFlags(&x->als_side, cudaStreamNonBlocking) == cudaSuccess &&
         cudaEventCreateWithFlags(&x->als_fork, cudaEventDisableTiming) == cudaSuccess &&
         cudaEventCreateWithFlags(&x->als_join, cudaEventDisableTiming) == cudaSuccess &&
         cudaEventCreateWithFlags(&x->pair_fork, cudaEventDisableTiming) == cudaSuccess &&
         cudaEventCreateWithFlags(&x->pair_join, cudaEventDisableTiming) == cudaSuccess;
  }
  if (ok && x->als_tc && c.Q >= 32) {
    x->als_groups = als_groups_wanted(c.P);
    if (x->als_groups > 1)
      ok = cudaEventCreateWithFlags(&x->grp_split, cudaEventDisableTiming) == cudaSuccess;
    for (int g = 0; g + 1 < x->als_groups && ok; ++g)
      ok = cudaEventCreateWithFlags(&x->grp_first[g], cudaEventDisableTiming) == cudaSuccess;
    for (int g = 1; g < x->als_groups && ok; ++g) {
      ok = cudaStreamCreateWithFlags(&x->grp_st[g], cudaStreamNonBlocking) == cudaSuccess &&
           cudaStreamCreateWithFlags(&x->grp_side[g], cudaStreamNonBlocking) == cudaSuccess &&
           cudaEventCreateWithFlags(&x->grp_fork[g], cudaEventDisableTiming) == cudaSuccess &&
           cudaEventCreateWithFlags(&x->grp_join[g], cudaEventDisableTiming) == cudaSuccess &&
           cudaEventCreateWithFlags(&x->grp_done[g], cudaEventDisableTiming) == cudaSuccess;
    }
  }
  if (!ok) {
    cudaGetLastError();
    delete x;
    return OCTEN_ENOMEM;
  }
  cudaMemsetAsync(x->Y, 0, P * Q * Q * Q * sizeof(float), x->st);
  cudaMemsetAsync(x->G, 0, P * Q * c.R * sizeof(float), x->st);
  cudaMemsetAsync(x->dstatus, 0, sizeof(int), x->st);
  if (x->sync_check("create") != OCTEN_OK) {
    delete x;
    return OCTEN_ECUDA;
  }
  *out = x;
  return OCTEN_OK;
}

octen_status octen_init(octen_ctx *x, const void *X_old, int64_t t_old, const float *U_all,
                        const float *V_all, const float *W_old, const float *A0,
                        const float *B0, const float *C0) {
  if (!x) return OCTEN_EINVAL;
  if (x->initialized) return x->fail(OCTEN_ESTATE, "octen_init called twice");
  if (!X_old || !U_all || !V_all || !W_old || !A0 || !B0 || t_old < 1)
    return x->fail(OCTEN_EINVAL,
                   "octen_init: X_old, U_all, V_all, W_old, A0, B0 are required and t_old >= 1");
  const bool decompose = C0 == nullptr;   // A0, B0 are starting guesses
  const octen_config &c = x->cfg;
  // the decomposition's per-slice products are a grid dimension, and its
  // (slice, row) GEMM has t_old * I rows
  if (decompose && (t_old > kGridYZMax || t_old * c.I > INT32_MAX))
    return x->fail(OCTEN_EINVAL,
                   "octen_init: decomposing X_old takes t_old <= %lld and t_old * I < 2^31 "
                   "(t_old=%lld, I=%lld)",
                   (long long)kGridYZMax, (long long)t_old, (long long)c.I);
  const int Qd = x->Qd;
  // projections: round once to the operand formats, build the operand layouts
  const float *Ud = static_cast<const float *>(x->stage_in(U_all, (size_t)c.I * Qd * 4, 0));
  if (!Ud) return x->fail(OCTEN_ENOMEM, "staging U");
  round_copy(Ud, x->U32, (int64_t)c.I * Qd, x->tu, x->st);
  const float *Vd = static_cast<const float *>(x->stage_in(V_all, (size_t)c.J * Qd * 4, 0));
  if (!Vd) return x->fail(OCTEN_ENOMEM, "staging V");
  round_copy(Vd, x->V32, (int64_t)c.J * Qd, x->tv, x->st);
  make_replica_transpose(x->U32, c.I, c.P, c.Q, c.S, Qd, x->Ut_rep, x->tu, x->st);
  make_transpose(x->V32, c.J, Qd, x->Vt, x->tv, x->st);
  octen_status s = x->sync_check("projection setup");
  if (s != OCTEN_OK) return s;
  // summaries of the existing tensor, chunk by chunk
  const size_t slice = (size_t)c.I * c.J * elem_size(x->xin);
  const float *Wd = static_cast<const float *>(x->stage_in(W_old, (size_t)t_old * Qd * 4, 1));
  if (!Wd) return x->fail(OCTEN_ENOMEM, "staging W_old");
  if (is_device_ptr(X_old)) {
    s = compress_all(x, X_old, t_old, Wd, x->Y);
    if (s != OCTEN_OK) return s;
  } else {
    const int64_t ck = chunk_slices(x);
    for (int64_t k0 = 0; k0 < t_old; k0 += ck) {
      const int64_t n = t_old - k0 < ck ? t_old - k0 : ck;
      const void *Xd = x->stage_in(static_cast<const char *>(X_old) + k0 * slice, n * slice, 2);
      if (!Xd) return x->fail(OCTEN_ENOMEM, "staging X_old");
      s = compress_chunk(x, Xd, n, Wd + k0 * Qd, x->Y);
      if (s != OCTEN_OK) return s;
      cudaStreamSynchronize(x->st);
    }
  }
  // existing factors (given, or a CP-ALS of X_old from A0, B0) and G_p = W_old,p^T C_old
  if (!ensure_c_capacity(x, t_old)) return x->fail(OCTEN_ENOMEM, "C");
  if (decompose) {
    const void *Xd = x->stage_in(X_old, t_old * slice, 2);
    const float *A0d = static_cast<const float *>(x->stage_in(A0, (size_t)c.I * c.R * 4, 0));
    const float *B0d = static_cast<const float *>(x->stage_in(B0, (size_t)c.J * c.R * 4, 1));
    if (!Xd || !A0d || !B0d) return x->fail(OCTEN_ENOMEM, "staging X_old, A0, B0");
    float *work = nullptr;
    const size_t wf = dense_cp_work_floats(t_old, c.I, c.J, x->RT);
    if (!x->dev_malloc(reinterpret_cast<void **>(&work), wf * sizeof(float)))
      return x->fail(OCTEN_ENOMEM, "dense CP-ALS workspace (%zu bytes)", wf * sizeof(float));
    DenseCpArgs a{};
    a.X = Xd; a.xt = x->xin; a.K = t_old; a.I = c.I; a.J = c.J; a.R = c.R;
    a.iters = c.als_iters; a.A0 = A0d; a.B0 = B0d;
    a.A_out = x->A; a.B_out = x->B; a.C_out = x->C; a.work = work;
    a.splitk = x->splitk; a.splitk_floats = octen_ctx::kSplitkFloats;
    a.status = x->dstatus; a.st = x->st;
    dense_cp(a, x->RT);
    s = x->sync_check("init decomposition");
    x->dev_free(work, wf * sizeof(float));
    if (s != OCTEN_OK) return s;
  } else {
    cudaMemcpyAsync(x->A, A0, (size_t)c.I * c.R * 4, cudaMemcpyDefault, x->st);
    cudaMemcpyAsync(x->B, B0, (size_t)c.J * c.R * 4, cudaMemcpyDefault, x->st);
    cudaMemcpyAsync(x->C, C0, (size_t)t_old * c.R * 4, cudaMemcpyDefault, x->st);
  }
  update_g(Wd, x->C, t_old, c.P, c.Q, c.S, Qd, c.R, x->G, x->st);
  s = x->sync_check("init summaries");
  if (s != OCTEN_OK) return s;
  x->K = t_old;
  s = build_lift(x, x->U32, c.I, x->La, x->a_over);
  if (s != OCTEN_OK) return s;
  s = build_lift(x, x->V32, c.J, x->Lb, x->b_over);
  if (s != OCTEN_OK) return s;
  x->initialized = true;
  return OCTEN_OK;
}

}  // extern "C"

namespace {

// The replica buffers of the CP-ALS of an append.
AlsBuffers als_buffers(octen_ctx *x) {
  AlsBuffers ab;
  ab.Af = x->At; ab.Bf = x->Bt; ab.Cf = x->Ct; ab.GA = x->GA; ab.GB = x->GB; ab.GC = x->GC;
  ab.M = x->M; ab.H = x->H; ab.status = x->dstatus;
  ab.use_tc = x->als_tc; ab.Xa = x->Xa; ab.Xc = x->Xc; ab.KR = x->KR; ab.Ct = x->Ctb;
  ab.Bt = x->Btb;
  ab.Mparts = x->Mparts; ab.ksplit = x->als_ks;
  ab.side = x->als_side; ab.ev_fork = x->als_fork; ab.ev_join = x->als_join; ab.L = x->Lfac;
  ab.layouts_ready = x->layouts_ready;
  ab.groups = x->als_groups;
  for (int g = 0; g < kMaxAlsGroups; ++g) {
    ab.gst[g] = x->grp_st[g]; ab.gside[g] = x->grp_side[g];
    ab.gev_fork[g] = x->grp_fork[g]; ab.gev_join[g] = x->grp_join[g];
    ab.gdone[g] = x->grp_done[g];
    ab.gfirst[g] = x->grp_first[g];
  }
  ab.gsplit = x->grp_split;
  ab.Qp = x->als_qp;
  ab.max_ctas = x->als_ctas;
  ab.pdl = pdl_wanted();
  ab.Af_pad = x->Apad; ab.Bf_pad = x->Bpad; ab.Cf_pad = x->Cpad;
  return ab;
}

// Mode 1 and mode 3 of the batch (after its mode 2), then the CP of every
// summary warm-started from the projected previous factors.  Returns false if
// a tensor-core launch of the CP was refused (nothing after the warm start is
// then enqueued).
bool tail_front(octen_ctx *x, int64_t t, const Marker &mk) {
  const octen_config &c = x->cfg;
  compress_finish(x, t, x->Wfix, x->Y, true);
  x->mark(kStWarm, 1);
  pair_fork(x);
  project(x, x->U32, c.I, x->A, x->PA, x->st, x->splitk);
  project(x, x->V32, c.J, x->B, x->PB, x->als_side, x->splitk2);
  warm_start(x->PA, c.P, c.Q, c.S, c.R, x->RT, x->At, x->GA, x->st);
  warm_start(x->PB, c.P, c.Q, c.S, c.R, x->RT, x->Bt, x->GB, x->als_side);
  pair_join(x);
  x->mark(kStWarm, 0);
  AlsBuffers ab = als_buffers(x);
  return als_run(x->Y, c.P, c.Q, c.R, x->RT, c.als_iters, ab, x->st, mk);
}

// Anchor match against u^T A_prev, v^T B_prev, lift of A and B, the new rows
// of C (into Cnew_fix) and the G_p update.
void tail_back(octen_ctx *x, int64_t t) {
  const octen_config &c = x->cfg;
  x->mark(kStAlign, 1);
  align_replicas(x->At, x->Bt, x->Ct, x->PA, x->PB, c.P, c.Q, c.S, c.R, x->RT, x->Ah, x->Bh,
                 x->Ch, x->perm, x->scales, x->align_scratch, x->st);
  x->mark(kStAlign, 0);
  x->mark(kStLift, 1);
  pair_fork(x);
  lift_mode(x, x->Ah, x->PA, x->La, x->a_over, c.I, x->A, false);
  lift_mode(x, x->Bh, x->PB, x->Lb, x->b_over, c.J, x->B, true);
  x->mark(kStLift, 0);
  // the new rows of C need only the aligned blocks, G and W: beside the B lift
  x->mark(kStCsolve, 1);
  solve_c_new(x->Wfix, x->Ch, x->G, t, c.P, c.Q, c.S, x->Qd, c.R, x->RT,
              static_cast<float *>(x->Wbuf.p), x->Cnew_fix, x->dstatus, x->st);
  update_g(x->Wfix, x->Cnew_fix, t, c.P, c.Q, c.S, x->Qd, c.R, x->G, x->st);
  x->mark(kStCsolve, 0);
  pair_join(x);
}

// Records the tail of a t-slice append (tail_front + tail_back) as a graph in
// a free slot of x->tails; nullptr if a launch was refused or the recording
// failed (the eager path runs then).  Every function of the tail enqueues on
// x->st, which points at the private capture stream while recording.
octen_ctx::TailGraph *capture_tail(octen_ctx *x, int64_t t) {
  if (x->captures >= octen_ctx::kMaxCaptures) return nullptr;
  ++x->captures;
  if (!x->cap_st && cudaStreamCreateWithFlags(&x->cap_st, cudaStreamNonBlocking) != cudaSuccess) {
    cudaGetLastError();
    x->cap_st = nullptr;
    return nullptr;
  }
  const uint64_t l0 = octen_launch_count(), t0 = octen_tc_launch_count();
  if (cudaStreamBeginCapture(x->cap_st, cudaStreamCaptureModeRelaxed) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  cudaStream_t home = x->st;
  x->st = x->cap_st;
  const bool ok = tail_front(x, t, Marker{});
  if (ok) tail_back(x, t);
  x->st = home;
  cudaGraph_t g = nullptr;
  const cudaError_t e = cudaStreamEndCapture(x->cap_st, &g);
  const int64_t dl = (int64_t)(octen_launch_count() - l0);
  const int64_t dt = (int64_t)(octen_tc_launch_count() - t0);
  adjust_launch_counts(-dl, -dt);   // recorded, not run
  octen_ctx::TailGraph *slot = nullptr;
  if (ok && e == cudaSuccess && g) {
    octen_ctx::TailGraph &tg = x->tails[x->next_tail];
    if (tg.exec) cudaGraphExecDestroy(tg.exec);
    if (tg.graph) cudaGraphDestroy(tg.graph);
    tg = octen_ctx::TailGraph{};
    if (cudaGraphInstantiate(&tg.exec, g, 0) == cudaSuccess) {
      tg.t = t;
      tg.graph = g;
      g = nullptr;
      tg.launches = dl;
      tg.tc = dt;
      slot = &tg;
      x->next_tail = (x->next_tail + 1) % octen_ctx::kTailGraphs;
    } else {
      tg.exec = nullptr;
    }
  }
  if (g) cudaGraphDestroy(g);
  cudaGetLastError();
  return slot;
}

// The tail of an append on x->st: the recorded graph for this batch size when
// there is one (recorded now if needed), else launch by launch.
void tail_enqueue(octen_ctx *x, int64_t t) {
  const octen_config &c = x->cfg;
  if (!x->timing && x->use_graph) {
    octen_ctx::TailGraph *tg = nullptr;
    for (octen_ctx::TailGraph &g : x->tails)
      if (g.exec && g.t == t) tg = &g;
    if (!tg && x->appends > 0) tg = capture_tail(x, t);
    if (tg && cudaGraphLaunch(tg->exec, x->st) == cudaSuccess) {
      adjust_launch_counts(tg->launches, tg->tc);
      return;
    }
    cudaGetLastError();
  }
  Marker mk;
  if (x->timing) { mk.fn = &octen_ctx::mark_cb; mk.arg = x; }
  if (!tail_front(x, t, mk)) {
    // a tensor-core launch was refused: redo the CP from the warm start on SIMT
    cudaGetLastError();
    count_tc_fallback("replica CP-ALS GEMM");
    x->als_tc = false;
    x->drop_graphs();
    AlsBuffers ab = als_buffers(x);
    ab.use_tc = false;
    warm_start(x->PA, c.P, c.Q, c.S, c.R, x->RT, x->At, x->GA, x->st);
    warm_start(x->PB, c.P, c.Q, c.S, c.R, x->RT, x->Bt, x->GB, x->st);
    als_run(x->Y, c.P, c.Q, c.R, x->RT, c.als_iters, ab, x->st, mk);
  }
  tail_back(x, t);
}

// Whether an append of t slices from X_new copies the host slices in pieces
// (each piece's mode-2 contraction starting as it lands).
bool host_pieces(const octen_ctx *x, const void *X_new, int64_t t) {
  return !is_device_ptr(X_new) && t >= 2 && (x->cfg.I * x->cfg.J) % 16 == 0 && x->copy_st;
}

// Checks an append's arguments and makes every allocation it needs, before
// any of its work is enqueued (a refused allocation leaves the context as it
// was).
octen_status append_prepare(octen_ctx *x, const void *X_new, int64_t t, const float *W_new) {
  if (!x) return OCTEN_EINVAL;
  if (!x->initialized) return x->fail(OCTEN_ESTATE, "octen_append before octen_init");
  if (!X_new || !W_new || t < 1 || t > chunk_slices(x))
    return x->fail(OCTEN_EINVAL, "octen_append: need X_new, W_new and 1 <= t <= %d",
                   (int)chunk_slices(x));
  const octen_config &c = x->cfg;
  const int Qd = x->Qd;
  if (!ensure_c_capacity(x, x->K + t)) return x->fail(OCTEN_ENOMEM, "C");
  const size_t cs = c_solve_scratch_floats(t, Qd, c.R);
  if (!x->grow(x->Wbuf, cs * sizeof(float))) return x->fail(OCTEN_ENOMEM, "C solve scratch");
  octen_status s = compress_scratch(x, t);
  if (s != OCTEN_OK) return s;
  const size_t slice = (size_t)c.I * c.J * elem_size(x->xin);
  if (host_pieces(x, X_new, t)) {
    if (!x->grow(x->xstage[x->xslot], t * slice))
      return x->fail(OCTEN_ENOMEM, "staging the batch");
  } else if (!is_device_ptr(X_new) && !x->grow(x->stage[2], t * slice)) {
    return x->fail(OCTEN_ENOMEM, "staging the batch");
  }
  if (!is_device_ptr(W_new) && !x->grow(x->stage[1], (size_t)t * Qd * 4))
    return x->fail(OCTEN_ENOMEM, "staging W_new");
  return OCTEN_OK;
}

// The head of a prepared append on x->st: the batch's W rows into Wfix, the
// quantisation (fp8) and the mode-2 contraction.
octen_status append_head(octen_ctx *x, const void *X_new, int64_t t, const float *W_new,
                         int pieces) {
  const octen_config &c = x->cfg;
  const size_t slice = (size_t)c.I * c.J * elem_size(x->xin);
  const float *Wd = static_cast<const float *>(x->stage_in(W_new, (size_t)t * x->Qd * 4, 1));
  if (!Wd) return x->fail(OCTEN_ECUDA, "staging W_new");
  cudaMemcpyAsync(x->Wfix, Wd, (size_t)t * x->Qd * sizeof(float), cudaMemcpyDeviceToDevice,
                  x->st);
  if (host_pieces(x, X_new, t)) return compress_mode2_host(x, X_new, t, pieces);
  const void *Xd = x->stage_in(X_new, t * slice, 2);
  if (!Xd) return x->fail(OCTEN_ECUDA, "staging the batch");
  compress_mode2(x, Xd, 0, t);
  return OCTEN_OK;
}

// Enqueues one prepared append on the context's stream (no final
// synchronisation; K is advanced by the caller once the stream has finished
// without error): the head, then the rest of the update (Y_p += Z_p, CP of
// every summary, anchor match, lift of A and B, the new rows of C and the
// G_p update), then the new rows into C.
octen_status append_launch(octen_ctx *x, const void *X_new, int64_t t, const float *W_new,
                           int pieces = octen_ctx::kCopyChunks) {
  octen_status s = append_head(x, X_new, t, W_new, pieces);
  if (s != OCTEN_OK) return s;
  tail_enqueue(x, t);
  cudaMemcpyAsync(x->C + x->K * x->cfg.R, x->Cnew_fix, (size_t)t * x->cfg.R * sizeof(float),
                  cudaMemcpyDeviceToDevice, x->st);
  ++x->appends;
  return OCTEN_OK;
}

octen_status append_enqueue(octen_ctx *x, const void *X_new, int64_t t, const float *W_new) {
  const octen_status s = append_prepare(x, X_new, t, W_new);
  return s != OCTEN_OK ? s : append_launch(x, X_new, t, W_new);
}

// The recorded tail of a t-slice append, if there is one.
octen_ctx::TailGraph *find_tail(octen_ctx *x, int64_t t) {
  for (octen_ctx::TailGraph &g : x->tails)
    if (g.exec && g.graph && g.t == t) return &g;
  return nullptr;
}

// The head of a prepared append of device arrays recorded as a graph on the
// context's capture stream (nullptr on failure).  Its kernels are not
// counted: they run when the step graph runs.
cudaGraph_t capture_head(octen_ctx *x, const void *X, int64_t t, const float *W,
                         int64_t &launches, int64_t &tc) {
  if (!x->cap_st && cudaStreamCreateWithFlags(&x->cap_st, cudaStreamNonBlocking) != cudaSuccess) {
    cudaGetLastError();
    x->cap_st = nullptr;
    return nullptr;
  }
  const uint64_t l0 = octen_launch_count(), t0 = octen_tc_launch_count();
  if (cudaStreamBeginCapture(x->cap_st, cudaStreamCaptureModeRelaxed) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  cudaStream_t home = x->st;
  x->st = x->cap_st;
  const octen_status s = append_head(x, X, t, W, octen_ctx::kCopyChunks);
  x->st = home;
  cudaGraph_t g = nullptr;
  const cudaError_t e = cudaStreamEndCapture(x->cap_st, &g);
  launches = (int64_t)(octen_launch_count() - l0);
  tc = (int64_t)(octen_tc_launch_count() - t0);
  adjust_launch_counts(-launches, -tc);
  if (s != OCTEN_OK || e != cudaSuccess || !g) {
    if (g) cudaGraphDestroy(g);
    cudaGetLastError();
    return nullptr;
  }
  return g;
}

// One step of octen_append_many as a single graph launch (see
// octen_ctx::StepGraph), after every context has been prepared.  Returns false,
// with nothing enqueued, when the step does not qualify (a context timing its
// stages or without graphs, host arrays, a context given twice, a batch size
// without a recorded tail) or the graph cannot be built; the caller then
// enqueues the appends one by one.
bool step_graph_launch(octen_ctx *const *ctxs, int n, const void *const *X, const int64_t *t,
                       const float *const *W) {
  octen_ctx *L = ctxs[0];
  std::vector<int64_t> key;
  key.reserve(3 * (size_t)n);
  for (int i = 0; i < n; ++i) {
    octen_ctx *x = ctxs[i];
    if (x->timing || !x->use_graph || !is_device_ptr(X[i]) || !is_device_ptr(W[i]) ||
        !find_tail(x, t[i]))
      return false;
    for (int j = 0; j < i; ++j)
      if (ctxs[j] == x) return false;
    key.push_back((int64_t)x->id);
    key.push_back((int64_t)x->gen);
    key.push_back(t[i]);
  }
  for (int i = 0; i < n; ++i) {
    octen_ctx *x = ctxs[i];
    if ((!x->step_ev && cudaEventCreateWithFlags(&x->step_ev, cudaEventDisableTiming) != cudaSuccess) ||
        (!x->step_done &&
         cudaEventCreateWithFlags(&x->step_done, cudaEventDisableTiming) != cudaSuccess)) {
      cudaGetLastError();
      return false;
    }
  }
  int64_t head_l = 0, head_tc = 0;
  bool fresh = L->step.exec == nullptr || L->step.key != key;
  if (!fresh) {
    // same contexts and shapes: new slices into the heads, new row offsets
    // into the C copies
    for (int i = 0; i < n && !fresh; ++i) {
      octen_ctx *x = ctxs[i];
      int64_t hl = 0, htc = 0;
      cudaGraph_t hg = capture_head(x, X[i], t[i], W[i], hl, htc);
      const bool ok =
          hg && cudaGraphExecChildGraphNodeSetParams(L->step.exec, L->step.head[i], hg) ==
                    cudaSuccess &&
          cudaGraphExecMemcpyNodeSetParams1D(
              L->step.exec, L->step.cmem[i], x->C + x->K * x->cfg.R, x->Cnew_fix,
              (size_t)t[i] * x->cfg.R * sizeof(float), cudaMemcpyDeviceToDevice) == cudaSuccess;
      if (hg) cudaGraphDestroy(hg);
      if (!ok) {
        cudaGetLastError();
        fresh = true;
      }
      head_l += hl;
      head_tc += htc;
    }
  }
  if (fresh) {
    L->drop_step();
    head_l = head_tc = 0;
    cudaGraph_t sg = nullptr;
    if (cudaGraphCreate(&sg, 0) != cudaSuccess) {
      cudaGetLastError();
      return false;
    }
    bool ok = true;
    octen_ctx::StepGraph st;
    for (int i = 0; i < n && ok; ++i) {
      octen_ctx *x = ctxs[i];
      int64_t hl = 0, htc = 0;
      cudaGraph_t hg = capture_head(x, X[i], t[i], W[i], hl, htc);
      octen_ctx::TailGraph *tg = find_tail(x, t[i]);
      cudaGraphNode_t hn = nullptr, tn = nullptr, cn = nullptr;
      ok = hg && tg && cudaGraphAddChildGraphNode(&hn, sg, nullptr, 0, hg) == cudaSuccess &&
           cudaGraphAddChildGraphNode(&tn, sg, &hn, 1, tg->graph) == cudaSuccess &&
           cudaGraphAddMemcpyNode1D(&cn, sg, &tn, 1, x->C + x->K * x->cfg.R, x->Cnew_fix,
                                    (size_t)t[i] * x->cfg.R * sizeof(float),
                                    cudaMemcpyDeviceToDevice) == cudaSuccess;
      if (hg) cudaGraphDestroy(hg);
      if (ok) {
        st.head.push_back(hn);
        st.cmem.push_back(cn);
        st.launches += tg->launches;
        st.tc += tg->tc;
        head_l += hl;
        head_tc += htc;
      }
    }
    if (ok && cudaGraphInstantiate(&st.exec, sg, 0) != cudaSuccess) {
      st.exec = nullptr;
      ok = false;
    }
    if (!ok) {
      cudaGraphDestroy(sg);
      cudaGetLastError();
      return false;
    }
    st.graph = sg;
    st.key = key;
    L->step = std::move(st);
  }
  // after the work already on every context's stream; before its next work
  for (int i = 0; i < n; ++i) {
    cudaEventRecord(ctxs[i]->step_ev, ctxs[i]->st);
    cudaStreamWaitEvent(L->st, ctxs[i]->step_ev, 0);
  }
  if (cudaGraphLaunch(L->step.exec, L->st) != cudaSuccess) {
    cudaGetLastError();
    L->drop_step();
    return false;
  }
  cudaEventRecord(L->step_done, L->st);
  for (int i = 0; i < n; ++i) {
    if (ctxs[i] != L) cudaStreamWaitEvent(ctxs[i]->st, L->step_done, 0);
    ++ctxs[i]->appends;
  }
  adjust_launch_counts(L->step.launches + head_l, L->step.tc + head_tc);
  return true;
}

// After a failed enqueue: nothing the call issued may still read the caller's
// buffers when it returns.
void drain(octen_ctx *x) {
  if (!x) return;
  if (x->copy_st) cudaStreamSynchronize(x->copy_st);
  cudaStreamSynchronize(x->st);
  cudaGetLastError();
}

}  // namespace

extern "C" {

octen_status octen_append(octen_ctx *x, const void *X_new, int64_t t, const float *W_new) {
  octen_status s = append_enqueue(x, X_new, t, W_new);
  if (s != OCTEN_OK) {
    drain(x);
    return s;
  }
  s = x->sync_check("append");
  x->done_ticket = x->next_ticket;   // every asynchronous append before it has run too
  if (s != OCTEN_OK) return s;
  x->K += t;
  return OCTEN_OK;
}

octen_status octen_wait(octen_ctx *x, int64_t ticket) {
  if (!x || ticket < 0 || ticket >= x->next_ticket) return OCTEN_EINVAL;
  if (ticket < x->done_ticket) return OCTEN_OK;
  const int slot = (int)(ticket % octen_ctx::kTickets);
  cudaError_t e = cudaEventSynchronize(x->ticket_ev[slot]);
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e != cudaSuccess) return x->fail(OCTEN_ECUDA, "wait: %s", cudaGetErrorString(e));
  const int flags = x->ticket_status[slot];
  x->done_ticket = ticket + 1;
  if (x->done_ticket == x->next_ticket) x->free_retired();   // nothing of the context in flight
  if (flags & kDevTimeout) return x->fail(OCTEN_ETIMEOUT, "append: a device wait ran out");
  if (flags) return x->fail(OCTEN_ENUMERIC, "append: a Cholesky pivot was not positive");
  return OCTEN_OK;
}

octen_status octen_append_async(octen_ctx *x, const void *X_new, int64_t t, const float *W_new,
                                float *A_out, float *B_out, float *C_new_out,
                                int64_t *ticket) {
  if (!x || !ticket) return OCTEN_EINVAL;
  // at most kTickets appends in flight: the oldest is waited for first
  if (x->next_ticket - x->done_ticket >= octen_ctx::kTickets) {
    const octen_status s = octen_wait(x, x->done_ticket);
    if (s != OCTEN_OK) return s;
  }
  octen_status s = append_prepare(x, X_new, t, W_new);
  // the copy of a host batch runs while the appends before it update, so it is
  // one piece and one contraction (the pieces of octen_append overlap the
  // copy with the contraction inside a single call)
  if (s == OCTEN_OK) s = append_launch(x, X_new, t, W_new, 1);
  if (s != OCTEN_OK) {
    drain(x);
    return s;
  }
  const octen_config &c = x->cfg;
  if (A_out) cudaMemcpyAsync(A_out, x->A, (size_t)c.I * c.R * 4, cudaMemcpyDefault, x->st);
  if (B_out) cudaMemcpyAsync(B_out, x->B, (size_t)c.J * c.R * 4, cudaMemcpyDefault, x->st);
  if (C_new_out)
    cudaMemcpyAsync(C_new_out, x->C + x->K * c.R, (size_t)t * c.R * 4, cudaMemcpyDefault, x->st);
  const int slot = (int)(x->next_ticket % octen_ctx::kTickets);
  cudaMemcpyAsync(x->ticket_status + slot, x->dstatus, sizeof(int), cudaMemcpyDeviceToHost, x->st);
  cudaEventRecord(x->ticket_ev[slot], x->st);
  x->K += t;
  *ticket = x->next_ticket++;
  return OCTEN_OK;
}

octen_status octen_append_many(octen_ctx *const *ctxs, int n, const void *const *X_new,
                               const int64_t *t, const float *const *W_new) {
  if (!ctxs || !X_new || !t || !W_new || n < 1) return OCTEN_EINVAL;
  octen_status first = OCTEN_OK;
  std::vector<char> ready(n, 0), enqueued(n, 0);
  // the ALS GEMMs of each context on a share of the SMs: 1 / min(n, 8) of
  // them, or OCTEN_MANY_CTAS CTAs (0: all)
  {
    int dev = 0, nsm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    int share = n > 1 ? nsm / (n < 8 ? n : 8) : 0;
    const char *v = getenv("OCTEN_MANY_CTAS");
    if (v && *v) share = atoi(v);
    if (share < 0 || share >= nsm) share = 0;
    for (int i = 0; i < n; ++i) {
      octen_ctx *x = ctxs[i];
      if (x && x->als_ctas != share) {
        x->als_ctas = share;
        x->drop_graphs();   // recorded with the old grid
        ++x->gen;
      }
    }
  }
  for (int i = 0; i < n; ++i) {
    const octen_status s = append_prepare(ctxs[i], X_new[i], t[i], W_new[i]);
    ready[i] = s == OCTEN_OK;
    if (s != OCTEN_OK && first == OCTEN_OK) first = s;
  }
  // every context prepared: the whole step as one graph launch when it qualifies
  bool all = first == OCTEN_OK;
  if (all && step_graph_launch(ctxs, n, X_new, t, W_new)) {
    for (int i = 0; i < n; ++i) enqueued[i] = 1;
  } else {
    for (int i = 0; i < n; ++i) {
      if (!ready[i]) continue;
      const octen_status s = append_launch(ctxs[i], X_new[i], t[i], W_new[i]);
      enqueued[i] = s == OCTEN_OK;
      if (s != OCTEN_OK) {
        drain(ctxs[i]);
        if (first == OCTEN_OK) first = s;
      }
    }
  }
  for (int i = 0; i < n; ++i) {
    if (!enqueued[i]) continue;
    const octen_status s = ctxs[i]->sync_check("append_many");
    if (s == OCTEN_OK) ctxs[i]->K += t[i];
    else if (first == OCTEN_OK) first = s;
  }
  return first;
}

octen_status octen_get_factors(const octen_ctx *cx, float *A, float *B, float *C,
                               int64_t *K_out) {
  octen_ctx *x = const_cast<octen_ctx *>(cx);
  if (!x) return OCTEN_EINVAL;
  if (!x->initialized) return x->fail(OCTEN_ESTATE, "no factors before octen_init");
  const octen_config &c = x->cfg;
  if (A) cudaMemcpyAsync(A, x->A, (size_t)c.I * c.R * 4, cudaMemcpyDefault, x->st);
  if (B) cudaMemcpyAsync(B, x->B, (size_t)c.J * c.R * 4, cudaMemcpyDefault, x->st);
  if (C) cudaMemcpyAsync(C, x->C, (size_t)x->K * c.R * 4, cudaMemcpyDefault, x->st);
  if (K_out) *K_out = x->K;
  return x->sync_check("get_factors");
}

int64_t octen_rows(const octen_ctx *x) { return x ? x->K : 0; }

uint64_t octen_device_bytes(const octen_ctx *x) { return x ? (uint64_t)x->held : 0; }

octen_status octen_fit(octen_ctx *x, const void *X_all, int64_t K, double *fit_out) {
  if (!x || !X_all || !fit_out) return OCTEN_EINVAL;
  if (!x->initialized) return x->fail(OCTEN_ESTATE, "octen_fit before octen_init");
  if (K != x->K) return x->fail(OCTEN_EINVAL, "octen_fit: K=%lld, rows=%lld",
                                (long long)K, (long long)x->K);
  const octen_config &c = x->cfg;
  if (c.I > fit_rows_max())
    return x->fail(OCTEN_EINVAL, "octen_fit: I=%lld above %lld", (long long)c.I,
                   (long long)fit_rows_max());
  const size_t slice = (size_t)c.I * c.J * elem_size(x->xin);
  const int64_t np = fit_partial_count(1, c.I, c.J);
  // slices are streamed in chunks (host inputs are staged chunk by chunk;
  // device inputs in chunks of at most kFitSlicesMax)
  const int64_t chunk = is_device_ptr(X_all) ? (K < kFitSlicesMax ? K : kFitSlicesMax) : 16;
  if (!x->grow(x->fitpart, (size_t)np * chunk * 2 * sizeof(double)))
    return x->fail(OCTEN_ENOMEM, "fit scratch");
  double total0 = 0.0, total1 = 0.0;
  for (int64_t k0 = 0; k0 < K; k0 += chunk) {
    const int64_t n = K - k0 < chunk ? K - k0 : chunk;
    const void *Xd = x->stage_in(static_cast<const char *>(X_all) + k0 * slice, n * slice, 3);
    if (!Xd) return x->fail(OCTEN_ENOMEM, "staging X_all");
    fit_sums(Xd, x->xin, n, c.I, c.J, x->A, x->B, x->C + k0 * c.R, c.R,
             static_cast<double *>(x->fitpart.p), x->dfit, x->st);
    double h[2];
    cudaMemcpyAsync(h, x->dfit, sizeof h, cudaMemcpyDeviceToHost, x->st);
    octen_status s = x->sync_check("fit");
    if (s != OCTEN_OK) return s;
    total0 += h[0];
    total1 += h[1];
  }
  *fit_out = total0 > 0.0 ? 1.0 - sqrt(total1) / sqrt(total0) : 0.0;
  return OCTEN_OK;
}

namespace {

// Device arrays that make up the state of an initialised context, in file order.
struct StateArray {
  void *p;
  size_t bytes;
};

std::vector<StateArray> state_arrays(octen_ctx *x) {
  const octen_config &c = x->cfg;
  const size_t P = c.P, Q = c.Q, Qd = x->Qd;
  return {
      {x->U32, (size_t)c.I * Qd * 4},
      {x->V32, (size_t)c.J * Qd * 4},
      {x->Ut_rep, P * Q * c.I * elem_size(x->tu)},
      {x->Vt, Qd * c.J * elem_size(x->tv)},
      {x->La, (size_t)c.I * Qd * 4},
      {x->Lb, (size_t)c.J * Qd * 4},
      {x->Y, P * Q * Q * Q * 4},
      {x->A, (size_t)c.I * c.R * 4},
      {x->B, (size_t)c.J * c.R * 4},
      {x->G, P * Q * c.R * 4},
      {x->C, (size_t)x->K * c.R * 4},
  };
}

const char kMagic[8] = {'O', 'C', 'T', 'E', 'N', 'S', 'T', '1'};

}  // namespace

octen_status octen_save(const octen_ctx *cx, const char *path) {
  octen_ctx *x = const_cast<octen_ctx *>(cx);
  if (!x || !path) return OCTEN_EINVAL;
  if (!x->initialized) return x->fail(OCTEN_ESTATE, "octen_save before octen_init");
  if (x->sync_check("save") != OCTEN_OK) return OCTEN_ECUDA;
  FILE *f = fopen(path, "wb");
  if (!f) return x->fail(OCTEN_EINVAL, "octen_save: cannot open %s", path);
  int64_t hdr[4] = {x->K, x->a_over, x->b_over, 0};
  bool ok = fwrite(kMagic, 1, 8, f) == 8 && fwrite(&x->cfg, sizeof x->cfg, 1, f) == 1 &&
            fwrite(hdr, sizeof hdr, 1, f) == 1;
  std::vector<char> host;
  for (const StateArray &a : state_arrays(x)) {
    if (!ok) break;
    host.resize(a.bytes);
    ok = cudaMemcpy(host.data(), a.p, a.bytes, cudaMemcpyDeviceToHost) == cudaSuccess &&
         fwrite(host.data(), 1, a.bytes, f) == a.bytes;
  }
  ok = (fclose(f) == 0) && ok;
  return ok ? OCTEN_OK : x->fail(OCTEN_ECUDA, "octen_save: writing %s failed", path);
}

octen_status octen_load(const char *path, void *cuda_stream, octen_ctx **out) {
  if (!path || !out) return OCTEN_EINVAL;
  FILE *f = fopen(path, "rb");
  if (!f) return OCTEN_EINVAL;
  char magic[8];
  octen_config cfg{};
  int64_t hdr[4];
  if (fread(magic, 1, 8, f) != 8 || memcmp(magic, kMagic, 8) != 0 ||
      fread(&cfg, sizeof cfg, 1, f) != 1 || fread(hdr, sizeof hdr, 1, f) != 1 || hdr[0] < 1 ||
      hdr[0] > kCRowsMax) {
    fclose(f);
    return OCTEN_EINVAL;
  }
  octen_ctx *x = nullptr;
  octen_status s = octen_create(&cfg, cuda_stream, &x);
  if (s != OCTEN_OK) {
    fclose(f);
    return s;
  }
  // the lift operators' layouts follow from the shapes (Qd above or below
  // the factor's rows); a header that disagrees was not written by octen_save
  if (hdr[1] != (x->Qd > cfg.I ? 1 : 0) || hdr[2] != (x->Qd > cfg.J ? 1 : 0)) {
    fclose(f);
    delete x;
    return OCTEN_EINVAL;
  }
  if (!ensure_c_capacity(x, hdr[0])) {
    fclose(f);
    delete x;
    return OCTEN_ENOMEM;
  }
  x->K = hdr[0];
  x->a_over = (int)hdr[1];
  x->b_over = (int)hdr[2];
  bool ok = true;
  std::vector<char> host;
  for (const StateArray &a : state_arrays(x)) {
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

octen_status octen_get_replicas(const octen_ctx *cx, float *Y) {
  octen_ctx *x = const_cast<octen_ctx *>(cx);
  if (!x || !Y) return OCTEN_EINVAL;
  const size_t n = (size_t)x->cfg.P * x->cfg.Q * x->cfg.Q * x->cfg.Q;
  cudaMemcpyAsync(Y, x->Y, n * 4, cudaMemcpyDefault, x->st);
  return x->sync_check("get_replicas");
}

octen_status octen_get_replica_factors(const octen_ctx *cx, int which, float *At, float *Bt,
                                       float *Ct, int32_t *perm, double *scales) {
  octen_ctx *x = const_cast<octen_ctx *>(cx);
  if (!x || (which != 0 && which != 1)) return OCTEN_EINVAL;
  const octen_config &c = x->cfg;
  const float *src[3] = {which ? x->Ah : x->At, which ? x->Bh : x->Bt, which ? x->Ch : x->Ct};
  float *dst[3] = {At, Bt, Ct};
  for (int i = 0; i < 3; ++i) {
    if (!dst[i]) continue;
    cudaMemcpy2DAsync(dst[i], c.R * 4, src[i], x->RT * 4, c.R * 4, (size_t)c.P * c.Q,
                      cudaMemcpyDefault, x->st);
  }
  if (perm) cudaMemcpyAsync(perm, x->perm, (size_t)c.P * c.R * 4, cudaMemcpyDefault, x->st);
  if (scales)
    cudaMemcpyAsync(scales, x->scales, (size_t)c.P * 2 * c.R * 8, cudaMemcpyDefault, x->st);
  return x->sync_check("get_replica_factors");
}

octen_status octen_compress(const octen_config *cfg, void *cuda_stream, const void *X, int64_t t,
                            const float *U_all, const float *V_all, const float *W_all,
                            float *Z) {
  std::string why;
  if (validate_config(cfg, why) != OCTEN_OK || !X || !U_all || !V_all || !W_all || !Z || t < 1)
    return OCTEN_EINVAL;
  // a light context: projections, scratch and a summary buffer only
  octen_ctx x;
  x.limit = device_memory_limit();
  x.cfg = *cfg;
  x.Qd = cfg->S + cfg->P * (cfg->Q - cfg->S);
  x.RT = round_rt(cfg->R);
  x.st = static_cast<cudaStream_t>(cuda_stream);
  set_types(&x);
  const octen_config &c = x.cfg;
  const size_t Qd = x.Qd, nz = (size_t)c.P * c.Q * c.Q * c.Q;
  float *Zd = nullptr;
  bool ok = x.alloc(x.U32, (size_t)c.I * Qd) && x.alloc(x.V32, (size_t)c.J * Qd) &&
            x.alloc(x.dstatus, 1) && x.alloc(Zd, nz);
  void *ut = nullptr, *vt = nullptr;
  if (ok) {
    const size_t ub = (size_t)c.P * c.Q * c.I * elem_size(x.tu), vb = Qd * c.J * elem_size(x.tv);
    ok = x.dev_malloc(&ut, ub) && x.dev_malloc(&vt, vb);
    if (ut) x.owned.push_back({ut, ub});
    if (vt) x.owned.push_back({vt, vb});
  }
  if (!ok) { cudaGetLastError(); return OCTEN_ENOMEM; }
  x.Ut_rep = ut;
  x.Vt = vt;
  cudaMemsetAsync(x.dstatus, 0, sizeof(int), x.st);
  cudaMemsetAsync(Zd, 0, nz * 4, x.st);
  const float *Ud = static_cast<const float *>(x.stage_in(U_all, (size_t)c.I * Qd * 4, 0));
  if (!Ud) return OCTEN_ENOMEM;
  round_copy(Ud, x.U32, (int64_t)c.I * Qd, x.tu, x.st);
  const float *Vd = static_cast<const float *>(x.stage_in(V_all, (size_t)c.J * Qd * 4, 1));
  if (!Vd) return OCTEN_ENOMEM;
  round_copy(Vd, x.V32, (int64_t)c.J * Qd, x.tv, x.st);
  make_replica_transpose(x.U32, c.I, c.P, c.Q, c.S, x.Qd, x.Ut_rep, x.tu, x.st);
  make_transpose(x.V32, c.J, x.Qd, x.Vt, x.tv, x.st);
  if (x.sync_check("compress setup") != OCTEN_OK) return OCTEN_ECUDA;
  const float *Wd = static_cast<const float *>(x.stage_in(W_all, (size_t)t * Qd * 4, 3));
  if (!Wd) return OCTEN_ENOMEM;
  const size_t slice = (size_t)c.I * c.J * elem_size(x.xin);
  octen_status s = OCTEN_OK;
  if (is_device_ptr(X)) {
    s = compress_all(&x, X, t, Wd, Zd);
  } else {
    const int64_t ck = chunk_slices(&x);
    for (int64_t k0 = 0; k0 < t && s == OCTEN_OK; k0 += ck) {
      const int64_t n = t - k0 < ck ? t - k0 : ck;
      const void *Xd = x.stage_in(static_cast<const char *>(X) + k0 * slice, n * slice, 2);
      if (!Xd) return OCTEN_ENOMEM;
      s = compress_chunk(&x, Xd, n, Wd + k0 * Qd, Zd);
      cudaStreamSynchronize(x.st);
    }
  }
  if (s != OCTEN_OK) return s;
  cudaMemcpyAsync(Z, Zd, nz * 4, cudaMemcpyDefault, x.st);
  return x.sync_check("compress");
}

void octen_destroy(octen_ctx *x) { delete x; }

const char *octen_last_error(const octen_ctx *x) {
  return x ? x->err.c_str() : "no context";
}

const char *octen_status_name(octen_status s) {
  switch (s) {
    case OCTEN_OK: return "OCTEN_OK";
    case OCTEN_EINVAL: return "OCTEN_EINVAL";
    case OCTEN_ENOMEM: return "OCTEN_ENOMEM";
    case OCTEN_ECUDA: return "OCTEN_ECUDA";
    case OCTEN_ETIMEOUT: return "OCTEN_ETIMEOUT";
    case OCTEN_ENUMERIC: return "OCTEN_ENUMERIC";
    case OCTEN_ESTATE: return "OCTEN_ESTATE";
  }
  return "OCTEN_UNKNOWN";
}

uint64_t octen_launch_count(void) { return g_launches.load(); }

uint64_t octen_tc_launch_count(void) { return g_tc_launches.load(); }

uint64_t octen_tc_fallback_count(void) { return g_tc_fallbacks.load(); }

static const char *kStageNames[kNumStages] = {"quantize", "mode2", "mode1", "mode3",
                                              "warm_start", "als_gemm", "als_aux", "als_solve",
                                              "align", "lift", "c_solve", "als_fused"};

int octen_stage_count(void) { return kNumStages; }

const char *octen_stage_name(int i) {
  return (i >= 0 && i < kNumStages) ? kStageNames[i] : "unknown";
}

octen_status octen_set_timing(octen_ctx *x, int on) {
  if (!x) return OCTEN_EINVAL;
  x->timing = on != 0;
  return OCTEN_OK;
}

octen_status octen_stage_times(const octen_ctx *cx, double *ms, uint64_t *launches) {
  octen_ctx *x = const_cast<octen_ctx *>(cx);
  if (!x) return OCTEN_EINVAL;
  for (int i = 0; i < kNumStages; ++i) {
    if (ms) ms[i] = x->stage_ms[i];
    if (launches) launches[i] = x->stage_n[i];
  }
  return OCTEN_OK;
}

octen_status octen_reset_stage_times(octen_ctx *x) {
  if (!x) return OCTEN_EINVAL;
  for (int i = 0; i < kNumStages; ++i) { x->stage_ms[i] = 0.0; x->stage_n[i] = 0; }
  return OCTEN_OK;
}

}  // extern "C"
