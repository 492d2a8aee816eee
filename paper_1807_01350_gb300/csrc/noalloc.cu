// Compression of one slice batch without any device allocation.
//
// Some callers cannot call cudaMalloc at all: a process that runs under a fixed
// device-memory budget handed out by its host framework, a plugin whose host
// forbids the CUDA allocator, or latency-critical code that must not pay for an
// allocation.  octen_compress_noalloc serves them: every scratch buffer the
// compression needs (the transposed projections, the mode-2 and mode-1
// intermediates, the e4m3 copy of the slices, the status word) lives in one
// file-scope device array of kNoAllocScratchBytes bytes, which every GPU that
// loads the library holds until the process exits.
//
// Set-up: the first call on a device looks up the array's device address with
// cudaGetSymbolAddress (with that device current) and caches it; make that
// first call before any stream capture.  The array is shared by every call:
// its contents are whatever the last call left, so each call clears what has
// to start at zero, and calls whose GPU work overlaps (other streams, other
// threads) race on it and must be serialised by the caller.
#include <mutex>

#include "octen_internal.cuh"

namespace {

constexpr size_t kNoAllocScratchBytes = size_t(64) << 20;   // 64 MiB
constexpr int kMaxDevices = 64;
constexpr int64_t kMaxChunk = 64;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

std::mutex g_setup_mu;
void *g_scratch_ptr[kMaxDevices] = {};

// Device address of the scratch array on the current device (set up once).
void *scratch_on_current_device() {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return nullptr;
  std::lock_guard<std::mutex> lock(g_setup_mu);
  if (!g_scratch_ptr[dev]) {
    void *p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    g_scratch_ptr[dev] = p;
  }
  return g_scratch_ptr[dev];
}

size_t align256(size_t n) { return (n + 255) & ~size_t(255); }

bool on_device(const void *p) {
  cudaPointerAttributes a{};
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

}  // namespace

using namespace octen;

extern "C" octen_status octen_compress_noalloc(const octen_config *cfg, void *cuda_stream,
                                               const void *X, int64_t t, const float *U_all,
                                               const float *V_all, const float *W_all,
                                               float *Z) {
  if (!cfg || !X || !U_all || !V_all || !W_all || !Z || t < 1) return OCTEN_EINVAL;
  std::string why;
  if (validate_config(cfg, why) != OCTEN_OK) {
    fprintf(stderr, "octen_compress_noalloc: %s\n", why.c_str());
    return OCTEN_EINVAL;
  }
  const octen_config &c = *cfg;
  const int Qd = c.S + c.P * (c.Q - c.S);
  const Elem tx = c.prec == OCTEN_FP32 ? Elem::F32 : Elem::BF16;
  const Elem tu = c.prec == OCTEN_FP32 ? Elem::F32 : Elem::BF16;
  const Elem tv = c.prec == OCTEN_FP32 ? Elem::F32
                                       : (c.prec == OCTEN_BF16 ? Elem::BF16 : Elem::E4M3);
  const Elem tmid = tu;
  const bool fp8 = c.prec == OCTEN_FP8E4M3;

  // scratch layout: status | Ut_rep | Vt | per-chunk [T_rep | T2 | X8 | scale]
  const size_t fixed = align256(sizeof(int)) +
                       align256((size_t)c.P * c.Q * c.I * elem_size(tu)) +
                       align256((size_t)Qd * c.J * elem_size(tv));
  const size_t per_slice_T = (size_t)c.P * c.Q * c.I * elem_size(tmid);
  const size_t per_slice_T2 = (size_t)c.P * c.Q * c.Q * sizeof(float);
  const size_t per_slice_X8 = fp8 ? (size_t)c.I * c.J : 0;
  const size_t per_slice = per_slice_T + per_slice_T2 + per_slice_X8 + (fp8 ? 4 : 0);
  // slices per pass: as many as the scratch holds, at most kMaxChunk, and at
  // most kGridYZMax / P (the batched mode-1 product has one GEMM per slice
  // and replica on a grid dimension)
  constexpr size_t kSlack = 4 * 256;   // alignment of the four per-pass buffers
  int64_t chunk = 0;
  if (fixed + kSlack < kNoAllocScratchBytes)
    chunk = (int64_t)((kNoAllocScratchBytes - fixed - kSlack) / per_slice);
  if (chunk > kMaxChunk) chunk = kMaxChunk;
  if (chunk > kGridYZMax / c.P) chunk = kGridYZMax / c.P;
  if (chunk > t) chunk = t;
  if (chunk < 1) {
    fprintf(stderr,
            "octen_compress_noalloc: shape needs %zu bytes of scratch for the projections plus "
            "%zu for one slice; the static scratch holds %zu bytes (use octen_compress)\n",
            fixed, per_slice, kNoAllocScratchBytes);
    return OCTEN_EINVAL;
  }
  // device memory only: copying host buffers would need a staging allocation
  if (!on_device(X) || !on_device(U_all) || !on_device(V_all) || !on_device(W_all) ||
      !on_device(Z)) {
    fprintf(stderr, "octen_compress_noalloc: every array must be device memory\n");
    return OCTEN_EINVAL;
  }
  unsigned char *base = static_cast<unsigned char *>(scratch_on_current_device());
  if (!base) return OCTEN_ECUDA;

  size_t off = 0;
  auto carve = [&](size_t bytes) {
    unsigned char *p = base + off;
    off += align256(bytes);
    return p;
  };
  int *status = reinterpret_cast<int *>(carve(sizeof(int)));
  void *Ut = carve((size_t)c.P * c.Q * c.I * elem_size(tu));
  void *Vt = carve((size_t)Qd * c.J * elem_size(tv));
  void *T = carve(chunk * per_slice_T);
  float *T2 = reinterpret_cast<float *>(carve(chunk * per_slice_T2));
  void *X8 = fp8 ? carve(chunk * per_slice_X8) : nullptr;
  float *scale = fp8 ? reinterpret_cast<float *>(carve(chunk * sizeof(float))) : nullptr;
  if (off > kNoAllocScratchBytes) return OCTEN_EINVAL;

  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  const size_t nz = (size_t)c.P * c.Q * c.Q * c.Q;
  cudaMemsetAsync(status, 0, sizeof(int), st);      // the scratch keeps the last call's data
  cudaMemsetAsync(Z, 0, nz * sizeof(float), st);    // mode 3 accumulates into Z
  make_replica_transpose(U_all, c.I, c.P, c.Q, c.S, Qd, Ut, tu, st);
  make_transpose(V_all, c.J, Qd, Vt, tv, st);
  const bool use_tc = c.prec != OCTEN_FP32 && tc_supported();
  const size_t slice_bytes = (size_t)c.I * c.J * elem_size(tx);
  for (int64_t k0 = 0; k0 < t; k0 += chunk) {
    const int64_t n = t - k0 < chunk ? t - k0 : chunk;
    const void *Xc = static_cast<const char *>(X) + k0 * slice_bytes;
    Mode2Args m2{};
    m2.X = Xc; m2.tx = tx; m2.Vt = Vt; m2.tv = tv; m2.slice_scale = nullptr;
    m2.T = T; m2.tt = tmid; m2.t = n; m2.I = c.I; m2.J = c.J;
    m2.P = c.P; m2.Q = c.Q; m2.S = c.S; m2.Qd = Qd;
    if (fp8) {
      quantize_e4m3(static_cast<const __nv_bfloat16 *>(Xc), n, c.I * c.J,
                    static_cast<__nv_fp8_e4m3 *>(X8), scale, st);
      m2.X = X8; m2.tx = Elem::E4M3; m2.slice_scale = scale;
    }
    if (!(use_tc && mode2_tc(m2, status, st))) {
      cudaGetLastError();
      if (use_tc) count_tc_fallback("mode-2 contraction");
      mode2_simt(m2, st);
    }
    Mode1Args m1{};
    m1.Ut = Ut; m1.T = T; m1.te = tmid; m1.T2 = T2; m1.t = n; m1.I = c.I; m1.P = c.P; m1.Q = c.Q;
    if (!(use_tc && mode1_tc(m1, status, st))) {
      cudaGetLastError();
      if (use_tc) count_tc_fallback("mode-1 contraction");
      mode1_simt(m1, st);
    }
    mode3_accumulate(T2, W_all + k0 * Qd, Z, n, c.P, c.Q, c.S, Qd, st);
  }
  int flags = 0;
  if (cudaMemcpyAsync(&flags, status, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess) {
    cudaGetLastError();
    return OCTEN_ECUDA;
  }
  // a launch refused above (a grid or resource limit) leaves Z incomplete
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    fprintf(stderr, "octen_compress_noalloc: %s\n", cudaGetErrorString(e));
    return OCTEN_ECUDA;
  }
  if (flags & kDevTimeout) return OCTEN_ETIMEOUT;
  return OCTEN_OK;
}
