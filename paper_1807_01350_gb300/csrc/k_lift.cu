// The lift of Eq. 7 for one non-temporal mode, shared by the 3-mode and the
// N-mode contexts: the pseudo-inverse of the stacked replica projections,
// applied through a precomputed operator.
//   Qd > rows (P~ has full column rank): L = (U Omega U^T)^-1 U, Omega weighting
//     the anchor columns by P (they appear once per replica in the stack);
//     F = F_prev + L e with e the stack's residual summed over the replicas.
//   Qd <= rows: L = U (U^T U)^-1 over the Qd distinct rows of the stack (stored
//     transposed), e with the anchor rows averaged over the replicas: the
//     minimum-change update.
// fp32 Grams, blocked Cholesky with fp64 diagonal blocks, triangular solves.
#include "octen_internal.cuh"

namespace octen {

bool lift_build(const LiftEnv &v, const float *Ur, int64_t rows, float *L, int &over) {
  const int Qd = v.Qd;
  over = Qd > rows ? 1 : 0;
  const int n = over ? (int)rows : Qd;
  float *Gm = nullptr;
  if (cudaMalloc(&Gm, (size_t)n * n * sizeof(float)) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  float *Uw = nullptr;
  GemmArgs g{};
  g.ta = Elem::F32; g.tb = Elem::F32; g.batch = 1; g.alpha = 1.f; g.beta = 0.f;
  g.D = Gm; g.sDm = n; g.sDn = 1; g.M = n; g.N = n;
  if (over) {
    if (cudaMalloc(&Uw, (size_t)rows * Qd * sizeof(float)) != cudaSuccess) {
      cudaGetLastError();
      cudaFree(Gm);
      return false;
    }
    scale_columns(Ur, rows, Qd, v.S, (float)v.P, Uw, v.st);
    g.A = Ur; g.sAm = Qd; g.sAk = 1;
    g.B = Uw; g.sBn = Qd; g.sBk = 1;
    g.K = Qd;
    gemm_strided(g, v.st);
    cholesky_f32(Gm, n, v.status, v.st);
    cudaMemcpyAsync(L, Ur, (size_t)rows * Qd * sizeof(float), cudaMemcpyDeviceToDevice, v.st);
    chol_solve_f32(Gm, n, L, Qd, v.st);
  } else {
    g.A = Ur; g.sAm = 1; g.sAk = Qd;
    g.B = Ur; g.sBn = 1; g.sBk = Qd;
    g.K = (int)rows;
    gemm_strided(g, v.st);
    cholesky_f32(Gm, n, v.status, v.st);
    transpose_f32(Ur, rows, Qd, L, v.st);   // L <- U^T (Qd x rows)
    chol_solve_f32(Gm, n, L, (int)rows, v.st);
  }
  const bool ok = cudaStreamSynchronize(v.st) == cudaSuccess;
  cudaFree(Gm);
  if (Uw) cudaFree(Uw);
  return ok;
}

void lift_apply(const LiftEnv &v, const float *Fh, const float *PF, const float *L, int over,
                int64_t rows, float *F) {
  lift_rhs(Fh, PF, v.P, v.Q, v.S, v.R, v.RT, v.Qd, over, v.e, v.st);
  GemmArgs g{};
  g.A = L; g.ta = Elem::F32;
  if (over) { g.sAm = v.Qd; g.sAk = 1; } else { g.sAm = 1; g.sAk = rows; }
  g.B = v.e; g.tb = Elem::F32; g.sBn = 1; g.sBk = v.R;
  g.D = F; g.sDm = v.R; g.sDn = 1;
  g.M = (int)rows; g.N = v.R; g.K = v.Qd; g.batch = 1; g.alpha = 1.f; g.beta = 1.f;
  g.split_scratch = v.splitk; g.split_scratch_floats = v.splitk_floats;
  gemm_strided(g, v.st);
}

}  // namespace octen
