"""Plain FP64 oracle of the OCTen online CP update (test infrastructure).

TEST INFRASTRUCTURE ONLY: imported by `tests/`, by `__graft_entry__.smoke()`
and by the CPU-baseline leg of `bench.py`, never by the library.  numpy float64
throughout; library primitives (matmul, tensordot, Cholesky, pinv) serve as
single steps, with no blocking, fusion or reordering beyond what each step's
definition states.

Readings of the paper that this file follows:

* Eq. 2's garbled "(+) Z_p (.) W'_p(k, q)" is the update X_p = Y_p + Z_p with
  Z_p = X_new x1 U_p^T x2 V_p^T x3 W_p^T (only summaries are stored).
* U_p, V_p are fixed for the whole stream; only W rows are drawn per batch.
* The anchors are the first S columns of every projection (Eq. 1).
* CP(X_p, R) of Algorithm 1 is CP-ALS with a warm start U_p^T A_prev,
  V_p^T B_prev (unit-l2 columns), sweep order C, A, B, a fixed number of
  sweeps and one final C update so that C carries the scale.
* Factor match (Sec. "Factor match for identifiability", Eq. 5): similarity of
  anchor rows against the previous global factors' anchor blocks, greedy
  permutation, least-squares anchor scales applied to A and B and their
  product to C (this replaces lambda^(1/N)).
* Eq. 7's P^-1 is the Moore-Penrose pseudo-inverse, applied as the
  minimum-change update A = A_prev + pinv(P_a) (A_s - P_a A_prev); C_old is
  kept and the new rows solve the least-squares system built from the stacked
  W_new,p^T and the replicas' C blocks minus G_p = W_old,p^T C_old.

parity pinned: every public function has a pin in tests/test_oracle_pins.py.
"""
from __future__ import annotations

import itertools

import numpy as np


# ----------------------------------------------------------------------------
# Eq. 1: replica p's projection = [shared anchors | its private columns]
# ----------------------------------------------------------------------------
def replica_block(M_all: np.ndarray, p: int, Q: int, S: int) -> np.ndarray:
    """Columns of replica p out of an all-replica matrix with Qd = S + P(Q-S)
    columns: the shared block [0, S) followed by [S + p(Q-S), S + (p+1)(Q-S))
    (Eq. 1, u / v / w shared by every replica)."""
    lo = S + p * (Q - S)
    return np.concatenate([M_all[:, :S], M_all[:, lo:lo + (Q - S)]], axis=1)


# ----------------------------------------------------------------------------
# Sec. "Parallel Compression and Decomposition": Z_p = X x1 U^T x2 V^T x3 W^T
# ----------------------------------------------------------------------------
def compress(X: np.ndarray, U: np.ndarray, V: np.ndarray, W: np.ndarray) -> np.ndarray:
    """Summary of a slice batch X (stored [k][i][j], K x I x J).

    Z[a, b, c] = sum_{i,j,k} X[k, i, j] U[i, a] V[j, b] W[k, c]  (the three
    mode products of the compression step), evaluated mode 2 (j), then mode 1
    (i), then the time mode (k).  Returns Z indexed [a][b][c].
    """
    X = np.asarray(X, dtype=np.float64)
    T = np.tensordot(X, V, axes=([2], [0]))       # [k, i, b]
    T = np.tensordot(T, U, axes=([1], [0]))       # [k, b, a]
    Z = np.tensordot(T, W, axes=([0], [0]))       # [b, a, c]
    return np.ascontiguousarray(Z.transpose(1, 0, 2))


# ----------------------------------------------------------------------------
# CP model helpers (Sec. "Preliminaries")
# ----------------------------------------------------------------------------
def khatri_rao(F: np.ndarray, G: np.ndarray) -> np.ndarray:
    """Column-wise Kronecker product, row index f * rows(G) + g."""
    R = F.shape[1]
    return (F[:, None, :] * G[None, :, :]).reshape(-1, R)


def mttkrp(X: np.ndarray, F: tuple, mode: int) -> np.ndarray:
    """Matricised tensor times Khatri-Rao product for a 3-way X[a][b][c].

    mode 0: M[a, r] = sum_{b,c} X[a,b,c] F_b[b,r] F_c[c,r]  (F = (F_b, F_c))
    mode 1: M[b, r] = sum_{a,c} X[a,b,c] F_a[a,r] F_c[c,r]  (F = (F_a, F_c))
    mode 2: M[c, r] = sum_{a,b} X[a,b,c] F_a[a,r] F_b[b,r]  (F = (F_a, F_b))
    i.e. X_(n) times the Khatri-Rao product of the other two factors.
    """
    Qa, Qb, Qc = X.shape
    if mode == 0:
        return X.reshape(Qa, Qb * Qc) @ khatri_rao(F[0], F[1])
    if mode == 1:
        Xm = X.transpose(1, 0, 2).reshape(Qb, Qa * Qc)
        return Xm @ khatri_rao(F[0], F[1])
    if mode == 2:
        Xm = X.reshape(Qa * Qb, Qc).T
        return Xm @ khatri_rao(F[0], F[1])
    raise ValueError(mode)


def _normal_solve(M: np.ndarray, Gm: np.ndarray) -> np.ndarray:
    """Least-squares factor update F = M Gm^-1 with Gm the R x R Hadamard
    product of Grams, by Cholesky; if the factorisation fails, the diagonal is
    loaded by 1e-12 * trace / R and the factorisation retried once."""
    try:
        L = np.linalg.cholesky(Gm)
    except np.linalg.LinAlgError:
        R = Gm.shape[0]
        L = np.linalg.cholesky(Gm + (1e-12 * np.trace(Gm) / R) * np.eye(R))
    Y = np.linalg.solve(L, M.T)          # L y = m
    return np.linalg.solve(L.T, Y).T     # L^T f = y


def _unit_columns(F: np.ndarray) -> np.ndarray:
    n = np.linalg.norm(F, axis=0)
    n = np.where(n > 0.0, n, 1.0)
    return F / n


def cp_als(X: np.ndarray, A0: np.ndarray, B0: np.ndarray, iters: int,
           history: list | None = None):
    """CP(X_p, R) of Algorithm 1 as alternating least squares.

    Warm start: unit-l2 columns of A0, B0.  Each of `iters` sweeps updates
    C = M_3 (A^T A * B^T B)^-1, then A = M_1 (B^T B * C^T C)^-1 and B =
    M_2 (A^T A * C^T C)^-1, normalising the columns of A and B to unit l2;
    a final C update after the last sweep carries the scale.  `history`, if
    given, receives (step, A, B, C) right after every least-squares solve,
    before the solved factor is normalised (for pins).
    """
    A = _unit_columns(np.asarray(A0, dtype=np.float64))
    B = _unit_columns(np.asarray(B0, dtype=np.float64))
    C = None
    for _ in range(iters):
        M = mttkrp(X, (A, B), 2)
        Gm = (A.T @ A) * (B.T @ B)
        C = _normal_solve(M, Gm)
        if history is not None:
            history.append(("C", A.copy(), B.copy(), C.copy()))
        M = mttkrp(X, (B, C), 0)
        Gm = (B.T @ B) * (C.T @ C)
        A = _normal_solve(M, Gm)
        if history is not None:
            history.append(("A", A.copy(), B.copy(), C.copy()))
        A = _unit_columns(A)
        M = mttkrp(X, (A, C), 1)
        Gm = (A.T @ A) * (C.T @ C)
        B = _normal_solve(M, Gm)
        if history is not None:
            history.append(("B", A.copy(), B.copy(), C.copy()))
        B = _unit_columns(B)
    M = mttkrp(X, (A, B), 2)
    Gm = (A.T @ A) * (B.T @ B)
    C = _normal_solve(M, Gm)
    if history is not None:
        history.append(("C", A.copy(), B.copy(), C.copy()))
    return A, B, C


def decompose_existing(X_old: np.ndarray, A0: np.ndarray, B0: np.ndarray, iters: int):
    """The existing decomposition when none is supplied (the paper assumes one
    exists, Sec. "Problem Formulation"): cp_als of the existing tensor, whose
    slices X_old[k] are I x J, in the mode order (i, j, k) of the model
    X_old[k][i][j] = sum_r A[i][r] B[j][r] C[k][r], from the guesses A0, B0."""
    return cp_als(np.transpose(np.asarray(X_old, dtype=np.float64), (1, 2, 0)), A0, B0, iters)


# ----------------------------------------------------------------------------
# Sec. "Factor match for identifiability" (Eq. 5, Algorithm 1 match loop)
# ----------------------------------------------------------------------------
def align(At: np.ndarray, Bt: np.ndarray, Ct: np.ndarray, ref_a: np.ndarray,
          ref_b: np.ndarray, S: int):
    """Fix the permutation and scale of one replica's factors.

    The anchor rows (first S) of At / Bt are compared with the reference
    anchor blocks ref_a = u^T A_prev, ref_b = v^T B_prev (S x R):
    sim[r, s] = |cos(At[:S, r], ref_a[:, s])| + |cos(Bt[:S, r], ref_b[:, s])|.
    Greedy matching takes the largest similarity among unmatched pairs, ties to
    the lowest s then the lowest r.  Scales are the least-squares anchor fits
    d_a[s] = <At[:S, pi(s)], ref_a[:, s]> / ||ref_a[:, s]||^2 (d_b alike); the
    aligned factors are At[:, pi(s)] / d_a[s], Bt[:, pi(s)] / d_b[s] and
    Ct[:, pi(s)] d_a[s] d_b[s], which leaves the replica's CP product unchanged.
    A zero scale (degenerate anchor block) leaves that column unscaled.
    Returns (Ah, Bh, Ch, perm, d_a, d_b) with perm[s] = pi(s).
    """
    R = At.shape[1]
    sa, sb = At[:S], Bt[:S]

    def cosines(F, G):
        nf = np.linalg.norm(F, axis=0)
        ng = np.linalg.norm(G, axis=0)
        den = np.outer(nf, ng)
        num = F.T @ G
        return np.where(den > 0.0, np.abs(num) / np.where(den > 0.0, den, 1.0), 0.0)

    sim = cosines(sa, ref_a) + cosines(sb, ref_b)         # [r, s]
    perm = -np.ones(R, dtype=np.int64)
    used_r = np.zeros(R, dtype=bool)
    for _ in range(R):
        best, br, bs = -1.0, -1, -1
        for s in range(R):            # ties -> lowest s, then lowest r
            if perm[s] >= 0:
                continue
            for r in range(R):
                if used_r[r]:
                    continue
                if sim[r, s] > best:
                    best, br, bs = sim[r, s], r, s
        perm[bs] = br
        used_r[br] = True

    d_a = np.empty(R)
    d_b = np.empty(R)
    for s in range(R):
        na = ref_a[:, s] @ ref_a[:, s]
        nb = ref_b[:, s] @ ref_b[:, s]
        d_a[s] = (sa[:, perm[s]] @ ref_a[:, s]) / na if na > 0.0 else 0.0
        d_b[s] = (sb[:, perm[s]] @ ref_b[:, s]) / nb if nb > 0.0 else 0.0
        if d_a[s] == 0.0:
            d_a[s] = 1.0
        if d_b[s] == 0.0:
            d_b[s] = 1.0
    Ah = At[:, perm] / d_a
    Bh = Bt[:, perm] / d_b
    Ch = Ct[:, perm] * (d_a * d_b)
    return Ah, Bh, Ch, perm, d_a, d_b


# ----------------------------------------------------------------------------
# Sec. "Update results" (Eq. 6 and Eq. 7)
# ----------------------------------------------------------------------------
def _pinv(M: np.ndarray) -> np.ndarray:
    """Moore-Penrose pseudo-inverse with singular values below
    max(rows, cols) * eps * sigma_max treated as zero (Matlab's default
    tolerance, the environment the paper's solves ran in).  The stacks of
    Eq. 6 repeat the anchor rows once per replica, so they are rank deficient
    by construction and the cut-off decides the answer."""
    return np.linalg.pinv(M, rtol=max(M.shape) * np.finfo(np.float64).eps)


def lift_factor(F_prev: np.ndarray, proj: list, F_hat: list) -> np.ndarray:
    """A (or B) from the aligned replica blocks, Eq. 7.

    P_a stacks U_p^T (pQ x I, the anchor rows repeated per replica, Eq. 6),
    A_s stacks the aligned replica factors (pQ x R).  The update is
    A = A_prev + pinv(P_a) (A_s - P_a A_prev): the least-squares solution of
    P_a A = A_s when P_a has full column rank, the one closest to A_prev
    otherwise.
    """
    Pm = np.vstack([Up.T for Up in proj])
    Fs = np.vstack(F_hat)
    return F_prev + _pinv(Pm) @ (Fs - Pm @ F_prev)


def lift_C(W_new: list, C_hat: list, G: list) -> np.ndarray:
    """New rows of C, Eq. 7's [C_old; P_c^-1 C_s] with C_old held fixed.

    Replica p's temporal factor sees every slice so far: C_hat_p ~ W_old,p^T
    C_old + W_new,p^T C_new = G_p + W_new,p^T C_new.  C_new is the
    least-squares solution of the stacked system (W_new,p^T) C_new = C_hat_p - G_p.
    """
    Pc = np.vstack([Wp.T for Wp in W_new])
    rhs = np.vstack([Ch - Gp for Ch, Gp in zip(C_hat, G)])
    return _pinv(Pc) @ rhs


# ----------------------------------------------------------------------------
# Sec. "Evaluation Measures": fitness
# ----------------------------------------------------------------------------
def fit(X: np.ndarray, A: np.ndarray, B: np.ndarray, C: np.ndarray) -> float:
    """1 - ||X - [[A, B, C]]||_F / ||X||_F over all slices of X[k][i][j]
    (the paper's Fitness(%) divided by 100), reconstructing slice by slice."""
    num = 0.0
    den = 0.0
    for k in range(X.shape[0]):
        Xk = np.asarray(X[k], dtype=np.float64)
        Rk = Xk - (A * C[k]) @ B.T
        num += float(np.sum(Rk * Rk))
        den += float(np.sum(Xk * Xk))
    return 1.0 - np.sqrt(num) / np.sqrt(den)


# ----------------------------------------------------------------------------
# Sec. "Factor match" Eq. 4 and Sec. "Parameter Sensitivity" Eq. 8
# ----------------------------------------------------------------------------
def eq8_min_replicas(I: int, J: int, K: int, Q: int, S: int) -> float:
    """Eq. 8: p >= max((I - shared)/(Q - shared), J/Q, K/Q)."""
    return max((I - S) / (Q - S), J / Q, K / Q)


def _kruskal_rank(F: np.ndarray, tol: float = 1e-9) -> int:
    R = F.shape[1]
    k = 0
    for r in range(1, R + 1):
        ok = True
        for cols in itertools.combinations(range(R), r):
            if np.linalg.matrix_rank(F[:, cols], tol=tol) < r:
                ok = False
                break
        if not ok:
            break
        k = r
    return k


def eq4_identifiable(Q: int, A: np.ndarray, B: np.ndarray, C: np.ndarray) -> bool:
    """Eq. 4: min(Q, k_A) + min(Q, k_B) + min(Q, k_C) >= 2R + 2 with k_F the
    Kruskal rank (brute force over column subsets: small R only)."""
    R = A.shape[1]
    kA, kB, kC = (_kruskal_rank(F) for F in (A, B, C))
    return min(Q, kA) + min(Q, kB) + min(Q, kC) >= 2 * R + 2


# ----------------------------------------------------------------------------
# Algorithm 1: the online update loop
# ----------------------------------------------------------------------------
class OctenOracle:
    """State and steps of Algorithm 1 for a 3-mode tensor growing in mode 3.

    State (Sec. "Complexity Analysis": only compression matrices, factors and
    summaries are kept): Y_p (Q x Q x Q), U_p, V_p, G_p = W_p^T C (Q x R) and
    the global factors A, B, C.
    """

    def __init__(self, I: int, J: int, R: int, P: int, Q: int, S: int, als_iters: int):
        if not (0 <= S <= Q and P >= 1 and R >= 1 and als_iters >= 1):
            raise ValueError("bad configuration")
        self.I, self.J, self.R, self.P, self.Q, self.S = I, J, R, P, Q, S
        self.als_iters = als_iters
        self.last: dict = {}

    def _split(self, M_all: np.ndarray) -> list:
        return [replica_block(M_all, p, self.Q, self.S) for p in range(self.P)]

    def init(self, X_old, U_all, V_all, W_old, A0, B0, C0):
        """Summaries of the existing tensor plus its existing decomposition
        (computed by decompose_existing from A0, B0 when C0 is None)."""
        self.U = self._split(np.asarray(U_all, dtype=np.float64))
        self.V = self._split(np.asarray(V_all, dtype=np.float64))
        W = self._split(np.asarray(W_old, dtype=np.float64))
        self.Y = [compress(X_old, self.U[p], self.V[p], W[p]) for p in range(self.P)]
        if C0 is None:
            # A0, B0 are starting guesses for a CP-ALS of the existing tensor
            A0, B0, C0 = decompose_existing(X_old, A0, B0, self.als_iters)
        self.A = np.asarray(A0, dtype=np.float64).copy()
        self.B = np.asarray(B0, dtype=np.float64).copy()
        self.C = np.asarray(C0, dtype=np.float64).copy()
        self.G = [W[p].T @ self.C for p in range(self.P)]

    def append(self, X_new, W_new):
        """One pass of Algorithm 1's loop body for a batch of new slices."""
        P, S = self.P, self.S
        W = self._split(np.asarray(W_new, dtype=np.float64))
        # compress and update the summaries: X_p = Y_p + Z_p
        for p in range(P):
            self.Y[p] = self.Y[p] + compress(X_new, self.U[p], self.V[p], W[p])
        # CP of every summary, warm-started from the projected previous factors
        A_prev, B_prev = self.A, self.B
        pa = [self.U[p].T @ A_prev for p in range(P)]
        pb = [self.V[p].T @ B_prev for p in range(P)]
        ref_a, ref_b = pa[0][:S], pb[0][:S]
        raw, hat = [], []
        for p in range(P):
            At, Bt, Ct = cp_als(self.Y[p], pa[p], pb[p], self.als_iters)
            raw.append((At, Bt, Ct))
            hat.append(align(At, Bt, Ct, ref_a, ref_b, S))
        # lift A and B, solve the new rows of C, update G_p
        A = lift_factor(A_prev, self.U, [h[0] for h in hat])
        B = lift_factor(B_prev, self.V, [h[1] for h in hat])
        C_new = lift_C(W, [h[2] for h in hat], self.G)
        self.G = [self.G[p] + W[p].T @ C_new for p in range(P)]
        self.A, self.B = A, B
        self.C = np.vstack([self.C, C_new])
        self.last = dict(raw=raw, hat=hat, C_new=C_new, pa=pa, pb=pb)
        return A, B, C_new
