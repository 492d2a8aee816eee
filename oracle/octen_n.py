"""Plain FP64 oracle of the N-mode online CP update (test infrastructure).

TEST INFRASTRUCTURE ONLY: imported by `tests/` and `bench.py`'s CPU legs,
never by the library.  Follows Sec. "Extending to Higher-Order Tensors" of the
paper: the existing tensor has N - 1 non-temporal modes I_1 x ... x I_{N-1}
and a time mode; every replica p compresses every mode with its own
projection (the first S columns shared, Eq. 1), summaries add up
(X_p = Y_p + Z_p), each summary gets a CP decomposition, the replicas are
matched on their anchor rows in every non-temporal mode, and every
non-temporal factor is lifted as in Eq. 7 with its own stacked projection, the
new rows of the time factor as in the 3-mode case.

Readings: the same as the 3-mode oracle's, mode by mode;
one Q and one S for all modes; the CP sweep updates the time factor first,
then the non-temporal factors in mode order (each normalised to unit l2),
with a final time-factor update; the match similarity is the sum over the
non-temporal modes of |cos| between anchor blocks, the time factor's columns
are scaled by the product of the per-mode anchor scales.

Slices are stored time first, X[k][i_1]...[i_{N-1}]; summaries are indexed
[q_1]...[q_{N-1}][c] (time last).  With N = 3 every function here equals its
3-mode counterpart in octen.py (pinned in tests/test_oracle_pins_nmode.py).
"""
from __future__ import annotations

import numpy as np

from .octen import _normal_solve, _unit_columns, khatri_rao, lift_C, lift_factor, replica_block


def compress_n(X: np.ndarray, Us: list, W: np.ndarray) -> np.ndarray:
    """Z[q_1, ..., q_{N-1}, c] = sum X[k, i_1, ..., i_{N-1}] prod_n U_n[i_n, q_n]
    W[k, c]: the N mode products of the compression, the last non-temporal mode
    first, the time mode last."""
    T = np.asarray(X, dtype=np.float64)
    n_sp = T.ndim - 1
    for n in range(n_sp, 0, -1):            # contract i_n (axis n), append q_n at the end
        T = np.tensordot(T, Us[n - 1], axes=([n], [0]))
    # axes now: k, q_{N-1}, ..., q_1
    Z = np.tensordot(T, W, axes=([0], [0]))  # q_{N-1}, ..., q_1, c
    order = list(range(n_sp - 1, -1, -1)) + [n_sp]
    return np.ascontiguousarray(Z.transpose(order))


def khatri_rao_list(Fs: list) -> np.ndarray:
    """Khatri-Rao product of several factors, the first one varying slowest."""
    out = Fs[0]
    for F in Fs[1:]:
        out = khatri_rao(out, F)
    return out


def mttkrp_n(X: np.ndarray, Fs: list, mode: int) -> np.ndarray:
    """M[q, r] = sum over the other indices of X times the product of the other
    factors' rows: X unfolded along `mode` (the remaining axes in order) times
    the Khatri-Rao product of the other factors in the same order.  Fs holds
    one factor per mode of X (the entry for `mode` is ignored)."""
    Xm = np.moveaxis(X, mode, 0).reshape(X.shape[mode], -1)
    others = [Fs[m] for m in range(X.ndim) if m != mode]
    return Xm @ khatri_rao_list(others)


def cp_als_n(X: np.ndarray, F0: list, iters: int) -> list:
    """CP of an N-way summary X[q_1..q_{N-1}, c] by alternating least squares.
    Warm start: unit-l2 columns of the non-temporal guesses F0 (N - 1 of them).
    Each sweep updates the time factor, then the non-temporal factors in mode
    order (normalised to unit l2); a final time-factor update carries the
    scale.  Returns [F_1, ..., F_{N-1}, C]."""
    n_sp = X.ndim - 1
    Fs = [_unit_columns(np.asarray(F, dtype=np.float64)) for F in F0] + [None]

    def update(mode):
        M = mttkrp_n(X, Fs, mode)
        Gm = np.ones((M.shape[1], M.shape[1]))
        for m in range(X.ndim):
            if m != mode:
                Gm = Gm * (Fs[m].T @ Fs[m])
        return _normal_solve(M, Gm)

    for _ in range(iters):
        Fs[n_sp] = update(n_sp)
        for n in range(n_sp):
            Fs[n] = _unit_columns(update(n))
    Fs[n_sp] = update(n_sp)
    return Fs


def align_n(Fs: list, C: np.ndarray, refs: list, S: int):
    """Permutation and scale of one replica (the 3-mode match, mode by mode):
    sim[r, s] = sum_n |cos(F_n[:S, r], ref_n[:, s])|, greedy matching (largest
    first, ties to the lowest s then r), least-squares anchor scales d_n[s]
    (0 -> 1); F_n[:, pi] / d_n and C[:, pi] * prod_n d_n.
    Returns (F_hat list, C_hat, perm)."""
    R = C.shape[1]

    def cosines(F, G):
        nf = np.linalg.norm(F, axis=0)
        ng = np.linalg.norm(G, axis=0)
        den = np.outer(nf, ng)
        num = F.T @ G
        return np.where(den > 0.0, np.abs(num) / np.where(den > 0.0, den, 1.0), 0.0)

    sim = sum(cosines(F[:S], ref) for F, ref in zip(Fs, refs))
    perm = -np.ones(R, dtype=np.int64)
    used_r = np.zeros(R, dtype=bool)
    for _ in range(R):
        best, br, bs = -1.0, -1, -1
        for s in range(R):
            if perm[s] >= 0:
                continue
            for r in range(R):
                if used_r[r]:
                    continue
                if sim[r, s] > best:
                    best, br, bs = sim[r, s], r, s
        perm[bs] = br
        used_r[br] = True
    Fh = []
    scale_c = np.ones(R)
    for F, ref in zip(Fs, refs):
        d = np.empty(R)
        for s in range(R):
            n2 = ref[:, s] @ ref[:, s]
            d[s] = (F[:S, perm[s]] @ ref[:, s]) / n2 if n2 > 0.0 else 0.0
            if d[s] == 0.0:
                d[s] = 1.0
        Fh.append(F[:, perm] / d)
        scale_c = scale_c * d
    return Fh, C[:, perm] * scale_c, perm


def decompose_existing_n(X_old: np.ndarray, A0s: list, iters: int) -> list:
    """The existing decomposition when none is supplied (the paper assumes one
    exists, Sec. "Problem Formulation"): cp_als_n of the existing tensor, whose
    slices X_old[k] are I_1 x ... x I_{N-1}, in the mode order (i_1, ..., k) of
    the model X_old[k][i..] = sum_r prod_n A_n[i_n][r] C[k][r], from the guesses
    A0s.  Returns [A_1, ..., A_{N-1}, C]."""
    X = np.asarray(X_old, dtype=np.float64)
    order = list(range(1, X.ndim)) + [0]
    return cp_als_n(np.transpose(X, order), A0s, iters)


def fit_n(X: np.ndarray, As: list, C: np.ndarray) -> float:
    """1 - ||X - [[A_1, ..., A_{N-1}, C]]||_F / ||X||_F, X[k][i_1]...[i_{N-1}]."""
    num = 0.0
    den = 0.0
    for k in range(X.shape[0]):
        Xk = np.asarray(X[k], dtype=np.float64)
        model = khatri_rao_list(As) @ C[k]
        Rk = Xk.reshape(-1) - model
        num += float(Rk @ Rk)
        den += float(np.sum(Xk * Xk))
    return 1.0 - np.sqrt(num) / np.sqrt(den)


class OctenOracleN:
    """Algorithm 1 for an N-mode tensor growing in its time mode (the paper's
    higher-order extension).  State: the summaries Y_p, the projections of every
    non-temporal mode, G_p = W_p^T C and the global factors."""

    def __init__(self, dims: list, R: int, P: int, Q: int, S: int, als_iters: int):
        self.dims = list(dims)
        self.R, self.P, self.Q, self.S, self.als_iters = R, P, Q, S, als_iters
        self.last = {}

    def _split(self, M_all):
        return [replica_block(M_all, p, self.Q, self.S) for p in range(self.P)]

    def init(self, X_old, Us_all: list, W_old, A0s: list, C0):
        self.U = [self._split(np.asarray(U, dtype=np.float64)) for U in Us_all]   # [mode][p]
        W = self._split(np.asarray(W_old, dtype=np.float64))
        self.Y = [compress_n(X_old, [self.U[n][p] for n in range(len(self.dims))], W[p])
                  for p in range(self.P)]
        if C0 is None:   # A0s are starting guesses: decompose the existing tensor
            out = decompose_existing_n(X_old, A0s, self.als_iters)
            self.A, self.C = out[:-1], out[-1]
        else:
            self.A = [np.asarray(A, dtype=np.float64).copy() for A in A0s]
            self.C = np.asarray(C0, dtype=np.float64).copy()
        self.G = [W[p].T @ self.C for p in range(self.P)]

    def append(self, X_new, W_new):
        P, S, nm = self.P, self.S, len(self.dims)
        W = self._split(np.asarray(W_new, dtype=np.float64))
        for p in range(P):
            self.Y[p] = self.Y[p] + compress_n(X_new, [self.U[n][p] for n in range(nm)], W[p])
        proj = [[self.U[n][p].T @ self.A[n] for p in range(P)] for n in range(nm)]
        refs = [proj[n][0][:S] for n in range(nm)]
        raw, hat = [], []
        for p in range(P):
            Fs = cp_als_n(self.Y[p], [proj[n][p] for n in range(nm)], self.als_iters)
            raw.append(Fs)
            hat.append(align_n(Fs[:nm], Fs[nm], refs, S))
        self.A = [lift_factor(self.A[n], self.U[n], [h[0][n] for h in hat]) for n in range(nm)]
        C_new = lift_C(W, [h[1] for h in hat], self.G)
        self.C = np.vstack([self.C, C_new])
        self.G = [self.G[p] + W[p].T @ C_new for p in range(P)]
        self.last = {"raw": raw, "hat": hat}
