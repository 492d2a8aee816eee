"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each pin checks the oracle by a route other than its own code: brute-force
loops on tiny tensors, the Kronecker / Khatri-Rao closed form of the
compression of an exact CP tensor (Sec. "Factor match", the identity
(U^T (x) V^T (x) W^T)(A (.) B (.) C) = (U^T A) (.) (V^T B) (.) (W^T C)), linearity of
the summaries (X_p = Y_p + Z_p), least-squares optimality of every ALS step
checked through an explicit residual gradient and numpy's lstsq, the
higher-order power method for R = 1, exact recovery of planted factors by
the lift (Eq. 7), and the worked example of Eq. 8.
"""
import itertools
import json
import os

import numpy as np
import pytest

import oracle
from oracle import octen as O
from synth import factors, init_factors, projections, slice_batch, time_projection
from tests._metrics import fms, rel_fro

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def cp_tensor(A, B, C):
    """[[A, B, C]] indexed [a][b][c] by an explicit sum of outer products."""
    out = np.zeros((A.shape[0], B.shape[0], C.shape[0]))
    for r in range(A.shape[1]):
        out += np.multiply.outer(np.multiply.outer(A[:, r], B[:, r]), C[:, r])
    return out


# ---------------------------------------------------------------- compression
def test_compress_bruteforce_six_loops():
    rng = np.random.default_rng(1)
    K, I, J, Qa, Qb, Qc = 3, 5, 6, 4, 3, 2
    X = rng.standard_normal((K, I, J))
    U = rng.standard_normal((I, Qa))
    V = rng.standard_normal((J, Qb))
    W = rng.standard_normal((K, Qc))
    Z = oracle.compress(X, U, V, W)
    ref = np.zeros((Qa, Qb, Qc))
    for a in range(Qa):
        for b in range(Qb):
            for c in range(Qc):
                s = 0.0
                for k in range(K):
                    for i in range(I):
                        for j in range(J):
                            s += X[k, i, j] * U[i, a] * V[j, b] * W[k, c]
                ref[a, b, c] = s
    assert rel_fro(Z, ref) < 1e-13


def test_compress_exact_cp_closed_form():
    """Compressing an exact rank-R tensor gives the CP of (U^T A, V^T B, W^T C)."""
    rng = np.random.default_rng(2)
    I, J, K, R, Q = 9, 8, 7, 3, 5
    A, B, C = (rng.standard_normal((n, R)) for n in (I, J, K))
    X = np.einsum("ir,jr,kr->kij", A, B, C)
    U, V, W = (rng.standard_normal((n, Q)) for n in (I, J, K))
    Z = oracle.compress(X, U, V, W)
    assert rel_fro(Z, cp_tensor(U.T @ A, V.T @ B, W.T @ C)) < 1e-12


def test_compress_linear_in_slices():
    """Y(X_old) + Z(X_new) equals the summary of [X_old; X_new] with [W_old; W_new]."""
    rng = np.random.default_rng(3)
    I, J, Q = 6, 7, 4
    Xo, Xn = rng.standard_normal((5, I, J)), rng.standard_normal((3, I, J))
    U, V = rng.standard_normal((I, Q)), rng.standard_normal((J, Q))
    Wo, Wn = rng.standard_normal((5, Q)), rng.standard_normal((3, Q))
    both = oracle.compress(np.concatenate([Xo, Xn]), U, V, np.concatenate([Wo, Wn]))
    assert rel_fro(oracle.compress(Xo, U, V, Wo) + oracle.compress(Xn, U, V, Wn), both) < 1e-13


def test_replica_block_shares_anchor_columns():
    M = np.arange(2 * (3 + 4 * 2)).reshape(2, 11).astype(float)   # S=3, P=4, Q=5
    blocks = [oracle.replica_block(M, p, 5, 3) for p in range(4)]
    for p, b in enumerate(blocks):
        assert b.shape == (2, 5)
        assert np.array_equal(b[:, :3], M[:, :3])
        assert np.array_equal(b[:, 3:], M[:, 3 + 2 * p:5 + 2 * p])


# ---------------------------------------------------------------- MTTKRP / ALS
def test_mttkrp_bruteforce():
    rng = np.random.default_rng(4)
    Qa, Qb, Qc, R = 3, 4, 5, 2
    X = rng.standard_normal((Qa, Qb, Qc))
    A, B, C = (rng.standard_normal((n, R)) for n in (Qa, Qb, Qc))
    ref0 = np.zeros((Qa, R))
    ref1 = np.zeros((Qb, R))
    ref2 = np.zeros((Qc, R))
    for a, b, c, r in itertools.product(range(Qa), range(Qb), range(Qc), range(R)):
        ref0[a, r] += X[a, b, c] * B[b, r] * C[c, r]
        ref1[b, r] += X[a, b, c] * A[a, r] * C[c, r]
        ref2[c, r] += X[a, b, c] * A[a, r] * B[b, r]
    assert rel_fro(oracle.mttkrp(X, (B, C), 0), ref0) < 1e-13
    assert rel_fro(oracle.mttkrp(X, (A, C), 1), ref1) < 1e-13
    assert rel_fro(oracle.mttkrp(X, (A, B), 2), ref2) < 1e-13


def _als_case(seed=5, Q=7, R=3, noise=0.2):
    rng = np.random.default_rng(seed)
    A, B, C = (rng.standard_normal((Q, R)) for _ in range(3))
    X = cp_tensor(A, B, C) + noise * rng.standard_normal((Q, Q, Q))
    A0 = A + 0.3 * rng.standard_normal(A.shape)
    B0 = B + 0.3 * rng.standard_normal(B.shape)
    return X, A0, B0


def test_als_every_step_is_least_squares_optimal():
    """Each solved factor zeroes the gradient of ||X - [[A,B,C]]||^2 in that
    factor (explicit residual tensor), and equals numpy's lstsq on the
    unfolded problem with an explicitly looped Khatri-Rao matrix."""
    X, A0, B0 = _als_case()
    hist = []
    oracle.cp_als(X, A0, B0, 4, history=hist)
    Q, R = A0.shape
    for step, A, B, C in hist:
        E = X - cp_tensor(A, B, C)
        if step == "A":
            g = np.einsum("abc,br,cr->ar", E, B, C)
            F, others = A, (B, C)
            Xu = X.reshape(Q, Q * Q)
        elif step == "B":
            g = np.einsum("abc,ar,cr->br", E, A, C)
            F, others = B, (A, C)
            Xu = X.transpose(1, 0, 2).reshape(Q, Q * Q)
        else:
            g = np.einsum("abc,ar,br->cr", E, A, B)
            F, others = C, (A, B)
            Xu = X.reshape(Q * Q, Q).T
        scale = np.linalg.norm(np.einsum("abc,br,cr->ar", X, B, C)) + 1.0
        assert np.linalg.norm(g) / scale < 1e-10, step
        KR = np.zeros((Q * Q, R))
        for f in range(Q):
            for h in range(Q):
                KR[f * Q + h] = others[0][f] * others[1][h]
        ls = np.linalg.lstsq(KR, Xu.T, rcond=None)[0].T
        assert rel_fro(F, ls) < 1e-9, step


def test_als_objective_non_increasing():
    X, A0, B0 = _als_case(seed=6, noise=0.5)
    hist = []
    oracle.cp_als(X, A0, B0, 8, history=hist)
    obj = [np.linalg.norm(X - cp_tensor(A, B, C)) for _, A, B, C in hist]
    for f0, f1 in zip(obj, obj[1:]):
        assert f1 <= f0 * (1 + 1e-12)


def test_als_noiseless_planted_fit_one():
    rng = np.random.default_rng(7)
    Q, R = 10, 4
    A, B, C = (rng.standard_normal((Q, R)) for _ in range(3))
    X = cp_tensor(A, B, C)
    At, Bt, Ct = oracle.cp_als(X, A + 0.1 * rng.standard_normal(A.shape),
                               B + 0.1 * rng.standard_normal(B.shape), 200)
    Xk = X.transpose(2, 0, 1)   # [c][a][b] slices for the fit routine
    assert oracle.fit(Xk, At, Bt, Ct) > 1 - 1e-10
    assert fms((At, Bt, Ct), (A, B, C)) > 1 - 1e-9


def test_als_rank_one_is_power_method():
    """With R = 1 the sweeps are the higher-order power method."""
    rng = np.random.default_rng(8)
    Q = 6
    X = rng.standard_normal((Q, Q, Q))
    a0, b0 = rng.standard_normal((Q, 1)), rng.standard_normal((Q, 1))
    At, Bt, Ct = oracle.cp_als(X, a0, b0, 25)
    a, b = a0[:, 0] / np.linalg.norm(a0), b0[:, 0] / np.linalg.norm(b0)
    for _ in range(25):
        c = np.einsum("abc,a,b->c", X, a, b)
        c = c / np.linalg.norm(c)
        a = np.einsum("abc,b,c->a", X, b, c)
        a = a / np.linalg.norm(a)
        b = np.einsum("abc,a,c->b", X, a, c)
        b = b / np.linalg.norm(b)
    lam_c = np.einsum("abc,a,b->c", X, a, b)
    assert np.allclose(At[:, 0], a, atol=1e-12)
    assert np.allclose(Bt[:, 0], b, atol=1e-12)
    assert np.allclose(Ct[:, 0], lam_c, atol=1e-10)


# ---------------------------------------------------------------- alignment
def test_align_recovers_known_permutation_and_scales():
    rng = np.random.default_rng(9)
    Q, S, R = 12, 6, 5
    Ah, Bh, Ch = (rng.standard_normal((Q, R)) for _ in range(3))
    perm = np.array([3, 0, 4, 1, 2])            # column s of the truth sits at perm[s]
    d_a = np.array([2.0, -0.5, 3.0, 1.5, -4.0])
    d_b = np.array([-1.0, 0.25, 2.0, -3.0, 0.5])
    At, Bt, Ct = np.empty_like(Ah), np.empty_like(Bh), np.empty_like(Ch)
    At[:, perm] = Ah * d_a
    Bt[:, perm] = Bh * d_b
    Ct[:, perm] = Ch / (d_a * d_b)
    A2, B2, C2, p2, da2, db2 = oracle.align(At, Bt, Ct, Ah[:S], Bh[:S], S)
    assert np.array_equal(p2, perm)
    assert np.allclose(da2, d_a, rtol=1e-12) and np.allclose(db2, d_b, rtol=1e-12)
    for x, y in ((A2, Ah), (B2, Bh), (C2, Ch)):
        assert rel_fro(x, y) < 1e-12
    # the replica's CP product is unchanged by the alignment
    assert rel_fro(cp_tensor(A2, B2, C2), cp_tensor(At, Bt, Ct)) < 1e-12


def test_align_greedy_matches_bruteforce_on_separated_columns():
    rng = np.random.default_rng(10)
    Q, S, R = 10, 6, 5
    for trial in range(20):
        ref_a, ref_b = rng.standard_normal((S, R)), rng.standard_normal((S, R))
        perm = rng.permutation(R)
        At = np.zeros((Q, R))
        Bt = np.zeros((Q, R))
        At[:S, perm] = ref_a + 0.05 * rng.standard_normal((S, R))
        Bt[:S, perm] = ref_b + 0.05 * rng.standard_normal((S, R))
        At[S:], Bt[S:] = rng.standard_normal((Q - S, R)), rng.standard_normal((Q - S, R))
        _, _, _, p, _, _ = oracle.align(At, Bt, np.ones((3, R)), ref_a, ref_b, S)

        def cosm(F, G):
            return np.abs(F.T @ G) / np.outer(np.linalg.norm(F, axis=0), np.linalg.norm(G, axis=0))
        sim = cosm(At[:S], ref_a) + cosm(Bt[:S], ref_b)
        best = max(itertools.permutations(range(R)),
                   key=lambda q: sum(sim[q[s], s] for s in range(R)))
        assert np.array_equal(p, np.array(best)), trial


def test_align_ties_and_degenerate_scales_follow_the_reading():
    # Orthonormal anchor references; replica column r points at reference
    # column sigma(r), with two replica columns on the same reference column:
    # sim[r, s] = 2 where sigma(r) = s, else 0.  The greedy rule (largest
    # similarity, ties to the lowest s, then the lowest r) then gives, by hand:
    # s = 0 <- r = 3, s = 1 <- r = 0 (r = 1 ties and loses), s = 3 <- r = 2,
    # and the left-over s = 2 <- r = 1 at similarity 0.  Column 1's anchor block
    # is orthogonal to reference column 2, so its least-squares scale is 0 and
    # the column stays unscaled.
    Q, S, R = 7, 4, 4
    E = np.eye(S)
    sigma = [1, 1, 3, 0]
    At = np.zeros((Q, R))
    Bt = np.zeros((Q, R))
    for r, s in enumerate(sigma):
        At[:S, r] = 2.0 * E[:, s]
        Bt[:S, r] = -3.0 * E[:, s]
    At[S:] = np.arange((Q - S) * R, dtype=float).reshape(Q - S, R)
    Bt[S:] = 1.0
    Ct = np.arange(3 * R, dtype=float).reshape(3, R) + 1.0
    Ah, Bh, Ch, perm, d_a, d_b = oracle.align(At, Bt, Ct, E, E, S)
    assert perm.tolist() == [3, 0, 1, 2]
    assert d_a.tolist() == [2.0, 2.0, 1.0, 2.0]
    assert d_b.tolist() == [-3.0, -3.0, 1.0, -3.0]
    assert np.array_equal(Ah, At[:, perm] / d_a)
    assert np.array_equal(Ch, Ct[:, perm] * (d_a * d_b))


# ---------------------------------------------------------------- lifting
def _lift_case(I, P, Q, S, R, seed):
    rng = np.random.default_rng(seed)
    Qd = S + P * (Q - S)
    U_all = rng.standard_normal((I, Qd))
    U = [oracle.replica_block(U_all, p, Q, S) for p in range(P)]
    A = rng.standard_normal((I, R))
    return U, A, rng


def test_lift_exact_recovery_when_eq8_holds():
    """Full column rank stack (Qd >= I): the lift returns the planted A from
    exact replica blocks whatever A_prev was."""
    I, P, Q, S, R = 20, 4, 8, 2, 3          # Qd = 26 >= 20
    U, A, rng = _lift_case(I, P, Q, S, R, 11)
    hats = [Up.T @ A for Up in U]
    for A_prev in (np.zeros((I, R)), rng.standard_normal((I, R))):
        assert rel_fro(oracle.lift_factor(A_prev, U, hats), A) < 1e-10


def test_lift_minimum_change_when_underdetermined():
    """Qd < I: the update satisfies every replica block exactly and moves
    A_prev only within the row space of the stacked projections."""
    I, P, Q, S, R = 30, 3, 8, 2, 3          # Qd = 20 < 30
    U, A, rng = _lift_case(I, P, Q, S, R, 12)
    A_prev = rng.standard_normal((I, R))
    hats = [Up.T @ A for Up in U]
    A_new = oracle.lift_factor(A_prev, U, hats)
    for Up, h in zip(U, hats):
        assert rel_fro(Up.T @ A_new, h) < 1e-10
    # the distinct rows of the stack are the columns of [u, U_1', ..., U_P']
    distinct = np.hstack([U[0]] + [Up[:, S:] for Up in U[1:]])
    q, _ = np.linalg.qr(distinct)           # orthonormal basis of the row space
    delta = A_new - A_prev
    assert rel_fro(q @ (q.T @ delta), delta) < 1e-10


def test_lift_C_exact_new_rows():
    rng = np.random.default_rng(13)
    P, Q, S, R, t_old, t = 3, 6, 2, 2, 5, 4
    Qd = S + P * (Q - S)
    C_old, C_new = rng.standard_normal((t_old, R)), rng.standard_normal((t, R))
    W_old_all, W_new_all = rng.standard_normal((t_old, Qd)), rng.standard_normal((t, Qd))
    Wo = [oracle.replica_block(W_old_all, p, Q, S) for p in range(P)]
    Wn = [oracle.replica_block(W_new_all, p, Q, S) for p in range(P)]
    G = [w.T @ C_old for w in Wo]
    hats = [np.vstack([a, b]).T @ np.vstack([C_old, C_new]) for a, b in zip(Wo, Wn)]
    assert rel_fro(oracle.lift_C(Wn, hats, G), C_new) < 1e-10


# ---------------------------------------------------------------- Eq. 8 / Eq. 4 / fit
def test_eq8_worked_example_golden():
    with open(os.path.join(GOLDEN, "eq8_worked_example.json")) as f:
        g = json.load(f)
    i = g["inputs"]
    v = oracle.eq8_min_replicas(i["I"], i["J"], i["K"], i["Q"], i["S"])
    assert v == pytest.approx(g["p_min"], abs=1e-12)
    assert round(v) == g["p_min_rounded"]


def test_eq4_kruskal_condition():
    rng = np.random.default_rng(14)
    A, B, C = (rng.standard_normal((6, 3)) for _ in range(3))
    assert oracle.eq4_identifiable(6, A, B, C)          # 3+3+3 >= 8
    A2 = A.copy()
    A2[:, 1] = A2[:, 0]                                  # Kruskal rank 1
    B2 = B.copy()
    B2[:, 2] = 2 * B2[:, 0]
    assert O._kruskal_rank(A2) == 1
    assert not oracle.eq4_identifiable(6, A2, B2, C)    # 1+1+3 < 8


def test_fit_bruteforce_and_limits():
    rng = np.random.default_rng(15)
    I, J, K, R = 4, 3, 5, 2
    A, B, C = (rng.standard_normal((n, R)) for n in (I, J, K))
    X = rng.standard_normal((K, I, J))
    num = den = 0.0
    for k, i, j in itertools.product(range(K), range(I), range(J)):
        xh = sum(A[i, r] * B[j, r] * C[k, r] for r in range(R))
        num += (X[k, i, j] - xh) ** 2
        den += X[k, i, j] ** 2
    assert oracle.fit(X, A, B, C) == pytest.approx(1 - np.sqrt(num / den), abs=1e-13)
    Xe = np.einsum("ir,jr,kr->kij", A, B, C)
    assert oracle.fit(Xe, A, B, C) == pytest.approx(1.0, abs=1e-13)
    assert oracle.fit(X, 0 * A, B, C) == pytest.approx(0.0, abs=1e-13)


# ---------------------------------------------------------------- whole update
def _run(I, J, R, P, Q, S, t_old, t, iters, noise, rel, seed):
    A, B, C = factors(I, J, t_old + t, R, seed)
    X = slice_batch(A, B, C, 0, t_old + t, noise, seed)
    U, V = projections(I, J, P, Q, S, seed)
    Wo = time_projection(t_old, P, Q, S, seed, -1)
    Wn = time_projection(t, P, Q, S, seed, 0)
    if rel > 0.0:
        A0, B0, C0 = init_factors(A, B, C[:t_old], rel, seed)
    else:                                    # the exact (unrounded) decomposition
        A0, B0, C0 = A, B, C[:t_old]
    o = oracle.OctenOracle(I, J, R, P, Q, S, iters)
    o.init(X[:t_old], U, V, Wo, A0, B0, C0)
    o.append(X[t_old:], Wn)
    return o, X, (A, B, C)


def test_update_exact_on_noiseless_data_with_exact_start():
    o, X, (A, B, C) = _run(12, 10, 3, 4, 6, 2, 8, 4, 40, 0.0, 0.0, 16)   # Qd = 18 >= 12
    assert rel_fro(o.A, A) < 1e-10 and rel_fro(o.B, B) < 1e-10
    assert rel_fro(o.C, C) < 1e-10
    assert oracle.fit(X, o.A, o.B, o.C) > 1 - 1e-10


def test_update_recovers_planted_factors_with_noise():
    """1 % relative noise: from the exact existing decomposition the update
    keeps fit near 1 - noise; from a 1 % perturbed one the factors still
    match the planted ones (underdetermined lift: Qd = 65 < I = 100)."""
    o, X, planted = _run(100, 100, 5, 4, 20, 5, 80, 20, 50, 0.01, 0.0, 0)
    assert oracle.fit(X, o.A, o.B, o.C) > 0.985
    assert fms((o.A, o.B, o.C), planted) > 0.999
    o, X, planted = _run(100, 100, 5, 4, 20, 5, 80, 20, 50, 0.01, 0.01, 0)
    assert oracle.fit(X, o.A, o.B, o.C) > 0.97
    assert fms((o.A, o.B, o.C), planted) > 0.99


# ---------------------------------------------------------------- planted mistakes
def test_pins_catch_planted_mistakes(monkeypatch):
    """Plausible slips planted in the oracle, on the CPU, each fail a pin."""
    real_compress = O.compress

    def transposed_U(X, U, V, W):
        return real_compress(X, V[:U.shape[0]], U[:V.shape[0]], W) if U.shape == V.shape \
            else real_compress(X, U, V, W) * 1.0001
    monkeypatch.setattr(O, "compress", transposed_U)
    monkeypatch.setattr(oracle, "compress", transposed_U)
    with pytest.raises(AssertionError):
        test_compress_exact_cp_closed_form()
    monkeypatch.undo()

    real_solve = O._normal_solve

    def wrong_gram(M, Gm):
        return real_solve(M, Gm + 0.01 * np.eye(Gm.shape[0]))
    monkeypatch.setattr(O, "_normal_solve", wrong_gram)
    with pytest.raises(AssertionError):
        test_als_every_step_is_least_squares_optimal()
    monkeypatch.undo()

    real_lift = O.lift_factor

    def no_prev(F_prev, proj, F_hat):
        return real_lift(np.zeros_like(F_prev), proj, F_hat)
    monkeypatch.setattr(O, "lift_factor", no_prev)
    monkeypatch.setattr(oracle, "lift_factor", no_prev)
    with pytest.raises(AssertionError):
        test_lift_minimum_change_when_underdetermined()
    monkeypatch.undo()

    real_align = O.align

    def no_sign(At, Bt, Ct, ra, rb, S):
        Ah, Bh, Ch, p, da, db = real_align(At, Bt, Ct, ra, rb, S)
        return Ah * np.sign(da), Bh, Ch, p, np.abs(da), db
    monkeypatch.setattr(O, "align", no_sign)
    monkeypatch.setattr(oracle, "align", no_sign)
    with pytest.raises(AssertionError):
        test_align_recovers_known_permutation_and_scales()


def test_existing_decomposition_recovers_planted_factors():
    """decompose_existing (the init without a supplied decomposition) on an exact
    rank-R tensor X_old[k][i][j] = sum_r A[i][r] B[j][r] C[k][r], from perturbed
    guesses, reproduces the tensor (fit 1) and its factors up to permutation and
    scale (FMS 1)."""
    rng = np.random.default_rng(61)
    I, J, K, R = 12, 10, 9, 3
    A, B, C = rng.standard_normal((I, R)), rng.standard_normal((J, R)), rng.standard_normal((K, R))
    X = np.stack([(A * C[k]) @ B.T for k in range(K)])   # [k][i][j]
    A0 = A + 0.05 * rng.standard_normal(A.shape)
    B0 = B + 0.05 * rng.standard_normal(B.shape)
    Ah, Bh, Ch = oracle.decompose_existing(X, A0, B0, 60)
    assert oracle.fit(X, Ah, Bh, Ch) > 1 - 1e-9
    assert fms((Ah, Bh, Ch), (A, B, C)) > 1 - 1e-9
    assert Ah.shape == (I, R) and Bh.shape == (J, R) and Ch.shape == (K, R)
