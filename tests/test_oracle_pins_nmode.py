"""Pins of the N-mode oracle (oracle/octen_n.py, the paper's higher-order
extension) against what the mathematics fixes: with three modes every function
equals the 3-mode oracle (itself pinned in test_oracle_pins.py); for four modes,
the compression equals six nested loops on tiny inputs and the Kronecker closed
form on an exact rank-R tensor, the CP-ALS fits noiseless low-rank data
exactly, and the whole update from the exact decomposition of noiseless data
returns the planted factors; a planted mistake fails."""
import itertools

import numpy as np

import oracle
from oracle import octen_n as N
from tests._metrics import fms


def _rng(s):
    return np.random.default_rng(s)


def test_three_modes_equal_the_three_mode_oracle():
    rng = _rng(70)
    I, J, K, R, P, Q, S = 11, 9, 7, 3, 3, 5, 2
    A, B, C = rng.standard_normal((I, R)), rng.standard_normal((J, R)), rng.standard_normal((K + 4, R))
    X = np.stack([(A * C[k]) @ B.T for k in range(K + 4)]) + 0.01 * rng.standard_normal((K + 4, I, J))
    Qd = S + P * (Q - S)
    U, V = rng.standard_normal((I, Qd)), rng.standard_normal((J, Qd))
    W0, W1 = rng.standard_normal((K, Qd)), rng.standard_normal((4, Qd))
    Up, Vp, Wp = (oracle.replica_block(M, 1, Q, S) for M in (U, V, W0))
    assert np.array_equal(N.compress_n(X[:K], [Up, Vp], Wp), oracle.compress(X[:K], Up, Vp, Wp))
    Y = oracle.compress(X[:K], Up, Vp, Wp)
    F3 = [rng.standard_normal((Q, R)) for _ in range(3)]
    for mode in range(3):
        args = [F3[m] for m in range(3) if m != mode]
        fl = [F3[m] if m != mode else None for m in range(3)]
        assert np.array_equal(N.mttkrp_n(Y, fl, mode), oracle.mttkrp(Y, args, mode))
    a3 = oracle.cp_als(Y, Up.T @ A, Vp.T @ B, 6)
    an = N.cp_als_n(Y, [Up.T @ A, Vp.T @ B], 6)
    for x, y in zip(an, a3):
        assert np.array_equal(x, y)
    o3 = oracle.OctenOracle(I, J, R, P, Q, S, 6)
    on = N.OctenOracleN([I, J], R, P, Q, S, 6)
    A0, B0, C0 = A + 0.01, B - 0.01, C[:K] * 1.01
    o3.init(X[:K], U, V, W0, A0, B0, C0)
    on.init(X[:K], [U, V], W0, [A0, B0], C0)
    o3.append(X[K:], W1)
    on.append(X[K:], W1)
    assert np.array_equal(on.A[0], o3.A) and np.array_equal(on.A[1], o3.B)
    assert np.array_equal(on.C, o3.C)
    assert N.fit_n(X, on.A, on.C) == oracle.fit(X, o3.A, o3.B, o3.C)


def test_four_mode_compression_is_the_nested_sum():
    rng = _rng(71)
    K, I1, I2, I3, Q = 2, 3, 2, 3, 2
    X = rng.standard_normal((K, I1, I2, I3))
    Us = [rng.standard_normal((I, Q)) for I in (I1, I2, I3)]
    W = rng.standard_normal((K, Q))
    Z = N.compress_n(X, Us, W)
    ref = np.zeros((Q, Q, Q, Q))
    for q1, q2, q3, c in itertools.product(range(Q), repeat=4):
        s = 0.0
        for k, i1, i2, i3 in itertools.product(range(K), range(I1), range(I2), range(I3)):
            s += X[k, i1, i2, i3] * Us[0][i1, q1] * Us[1][i2, q2] * Us[2][i3, q3] * W[k, c]
        ref[q1, q2, q3, c] = s
    assert np.allclose(Z, ref, rtol=1e-12, atol=1e-12)


def _planted4(rng, dims, K, R):
    As = [rng.standard_normal((I, R)) for I in dims]
    C = rng.standard_normal((K, R))
    X = np.einsum("ar,br,cr,kr->kabc", As[0], As[1], As[2], C)
    return As, C, X


def test_four_mode_compression_of_rank_r_is_cp_of_projected_factors():
    rng = _rng(72)
    dims, K, R, Q = (6, 5, 4), 5, 2, 3
    As, C, X = _planted4(rng, dims, K, R)
    Us = [rng.standard_normal((I, Q)) for I in dims]
    W = rng.standard_normal((K, Q))
    Z = N.compress_n(X, Us, W)
    ref = np.einsum("ar,br,cr,kr->abck", *(U.T @ A for U, A in zip(Us, As)), W.T @ C)
    assert np.allclose(Z, ref, rtol=1e-12, atol=1e-10)


def test_four_mode_cp_als_fits_noiseless_low_rank():
    rng = _rng(73)
    R = 2
    Fs = [rng.standard_normal((5, R)) for _ in range(4)]
    Y = np.einsum("ar,br,cr,kr->abck", *Fs)
    out = N.cp_als_n(Y, [F + 0.05 * rng.standard_normal(F.shape) for F in Fs[:3]], 60)
    model = np.einsum("ar,br,cr,kr->abck", *out)
    assert np.linalg.norm(model - Y) / np.linalg.norm(Y) < 1e-9
    assert fms(out[:2] + [out[3]], Fs[:2] + [Fs[3]]) > 1 - 1e-9


def _exact_update(rng):
    dims, R, P, Q, S = (9, 8, 7), 2, 4, 5, 2
    K0, t = 8, 4
    As, C, X = _planted4(rng, dims, K0 + t, R)
    Qd = S + P * (Q - S)
    Us = [rng.standard_normal((I, Qd)) for I in dims]
    W0, W1 = rng.standard_normal((K0, Qd)), rng.standard_normal((t, Qd))
    o = N.OctenOracleN(list(dims), R, P, Q, S, 80)
    o.init(X[:K0], Us, W0, As, C[:K0])
    o.append(X[K0:], W1)
    return o, As, C, X


def test_four_mode_update_is_exact_on_noiseless_data():
    o, As, C, X = _exact_update(_rng(74))
    assert N.fit_n(X, o.A, o.C) > 1 - 1e-8
    assert fms(o.A[:2] + [o.C], As[:2] + [C]) > 1 - 1e-8


def test_four_mode_planted_mistake_fails(monkeypatch):
    # a Khatri-Rao product with the factors in the wrong order (a transposed
    # unfolding) breaks the MTTKRP of the 4-mode CP and the update with it
    monkeypatch.setattr(N, "khatri_rao_list",
                        lambda Fs: N.khatri_rao(Fs[-1], N.khatri_rao(Fs[1], Fs[0]))
                        if len(Fs) == 3 else N.khatri_rao(Fs[1], Fs[0]))
    o, As, C, X = _exact_update(_rng(74))
    model = np.einsum("ar,br,cr,kr->kabc", *o.A, o.C)   # the fit without the patched helper
    assert np.linalg.norm(X - model) / np.linalg.norm(X) > 1e-3


def test_four_mode_mttkrp_is_the_nested_sum():
    rng = _rng(75)
    X = rng.standard_normal((3, 2, 4, 3))
    R = 2
    Fs = [rng.standard_normal((n, R)) for n in X.shape]
    for mode in range(4):
        M = N.mttkrp_n(X, Fs, mode)
        ref = np.zeros((X.shape[mode], R))
        for idx in itertools.product(*(range(n) for n in X.shape)):
            for r in range(R):
                w = X[idx]
                for m in range(4):
                    if m != mode:
                        w *= Fs[m][idx[m], r]
                ref[idx[mode], r] += w
        assert np.allclose(M, ref, rtol=1e-12, atol=1e-12), mode


def test_four_mode_match_recovers_a_known_permutation_and_scales():
    # replica factors = the references permuted, each mode scaled per column
    # by d_n (signs included); the match must undo the permutation, divide
    # every mode by its d_n and multiply the time factor by the product
    rng = _rng(76)
    R, S, Q = 4, 5, 7
    refs = [rng.standard_normal((S, R)) for _ in range(3)]
    perm = np.array([2, 0, 3, 1])                    # reference column s sits at replica column perm[s]
    inv = np.argsort(perm)
    d = [rng.uniform(0.5, 2.0, R) * rng.choice([-1.0, 1.0], R) for _ in range(3)]
    Fs, tails = [], []
    for n in range(3):
        tail = rng.standard_normal((Q - S, R))
        full = np.vstack([refs[n], tail])            # columns in reference order
        Fs.append((full * d[n])[:, inv])             # scaled, then permuted
        tails.append(tail)
    Ctrue = rng.standard_normal((6, R))
    C = (Ctrue / (d[0] * d[1] * d[2]))[:, inv]
    Fh, Ch, got = N.align_n(Fs, C, refs, S)
    assert np.array_equal(got, perm)
    for n in range(3):
        assert np.allclose(Fh[n][:S], refs[n], rtol=1e-12, atol=1e-12)
        assert np.allclose(Fh[n][S:], tails[n], rtol=1e-12, atol=1e-12)
    assert np.allclose(Ch, Ctrue, rtol=1e-12, atol=1e-12)


def test_four_mode_fit_is_the_explicit_residual():
    rng = _rng(77)
    As = [rng.standard_normal((n, 2)) for n in (3, 2, 4)]
    C = rng.standard_normal((3, 2))
    X = rng.standard_normal((3, 3, 2, 4))
    num = den = 0.0
    for k, a, b, c in itertools.product(range(3), range(3), range(2), range(4)):
        model = sum(C[k, r] * As[0][a, r] * As[1][b, r] * As[2][c, r] for r in range(2))
        num += (X[k, a, b, c] - model) ** 2
        den += X[k, a, b, c] ** 2
    assert abs(N.fit_n(X, As, C) - (1 - np.sqrt(num) / np.sqrt(den))) < 1e-12
    exact = np.einsum("ar,br,cr,kr->kabc", *As, C)
    assert abs(N.fit_n(exact, As, C) - 1.0) < 1e-12


def test_four_mode_existing_decomposition_recovers_planted_factors():
    # noiseless planted 4-mode data: the decomposition of the existing tensor
    # from perturbed guesses reproduces it (fit 1) and its factors (FMS 1),
    # directly and through the oracle's init with the time factor omitted
    rng = _rng(78)
    dims, K, R = (7, 6, 5), 12, 2
    As, C, X = _planted4(rng, dims, K, R)
    out = N.decompose_existing_n(X, [A + 0.05 * rng.standard_normal(A.shape) for A in As], 80)
    assert N.fit_n(X, out[:-1], out[-1]) > 1 - 1e-9
    assert fms(out[:2] + [out[-1]], As[:2] + [C]) > 1 - 1e-9
    # the same through the oracle's init with C0 omitted
    P, Q, S = 3, 4, 2
    Qd = S + P * (Q - S)
    Us = [rng.standard_normal((I, Qd)) for I in dims]
    W0 = rng.standard_normal((K, Qd))
    o = N.OctenOracleN(list(dims), R, P, Q, S, 80)
    o.init(X, Us, W0, [A + 0.05 * rng.standard_normal(A.shape) for A in As], None)
    assert N.fit_n(X, o.A, o.C) > 1 - 1e-9
