"""The seeded input generators (no method arithmetic): their recipes hold as
stated — noiseless slices are the planted CP model, the noise has the stated
relative size, every slice can be regenerated alone, projections carry the
anchor-column layout and are exactly representable in their formats."""
import numpy as np

from synth import (factors, nfactors, nprojections, nslice_batch, projections, round_to,
                   slice_batch, time_projection)


def test_three_mode_slices_are_the_planted_model_plus_relative_noise():
    A, B, C = factors(9, 7, 6, 3, seed=1)
    X0 = slice_batch(A, B, C, 0, 6, 0.0, seed=1)
    assert np.allclose(X0, np.einsum("ir,jr,kr->kij", A, B, C), atol=1e-12)
    X = slice_batch(A, B, C, 0, 6, 0.05, seed=1)
    for k in range(6):
        rel = np.linalg.norm(X[k] - X0[k]) / np.linalg.norm(X0[k])
        assert abs(rel - 0.05) < 1e-12
    # any slice regenerates alone, with the same noise
    assert np.array_equal(slice_batch(A, B, C, 4, 5, 0.05, seed=1)[0], X[4])


def test_n_mode_slices_are_the_planted_model_plus_relative_noise():
    As, C = nfactors((4, 3, 5, 2), 5, 2, seed=2)
    X0 = nslice_batch(As, C, 0, 5, 0.0, seed=2)
    ref = np.einsum("ar,br,cr,dr,kr->kabcd", *As, C)
    assert np.allclose(X0, ref, atol=1e-12)
    X = nslice_batch(As, C, 0, 5, 0.02, seed=2)
    for k in range(5):
        rel = np.linalg.norm(X[k] - X0[k]) / np.linalg.norm(X0[k])
        assert abs(rel - 0.02) < 1e-12
    assert np.array_equal(nslice_batch(As, C, 3, 4, 0.02, seed=2)[0], X[3])


def test_projections_are_exact_in_their_formats_and_sized_by_the_anchor_layout():
    P, Q, S = 3, 6, 2
    Qd = S + P * (Q - S)
    U, V = projections(11, 13, P, Q, S, seed=3, prec="fp8")
    assert U.shape == (11, Qd) and V.shape == (13, Qd)
    assert np.array_equal(U, round_to(U, "bf16")) and np.array_equal(V, round_to(V, "e4m3"))
    W = time_projection(4, P, Q, S, seed=3, batch=0)
    assert W.shape == (4, Qd) and np.array_equal(W, round_to(W, "fp32"))
    assert not np.array_equal(W, time_projection(4, P, Q, S, seed=3, batch=1))
    Us = nprojections((5, 6, 7), P, Q, S, seed=3)
    assert [u.shape for u in Us] == [(5, Qd), (6, Qd), (7, Qd)]
    assert all(np.array_equal(u, round_to(u, "fp32")) for u in Us)
