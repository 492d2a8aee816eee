"""Comparison measures used by the tests (not part of the method).

* rel_fro: relative Frobenius error ||x - ref|| / ||ref||.
* fms: factor-match score between two CP models, (1/R) sum_r of the product
  over modes of |cos| between matched columns, matched by the permutation
  that maximises the sum (brute force for R <= 8, Hungarian otherwise), with
  no penalty on the scales.
"""
from __future__ import annotations

import itertools

import numpy as np


def rel_fro(x, ref) -> float:
    x = np.asarray(x, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    den = np.linalg.norm(ref)
    return float(np.linalg.norm(x - ref) / (den if den > 0 else 1.0))


def _abs_cos(F, G):
    nf = np.linalg.norm(F, axis=0)
    ng = np.linalg.norm(G, axis=0)
    return np.abs(F.T @ G) / np.outer(np.where(nf > 0, nf, 1), np.where(ng > 0, ng, 1))


def fms(model, ref) -> float:
    """Factor-match score of `model` = (A, B, C) against `ref` = (A, B, C)."""
    R = ref[0].shape[1]
    sim = np.ones((R, R))
    for F, G in zip(model, ref):
        sim = sim * _abs_cos(np.asarray(F, np.float64), np.asarray(G, np.float64))
    if R <= 8:
        best = 0.0
        for perm in itertools.permutations(range(R)):
            best = max(best, sum(sim[perm[s], s] for s in range(R)))
        return best / R
    from scipy.optimize import linear_sum_assignment

    rows, cols = linear_sum_assignment(-sim)
    return float(sim[rows, cols].sum() / R)
