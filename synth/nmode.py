"""Planted N-mode workloads (seeded) for the higher-order extension.

Recipe, the 3-mode one mode by mode: factors A_n (I_n x R) and the time
factor C (K x R) with i.i.d. N(0, 1) entries; slice k is
sum_r C[k, r] A_1[:, r] o ... o A_{N-1}[:, r] plus Gaussian noise rescaled to
`noise` times the clean slice's Frobenius norm, drawn from a generator seeded
by (seed, k); one projection U_n,all (I_n x Qd, i.i.d. N(0, 1), rounded to
fp32) per non-temporal mode and W (t x Qd) per batch as in planted.py.  The
update runs in fp32, so every array is handed over as fp32-exact float64.
"""
from __future__ import annotations

import dataclasses

import numpy as np

from .planted import round_to


@dataclasses.dataclass(frozen=True)
class NWorkload:
    name: str
    dims: tuple
    t_old: int
    batch: int
    updates: int
    P: int
    Q: int
    S: int
    R: int
    als_iters: int
    noise: float

    @property
    def N(self) -> int:
        return len(self.dims) + 1

    @property
    def K(self) -> int:
        return self.t_old + self.batch * self.updates

    @property
    def Qd(self) -> int:
        return self.S + self.P * (self.Q - self.S)

    @property
    def slice_elems(self) -> int:
        return int(np.prod(self.dims))


NWORKLOADS = {
    # four modes, 100^3 per slice (the small dense workload with one more mode),
    # rank 5, P = 8 replicas of Q = 10 (S = 3 anchors), 10 new slices per update
    "n4_100": NWorkload("n4_100", (100, 100, 100), 20, 10, 10, 8, 10, 3, 5, 50, 0.01),
    # five modes, 30^4 per slice, rank 4, P = 8, Q = 8, S = 3
    "n5_30": NWorkload("n5_30", (30, 30, 30, 30), 20, 10, 10, 8, 8, 3, 4, 50, 0.01),
}


def nfactors(dims, K: int, R: int, seed: int):
    """Planted factors ([A_1, ..., A_{N-1}], C) as float64 arrays."""
    rng = np.random.default_rng([seed, 0xC0FFEE, len(dims)])
    As = [rng.standard_normal((int(I), R)) for I in dims]
    C = rng.standard_normal((K, R))
    return As, C


def _clean_slice(As, c_row):
    """sum_r c_row[r] A_1[:, r] o ... o A_{N-1}[:, r]: rank-one terms built
    mode by mode (rows of T index (i_1, .., i_n), columns r)."""
    R = As[0].shape[1]
    T = As[0] * np.asarray(c_row, dtype=np.float64)
    for A in As[1:]:
        T = (T[:, None, :] * A[None, :, :]).reshape(-1, R)
    return T.sum(axis=1).reshape([A.shape[0] for A in As])


def nslice_batch(As, C, k0: int, k1: int, noise: float, seed: int) -> np.ndarray:
    """Slices k0..k1-1 laid out [k][i_1]...[i_{N-1}], float64."""
    shape = [A.shape[0] for A in As]
    out = np.empty([k1 - k0] + shape)
    for n, k in enumerate(range(k0, k1)):
        clean = _clean_slice(As, C[k])
        if noise > 0.0:
            nz = np.random.default_rng([seed, 0x51CE, k, len(As)]).standard_normal(shape)
            clean = clean + (noise * np.linalg.norm(clean) / np.linalg.norm(nz)) * nz
        out[n] = clean
    return out


def nprojections(dims, P: int, Q: int, S: int, seed: int) -> list:
    """U_n,all (I_n x Qd) for every non-temporal mode, fp32-exact float64."""
    Qd = S + P * (Q - S)
    rng = np.random.default_rng([seed, 0x0AB1, len(dims)])
    return [round_to(rng.standard_normal((int(I), Qd)), "fp32") for I in dims]


def ninit_factors(As, C, rel: float, seed: int):
    """Planted factors plus a seeded relative Gaussian perturbation, rounded to
    fp32: the existing decomposition the online update starts from."""
    rng = np.random.default_rng([seed, 0x1417, len(As)])
    out = []
    for F in list(As) + [C]:
        Nz = rng.standard_normal(F.shape)
        out.append(round_to(F + rel * np.linalg.norm(F) / np.linalg.norm(Nz) * Nz, "fp32"))
    return out[:-1], out[-1]
