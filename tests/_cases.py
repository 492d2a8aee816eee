"""Seeded update cases shared by the GPU parity tests: the same inputs go to the
FP64 oracle and, through the C ABI, to the CUDA library."""
from __future__ import annotations

import dataclasses

import numpy as np

import oracle
from synth import factors, init_factors, projections, round_to, slice_batch, time_projection


@dataclasses.dataclass
class Case:
    I: int
    J: int
    R: int
    P: int
    Q: int
    S: int
    t_old: int
    batches: tuple
    iters: int
    prec: str = "fp32"
    noise: float = 0.01
    rel: float = 0.01
    seed: int = 0
    big_frac: float = 0.0
    cond: float | None = None

    def make(self):
        K = self.t_old + sum(self.batches)
        A, B, C = factors(self.I, self.J, K, self.R, self.seed, cond=self.cond,
                          big_frac=self.big_frac)
        X = slice_batch(A, B, C, 0, K, self.noise, self.seed)
        if self.prec != "fp32":
            X = round_to(X, "bf16")       # the slices the update receives are bf16
        else:
            X = round_to(X, "fp32")
        U, V = projections(self.I, self.J, self.P, self.Q, self.S, self.seed, self.prec)
        W = [time_projection(self.t_old, self.P, self.Q, self.S, self.seed, -1)]
        for b, t in enumerate(self.batches):
            W.append(time_projection(t, self.P, self.Q, self.S, self.seed, b))
        A0, B0, C0 = init_factors(A, B, C[:self.t_old], self.rel, self.seed)
        return dict(X=X, U=U, V=V, W=W, A0=A0, B0=B0, C0=C0, planted=(A, B, C))

    def oracle_run(self, d, upto=None):
        o = oracle.OctenOracle(self.I, self.J, self.R, self.P, self.Q, self.S, self.iters)
        o.init(d["X"][:self.t_old], d["U"], d["V"], d["W"][0], d["A0"], d["B0"], d["C0"])
        k = self.t_old
        states = []
        for b, t in enumerate(self.batches[:upto]):
            o.append(d["X"][k:k + t], d["W"][b + 1])
            k += t
            states.append(dict(Y=[y.copy() for y in o.Y], A=o.A.copy(), B=o.B.copy(),
                               C=o.C.copy(), raw=o.last["raw"], hat=o.last["hat"]))
        return o, states


def rel(x, ref) -> float:
    x = np.asarray(x, np.float64)
    ref = np.asarray(ref, np.float64)
    return float(np.linalg.norm(x - ref) / max(np.linalg.norm(ref), 1e-300))
