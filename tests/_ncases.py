"""Seeded N-mode update cases shared by the GPU parity tests of the
higher-order extension: the same inputs go to the FP64 N-mode oracle and,
through the C ABI, to the CUDA library."""
from __future__ import annotations

import dataclasses

import numpy as np

from oracle import octen_n
from synth import ninit_factors, nfactors, nprojections, nslice_batch, round_to, time_projection


@dataclasses.dataclass
class NCase:
    dims: tuple
    R: int
    P: int
    Q: int
    S: int
    t_old: int
    batches: tuple
    iters: int
    noise: float = 0.01
    rel: float = 0.01
    seed: int = 0

    @property
    def N(self) -> int:
        return len(self.dims) + 1

    def make(self):
        K = self.t_old + sum(self.batches)
        As, C = nfactors(self.dims, K, self.R, self.seed)
        X = round_to(nslice_batch(As, C, 0, K, self.noise, self.seed), "fp32")
        Us = nprojections(self.dims, self.P, self.Q, self.S, self.seed)
        W = [time_projection(self.t_old, self.P, self.Q, self.S, self.seed, -1)]
        for b, t in enumerate(self.batches):
            W.append(time_projection(t, self.P, self.Q, self.S, self.seed, b))
        A0s, C0 = ninit_factors(As, C[:self.t_old], self.rel, self.seed)
        return dict(X=X, U=Us, W=W, A0=A0s, C0=C0, planted=(As, C))

    def oracle_run(self, d, upto=None):
        o = octen_n.OctenOracleN(list(self.dims), self.R, self.P, self.Q, self.S, self.iters)
        o.init(d["X"][:self.t_old], d["U"], d["W"][0], d["A0"], d["C0"])
        k = self.t_old
        states = []
        for b, t in enumerate(self.batches[:upto]):
            o.append(d["X"][k:k + t], d["W"][b + 1])
            k += t
            states.append(dict(Y=[y.copy() for y in o.Y], A=[a.copy() for a in o.A],
                               C=o.C.copy(), raw=o.last["raw"], hat=o.last["hat"]))
        return o, states
