"""Planted-CP workloads and random projections (seeded, shape-faithful).

Recipe (the paper's synthetic tensors, Sec. "Experimental Setup" / Table 2,
are dense I x J x K tensors built from known random factors plus Gaussian
noise; the shapes below follow the five workload descriptions this library
is measured on):

* factors A (I x R), B (J x R), C (K x R) with i.i.d. N(0, 1) entries; for the
  conditioned workload each factor is Q_F diag(logspace(0, -log10(cond), R)) H
  scaled by sqrt(rows), with Q_F from the QR of a Gaussian and H a random
  orthogonal R x R matrix; for the "large slices" workload a seeded 20 % subset
  of time indices k has C[k, :] multiplied by 10;
* slice k is X_k = A diag(C[k, :]) B^T + N_k with N_k Gaussian, rescaled so that
  ||N_k||_F = noise * ||A diag(C[k, :]) B^T||_F (relative, per slice), and
  drawn from a generator seeded by (seed, k) so any slice can be regenerated
  alone;
* projection matrices U_all (I x Qd), V_all (J x Qd) and, per batch, W_all
  (t x Qd) with Qd = S + P (Q - S): columns [0, S) are the anchors shared by
  every replica (Eq. 1), replica p owns columns [S + p (Q - S), S + (p+1) (Q - S)).
  Entries are i.i.d. N(0, 1) (the paper draws uniform entries; any absolutely
  continuous law serves the identifiability argument of Sec. "Factor match").

Rounding to a compute format (bf16, e4m3) is done once, here, with torch's
round-to-nearest-even conversions; the rounded values *are* the matrices.
"""
from __future__ import annotations

import dataclasses

import numpy as np


@dataclasses.dataclass(frozen=True)
class Workload:
    name: str
    I: int
    J: int
    t_old: int
    batch: int
    updates: int
    P: int
    Q: int
    S: int
    R: int
    als_iters: int
    prec: str          # "fp32", "bf16" or "fp8"
    noise: float
    cond: float | None = None
    big_frac: float = 0.0
    big_mult: float = 10.0

    @property
    def K(self) -> int:
        return self.t_old + self.batch * self.updates

    @property
    def Qd(self) -> int:
        return self.S + self.P * (self.Q - self.S)

    def input_dtype(self) -> str:
        """Element type of the slice batch handed to the update."""
        return "fp32" if self.prec == "fp32" else "bf16"


WORKLOADS = {
    # dense 100^3, rank 5, 80 old slices + one batch of 20, P=4, Q=20, S=5
    "c1": Workload("c1_fp32_100x100x100_P4_Q20_R5", 100, 100, 80, 20, 1,
                   4, 20, 5, 5, 50, "fp32", 0.01),
    # dense 1000 x 1000 x 1000, rank 10, 900 old + 10 batches of 10, P=8, Q=100
    "c2": Workload("c2_fp32_1000x1000x1000_P8_Q100_R10", 1000, 1000, 900, 10, 10,
                   8, 100, 10, 10, 30, "fp32", 0.01),
    # 2000 x 2000 slices in bf16, rank 20, cond 10, 0.5 % noise, 20 x 50 slices
    "c3": Workload("c3_bf16_2000x2000_P16_Q200_R20", 2000, 2000, 100, 50, 20,
                   16, 200, 20, 20, 30, "bf16", 0.005, cond=10.0),
    # 4000 x 4000 slices, rank 32, 20 % of slices 10x larger, 32 x 16 slices
    "c4": Workload("c4_fp8_4000x4000_P16_Q256_R32", 4000, 4000, 64, 16, 32,
                   16, 256, 32, 32, 30, "fp8", 0.01, big_frac=0.2),
    # scalability replay (Sec. "[Q3] Scalability Evaluation"): small slices,
    # a long time mode, 10 % of it as the existing tensor, batches of 10.  The
    # paper does not give P, Q, S, R for these runs; the 100 x 100 one takes the
    # small dense workload's, the smaller ones scale them down.  `updates` is
    # the default replay length (a stream of 10^4 slices); bench.py --replay
    # extends it up to 10^6.
    "q3_20": Workload("q3_fp32_20x20_P4_Q8_R3", 20, 20, 1000, 10, 900,
                      4, 8, 3, 3, 50, "fp32", 0.01),
    "q3_50": Workload("q3_fp32_50x50_P4_Q12_R4", 50, 50, 1000, 10, 900,
                      4, 12, 4, 4, 50, "fp32", 0.01),
    "q3_100": Workload("q3_fp32_100x100_P4_Q20_R5", 100, 100, 1000, 10, 900,
                       4, 20, 5, 5, 50, "fp32", 0.01),
}


def uneven_streams(n: int = 64, seed: int = 0) -> list:
    """The batched uneven-streams workload: n independent planted-CP streams with
    I, J uniform in [200, 3000] (rounded up to a multiple of 8, the 16-byte row
    pitch the TMA loads of bf16 slices need), rank R uniform in [5, 32], batch
    size t uniform in [5, 50], compressed size Q uniform in [20, 150], P = 8,
    S = min(R, Q // 2), 30 sweeps, bf16 slices with 1 % noise; 5 t existing
    slices per stream.  Each entry is a Workload plus its own seed."""
    rng = np.random.default_rng(np.random.SeedSequence([seed, 5]))
    out = []
    for s in range(n):
        I = int(-(-int(rng.integers(200, 3001)) // 8) * 8)
        J = int(-(-int(rng.integers(200, 3001)) // 8) * 8)
        R = int(rng.integers(5, 33))
        t = int(rng.integers(5, 51))
        Q = int(rng.integers(20, 151))
        S = min(R, Q // 2)
        wl = Workload(f"c5_stream{s}_{I}x{J}_P8_Q{Q}_R{R}_t{t}", I, J, 5 * t, t, 1,
                      8, Q, S, R, 30, "bf16", 0.01)
        out.append((wl, seed * 1000 + s))
    return out


def _conditioned(rows: int, R: int, cond: float, rng: np.random.Generator) -> np.ndarray:
    q, _ = np.linalg.qr(rng.standard_normal((rows, R)))
    h, _ = np.linalg.qr(rng.standard_normal((R, R)))
    s = np.logspace(0.0, -np.log10(cond), R)
    return np.sqrt(rows) * (q * s) @ h


def factors(I: int, J: int, K: int, R: int, seed: int, cond: float | None = None,
            big_frac: float = 0.0, big_mult: float = 10.0):
    """Planted factors (A, B, C) as float64 arrays."""
    rng = np.random.default_rng([seed, 0xC0FFEE])
    if cond is None:
        A = rng.standard_normal((I, R))
        B = rng.standard_normal((J, R))
        C = rng.standard_normal((K, R))
    else:
        A = _conditioned(I, R, cond, rng)
        B = _conditioned(J, R, cond, rng)
        C = _conditioned(K, R, cond, rng)
    if big_frac > 0.0:
        nbig = int(round(big_frac * K))
        idx = rng.choice(K, size=nbig, replace=False)
        C[idx] *= big_mult
    return A, B, C


def _slice_noise(seed: int, k: int, I: int, J: int) -> np.ndarray:
    return np.random.default_rng([seed, 0x51CE, k]).standard_normal((I, J))


def slice_batch(A: np.ndarray, B: np.ndarray, C: np.ndarray, k0: int, k1: int,
                noise: float, seed: int) -> np.ndarray:
    """Slices k0..k1-1 as a float64 array laid out [k][i][j]."""
    I, J = A.shape[0], B.shape[0]
    out = np.empty((k1 - k0, I, J))
    for n, k in enumerate(range(k0, k1)):
        clean = (A * C[k]) @ B.T
        if noise > 0.0:
            nz = _slice_noise(seed, k, I, J)
            clean = clean + (noise * np.linalg.norm(clean) / np.linalg.norm(nz)) * nz
        out[n] = clean
    return out


def slice_batch_torch(A, B, C, k0: int, k1: int, noise: float, seed: int, device,
                      dtype):
    """Same recipe as `slice_batch`, drawn with torch on `device` (for large
    benchmark batches; the noise stream differs from numpy's, the law does not)."""
    import torch

    A = torch.as_tensor(A, dtype=torch.float32, device=device)
    B = torch.as_tensor(B, dtype=torch.float32, device=device)
    C = torch.as_tensor(C, dtype=torch.float32, device=device)
    I, J = A.shape[0], B.shape[0]
    out = torch.empty((k1 - k0, I, J), dtype=dtype, device=device)
    g = torch.Generator(device=device)
    for n, k in enumerate(range(k0, k1)):
        clean = (A * C[k]) @ B.T
        if noise > 0.0:
            g.manual_seed(int(seed) * 1_000_003 + int(k))
            nz = torch.randn((I, J), generator=g, device=device, dtype=torch.float32)
            clean = clean + (noise * torch.linalg.norm(clean) / torch.linalg.norm(nz)) * nz
        out[n] = clean.to(dtype)
    return out


def round_to(x: np.ndarray, fmt: str) -> np.ndarray:
    """Round to a storage format with round-to-nearest-even and return the
    rounded values as float64 (fp8 saturates to the finite e4m3 range)."""
    import torch

    t = torch.from_numpy(np.ascontiguousarray(x, dtype=np.float64))
    if fmt == "fp64":
        return t.numpy().copy()
    if fmt == "fp32":
        return t.to(torch.float32).to(torch.float64).numpy()
    if fmt == "bf16":
        return t.to(torch.float32).to(torch.bfloat16).to(torch.float64).numpy()
    if fmt == "e4m3":
        t32 = t.to(torch.float32).clamp(-448.0, 448.0)
        return t32.to(torch.float8_e4m3fn).to(torch.float64).numpy()
    raise ValueError(fmt)


def _prec_formats(prec: str):
    """(U format, V format) for each compute precision: the mode-2 operand V is
    stored in the contraction's input type, U in bf16 for both reduced paths."""
    return {"fp32": ("fp32", "fp32"), "bf16": ("bf16", "bf16"),
            "fp8": ("bf16", "e4m3")}[prec]


def projections(I: int, J: int, P: int, Q: int, S: int, seed: int, prec: str = "fp32"):
    """U_all (I x Qd) and V_all (J x Qd), float64, already rounded for `prec`."""
    Qd = S + P * (Q - S)
    rng = np.random.default_rng([seed, 0x0AB1])
    U = rng.standard_normal((I, Qd))
    V = rng.standard_normal((J, Qd))
    fu, fv = _prec_formats(prec)
    return round_to(U, fu), round_to(V, fv)


def time_projection(t: int, P: int, Q: int, S: int, seed: int, batch: int):
    """W_all (t x Qd) for batch number `batch` (batch -1 is the existing
    tensor), float64 values exactly representable in fp32."""
    Qd = S + P * (Q - S)
    rng = np.random.default_rng([seed, 0x7133, batch + 1])
    return round_to(rng.standard_normal((t, Qd)), "fp32")


def init_factors(A: np.ndarray, B: np.ndarray, C: np.ndarray, rel: float, seed: int):
    """Planted factors plus a seeded relative Gaussian perturbation, rounded to
    fp32: the 'existing decomposition' the online update starts from."""
    rng = np.random.default_rng([seed, 0x1417])
    out = []
    for F in (A, B, C):
        N = rng.standard_normal(F.shape)
        out.append(round_to(F + rel * np.linalg.norm(F) / np.linalg.norm(N) * N, "fp32"))
    return tuple(out)
