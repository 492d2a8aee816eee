"""Seeded synthetic inputs for the OCTen online CP update.

This package only draws random numbers and shapes them into the inputs that
both the CUDA path and the CPU oracle consume: planted low-rank CP slices with
relative Gaussian noise, the random projection matrices with their shared
anchor columns, and the perturbed initial factors.  It holds none of the
update's arithmetic (no compression, no ALS, no alignment, no lifting).
"""
from .planted import (  # noqa: F401
    WORKLOADS,
    Workload,
    factors,
    init_factors,
    projections,
    round_to,
    slice_batch,
    slice_batch_torch,
    time_projection,
    uneven_streams,
)
from .nmode import NWORKLOADS, NWorkload, nfactors, ninit_factors, nprojections, nslice_batch  # noqa: F401
