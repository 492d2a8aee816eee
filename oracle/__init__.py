"""FP64 CPU oracle of the OCTen online CP update.

TEST INFRASTRUCTURE ONLY.  Only `tests/`, `__graft_entry__.smoke()` and the
CPU-baseline leg of `bench.py` may import it.  It shares no code with the CUDA
library and never calls it.
"""
from .octen import (  # noqa: F401
    OctenOracle,
    align,
    compress,
    cp_als,
    decompose_existing,
    eq4_identifiable,
    eq8_min_replicas,
    fit,
    khatri_rao,
    lift_C,
    lift_factor,
    mttkrp,
    replica_block,
)
from .octen_n import (  # noqa: F401
    OctenOracleN,
    align_n,
    compress_n,
    cp_als_n,
    decompose_existing_n,
    fit_n,
    khatri_rao_list,
    mttkrp_n,
)
