"""GB300-native quasi-static xi-slice advance (WAND-PIC method, arXiv 2012.00881).

The computation lives in libqs.so (hand-written sm_103a CUDA behind the C ABI
of include/qs.h); this package is the thin Python binding.  Build the
library with ``paper_2012_00881_gb300.build.build()``.
"""
from ._binding import (FIELD_ALL, FIELD_BX, FIELD_BY, FIELD_BZ, FIELD_EZ, FIELD_JZB,
                       FIELD_NAMES, FIELD_PSI, PROTOTYPES, QS_ERR_ARG, QS_ERR_CUDA,
                       QS_ERR_NOT_CONVERGED, QS_ERR_OOM, QS_ERR_PSI_FLOOR, QS_ERR_STATE,
                       QS_ERR_TIMEOUT, QS_FP32_REFINED, QS_FP64, QS_OK, Beam, Context, QsConfig,
                       QsError, config_from_workload, default_config, load_library,
                       step3d_batched, cell_sort_noalloc, bigaussian_beam,
                       bigaussian_adjoint, NonuniformSolver, NonuniformPIC,
                       LaserEnvelope)
from .grad import WitnessGain, witness_gain

__all__ = [
    "Beam", "Context", "QsConfig", "QsError", "config_from_workload", "default_config",
    "step3d_batched", "cell_sort_noalloc", "bigaussian_beam", "bigaussian_adjoint",
    "WitnessGain", "witness_gain", "NonuniformSolver", "NonuniformPIC", "LaserEnvelope",
    "load_library", "PROTOTYPES", "FIELD_ALL", "FIELD_PSI", "FIELD_EZ", "FIELD_BZ", "FIELD_BX",
    "FIELD_BY", "FIELD_JZB", "FIELD_NAMES", "QS_FP64", "QS_FP32_REFINED",
]
