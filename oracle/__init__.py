"""FP64 CPU oracle of the quasi-static slice advance (test infrastructure).

Only tests/, the smoke check and the benchmark's CPU-baseline leg use this
package.  It shares no code with the CUDA library.
"""
from .qs_oracle import *  # noqa: F401,F403
from .qs_oracle import (Config, gamma_qs, Grid, Plasma, SliceFields, StepResult, cell_index,
                        cell_sort, config_from_workload, deposit, deposit_beam, gather,
                        init_plasma, laplacian, plasma_from_workload, push_beam,
                        push_plasma, refine_m, slice_fields, solve_poisson,
                        solve_screened, step3d, wake_at)
