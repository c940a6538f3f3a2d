"""EFE real-time TDDFT hot path for one GB300 (sm_103a).

The numerical work lives in libefe (CUDA, C ABI in include/efe.h); this
package holds its sources (csrc/), the in-tree build (build.py) and a thin
ctypes binding (_binding.py).  Importing the package does not load the
library; `Context` and `lib()` do, and raise if it has not been built.
"""
from ._binding import (EFE_FP64, EFE_HARTREE_FDM, EFE_HARTREE_PCG, EFE_MIXED, EFE_PAIR, EFE_TC, EFE_STEP_EXTRAPOLATED,  # noqa: F401
                       EFE_STEP_PC, EFE_XC_PW92, EFE_XC_PZ81, EXPORTED, Context, EfeError, Octree,
                       absorption_spectrum, adaptive_cell_boxes, atom_hartree_table, fields_array, lib,
                       lda_points, octree_constraints, pipe_peaks, power_spectrum, checkpoint_inspect,
                       checkpoint_write_host)

__all__ = ["Context", "Octree", "EfeError", "EFE_FP64", "EFE_MIXED", "EFE_PAIR", "EFE_TC", "EFE_XC_PW92", "EFE_XC_PZ81", "EFE_STEP_PC", "EFE_STEP_EXTRAPOLATED", "EFE_HARTREE_FDM", "EFE_HARTREE_PCG", "EXPORTED", "lib",
           "fields_array", "absorption_spectrum", "power_spectrum", "octree_constraints",
           "atom_hartree_table", "adaptive_cell_boxes", "lda_points", "pipe_peaks", "checkpoint_inspect", "checkpoint_write_host"]
