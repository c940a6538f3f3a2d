"""EFE real-time TDDFT hot path for one GB300 (sm_103a).

The numerical work lives in libefe (CUDA, C ABI in include/efe.h); this
package holds its sources (csrc/), the in-tree build (build.py) and a thin
ctypes binding (_binding.py).  Importing the package does not load the
library; `Context` and `lib()` do, and raise if it has not been built.
"""
from ._binding import (EFE_FP64, EFE_MIXED, EXPORTED, Context, EfeError, fields_array, lib)  # noqa: F401

__all__ = ["Context", "EfeError", "EFE_FP64", "EFE_MIXED", "EXPORTED", "lib", "fields_array"]
