"""GB300 exponential-Krylov solver for multi-frequency optical response.

Python face of the C ABI in include/kx.h (Botchev, Hanse & Uppu,
arXiv:1707.00023).  The compute path is the CUDA library libkx.so built
in-tree by ``paper_1707_00023_gb300.build``; this package only marshals
arguments.
"""
from ._binding import (KX_FP32, KX_FP64, KX_PEC, KX_PERIODIC, KX_PLAIN, KX_RSTDIM, KX_SPLIT, Batch, Context,
                       KxError, EXPORTS, intensity_loss, load_library, response_multi)

__all__ = ["Batch", "Context", "KxError", "load_library", "intensity_loss", "response_multi", "EXPORTS", "KX_FP32", "KX_FP64", "KX_PEC",
           "KX_PERIODIC", "KX_PLAIN", "KX_RSTDIM", "KX_SPLIT"]
