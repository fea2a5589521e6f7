"""GB300-native PVFinder inference (arXiv 2602.19959): libpvf.so plus its Python binding.

    from paper_2602_19959_gb300 import build, PVFinder
    build()                                   # nvcc, sm_103a, in-tree
    pv = PVFinder(weights, precision="bf16", max_events=1000)
    z, count = pv.infer(features_cuda, offsets_cuda)

The C ABI is declared in include/pvf.h; this package only marshals arguments.
"""

from .builder import build, LIB
from .weights import pack_blob, LAYER_ORDER
from .pvf import PVFinder, PvfError, load, pool_bytes_required, EXPORTED

__all__ = ["build", "LIB", "pack_blob", "LAYER_ORDER", "PVFinder", "PvfError", "load",
           "pool_bytes_required", "EXPORTED"]
