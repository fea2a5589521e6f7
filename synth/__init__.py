"""Seeded synthetic inputs shared by the CUDA path, the oracle, the tests and the bench.

This package draws random numbers and nothing else: it holds none of the method's
arithmetic (no slicing, no network, no histogram, no peak finding). Both sides of
every parity check receive the same arrays from here.

* :mod:`synth.events` -- collision events shaped like the paper's workload (§1: an
  average of 5.6 primary vertices per event; §2: nine features per track), stored as
  Structure-of-Arrays float32 features plus int32 per-event offsets.
* :mod:`synth.weights` -- He-initialised float32 master weights of the hybrid network
  (per-track FC net and 1D UNet of §2) in a fixed layer order.
"""

from .events import (EventBatch, FEATURE_NAMES, generate_standard, generate_uneven,
                     generate, concat_batches)
from .weights import LAYER_ORDER, layer_shapes, he_weights

__all__ = ["EventBatch", "FEATURE_NAMES", "generate_standard", "generate_uneven",
           "generate", "concat_batches", "LAYER_ORDER", "layer_shapes", "he_weights"]
