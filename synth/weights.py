"""He-initialised float32 master weights for the hybrid network.

The paper gives the structure (§2: six FC layers on nine track features feeding a
UNet-style 1D CNN) but no trained checkpoint is available, so weights are random:
W ~ N(0, 2 / fan_in) with fan_in = in_features for FC layers, C_in * 5 for the
kernel-5 convolutions and C_in * 2 for the stride-2 transposed convolutions.
Biases are zero unless ``bias_std`` > 0 (tests use non-zero biases to exercise
every bias path). All weights are drawn first, in LAYER_ORDER, then the biases,
so the weights do not depend on ``bias_std``.

Weight layouts (PyTorch conventions):
  FC         W[out][in]
  conv k5    W[C_out][C_in][5]
  ConvT k2s2 W[C_in][C_out][2]
"""

from __future__ import annotations

import numpy as np

LAYER_ORDER = ("fc1", "fc2", "fc3", "fc4", "fc5", "fc6",
               "enc1", "enc2", "enc3", "enc4",
               "up3", "dec3", "up2", "dec2", "up1", "dec1", "final")

N_FEATURES = 9


def layer_shapes(c0: int = 16, fc_hidden: int = 32, fc_out: int = 100) -> dict:
    """name -> (weight shape, bias length, fan_in) for a UNet of base width c0."""
    h, c1, c2, c3, c4 = fc_hidden, c0, 2 * c0, 4 * c0, 8 * c0
    shapes = {
        "fc1": ((h, N_FEATURES), h, N_FEATURES),
        "fc2": ((h, h), h, h), "fc3": ((h, h), h, h),
        "fc4": ((h, h), h, h), "fc5": ((h, h), h, h),
        "fc6": ((fc_out, h), fc_out, h),
        "enc1": ((c1, 1, 5), c1, 1 * 5),
        "enc2": ((c2, c1, 5), c2, c1 * 5),
        "enc3": ((c3, c2, 5), c3, c2 * 5),
        "enc4": ((c4, c3, 5), c4, c3 * 5),
        "up3": ((c4, c3, 2), c3, c4 * 2),
        "dec3": ((c3, 2 * c3, 5), c3, 2 * c3 * 5),
        "up2": ((c3, c2, 2), c2, c3 * 2),
        "dec2": ((c2, 2 * c2, 5), c2, 2 * c2 * 5),
        "up1": ((c2, c1, 2), c1, c2 * 2),
        "dec1": ((c1, 2 * c1, 5), c1, 2 * c1 * 5),
        "final": ((1, c1, 5), 1, c1 * 5),
    }
    return shapes


def he_weights(seed: int = 0, bias_std: float = 0.0, c0: int = 16,
               fc_hidden: int = 32, fc_out: int = 100) -> dict:
    """Returns {name: (W float32, b float32)} in LAYER_ORDER."""
    rng = np.random.default_rng(seed)
    shapes = layer_shapes(c0, fc_hidden, fc_out)
    out = {}
    for name in LAYER_ORDER:
        wshape, _, fan_in = shapes[name]
        out[name] = [rng.normal(0.0, np.sqrt(2.0 / fan_in), wshape).astype(np.float32), None]
    for name in LAYER_ORDER:
        nb = shapes[name][1]
        if bias_std > 0.0:
            out[name][1] = rng.normal(0.0, bias_std, nb).astype(np.float32)
        else:
            out[name][1] = np.zeros(nb, dtype=np.float32)
    return {k: (np.ascontiguousarray(v[0]), v[1]) for k, v in out.items()}
