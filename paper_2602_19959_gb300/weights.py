"""Writer of the "PVFW" v1 weight blob that pvf_create reads.

Layout (little endian):
  header (32 B)   magic "PVFW", u32 version = 1, u32 c0 (16 or 32), u32 fc_hidden = 32,
                  u32 fc_out = 100, u32 n_layers = 17, u32 reserved[2] = 0
  layer table     17 entries of 48 B, in the order LAYER_ORDER:
                  char name[8], u32 ndim, u32 shape[3], u32 n_bias, u32 pad,
                  u64 weight byte offset, u64 bias byte offset (from the blob start)
  data            float32 weights then biases of each layer, 16-byte aligned

Weight layouts are PyTorch's: FC W[out][in]; conv W[C_out][C_in][5];
ConvTranspose W[C_in][C_out][2]. The library converts them to its own layouts.
"""

from __future__ import annotations

import struct

import numpy as np

LAYER_ORDER = ("fc1", "fc2", "fc3", "fc4", "fc5", "fc6",
               "enc1", "enc2", "enc3", "enc4",
               "up3", "dec3", "up2", "dec2", "up1", "dec1", "final")


def unet_width(weights: dict) -> int:
    """UNet base width c0 of a weight set: the output channels of enc1."""
    return int(np.asarray(weights["enc1"][0]).shape[0])


def pack_blob(weights: dict) -> bytes:
    """weights: {name: (W, b)} with float32-convertible arrays, all 17 layers."""
    header = struct.pack("<4s7I", b"PVFW", 1, unet_width(weights), 32, 100, len(LAYER_ORDER), 0, 0)
    table_size = 48 * len(LAYER_ORDER)
    data = bytearray()
    entries = []
    base = len(header) + table_size

    def put(arr):
        nonlocal data
        pad = (-(base + len(data))) % 16
        data += b"\0" * pad
        off = base + len(data)
        data += np.ascontiguousarray(arr, dtype="<f4").tobytes()
        return off

    for name in LAYER_ORDER:
        W, b = weights[name]
        W = np.asarray(W, dtype=np.float32)
        b = np.asarray(b, dtype=np.float32).reshape(-1)
        shape = list(W.shape) + [0] * (3 - W.ndim)
        wo = put(W)
        bo = put(b)
        entries.append(struct.pack("<8s6IQQ", name.encode(), W.ndim, *shape, b.size, 0, wo, bo))
    blob = header + b"".join(entries) + bytes(data)
    assert len(header) == 32 and all(len(e) == 48 for e in entries)
    return blob
