"""Shared test utilities: GPU inputs, and the plain two-pointer PV matching that the
package's vectorised agreement (paper_2602_19959_gb300.agreement) is checked against."""

from __future__ import annotations

import numpy as np

from paper_2602_19959_gb300.agreement import pv_agreement  # noqa: F401  (re-exported)

N_BINS = 4000


def to_cuda(batch):
    import torch
    feats = torch.from_numpy(np.ascontiguousarray(batch.features)).cuda()
    offs = torch.from_numpy(np.ascontiguousarray(batch.offsets)).cuda()
    return feats, offs


def match_pvs(z_a, z_b, tol=0.1):
    """One-to-one two-pointer matching of two ascending z lists within tol (mm).
    Returns (matched pairs, unmatched indices of a, unmatched indices of b)."""
    i = j = 0
    pairs, ua, ub = [], [], []
    while i < len(z_a) and j < len(z_b):
        d = z_a[i] - z_b[j]
        if abs(d) <= tol:
            pairs.append((i, j))
            i += 1
            j += 1
        elif d < 0:
            ua.append(i)
            i += 1
        else:
            ub.append(j)
            j += 1
    ua.extend(range(i, len(z_a)))
    ub.extend(range(j, len(z_b)))
    return pairs, ua, ub


def logit_errors(ref_logit, got_logit):
    """Per-event max |d logit| / max |logit| (the per-bin error relative to the event's
    largest logit), as an array over events."""
    ref = np.asarray(ref_logit, np.float64)
    d = np.abs(np.asarray(got_logit, np.float64) - ref)
    return d.max(axis=1) / np.maximum(np.abs(ref).max(axis=1), 1e-30)
