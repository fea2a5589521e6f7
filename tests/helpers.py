"""Shared test utilities: GPU inputs, PV-list matching with the near-tie exemption."""

from __future__ import annotations

import numpy as np

N_BINS = 4000
THR_LOGIT = float(np.log(0.01 / 0.99))


def to_cuda(batch):
    import torch
    feats = torch.from_numpy(np.ascontiguousarray(batch.features)).cuda()
    offs = torch.from_numpy(np.ascontiguousarray(batch.offsets)).cuda()
    return feats, offs


def decision_margin(logit: np.ndarray, i: int) -> float:
    """Smallest distance of bin i's peak decision from flipping: to the threshold and
    to every neighbour inside the +-5 window (decisions are taken on the logits)."""
    lo, hi = max(0, i - 5), min(len(logit) - 1, i + 5)
    m = abs(logit[i] - THR_LOGIT)
    for j in range(lo, hi + 1):
        if j != i:
            m = min(m, abs(logit[i] - logit[j]))
    return m


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


def z_to_bin(z: float) -> int:
    return int(np.clip(np.floor((z + 100.0) / 0.1), 0, N_BINS - 1))


def pv_agreement(oracle_z, oracle_n, gpu_z, gpu_n, oracle_logit, eps: float, tol=0.1):
    """Agreement of PV lists, strict and with the near-tie exemption.

    PVs are matched one-to-one in z order within tol. A PV present on one side only is
    exempt when the oracle's decision at some bin within +-4 bins of it is within eps of
    flipping (a threshold crossing or a tie with a neighbour in the +-5 window): then both
    lists are correct results of the same rule under rounding of size eps.
      strict = matched / total,  exempt = 1 - (non-exempt unmatched) / total,
    with total = sum over events of max(n_oracle, n_gpu).
    Returns dict(strict, exempt, matched, total, unmatched, exempted, max_dz)."""
    matched = total = unmatched = exempted = 0
    max_dz = 0.0
    for e in range(len(oracle_n)):
        na, nb = int(oracle_n[e]), int(gpu_n[e])
        if na < 0 or nb < 0:
            assert na == nb, (e, na, nb)
            continue
        # compare the stored (possibly truncated) lists; counts are compared by the caller
        na, nb = min(na, len(oracle_z[e])), min(nb, len(gpu_z[e]))
        za, zb = oracle_z[e][:na], gpu_z[e][:nb]
        pairs, ua, ub = match_pvs(za, zb, tol)
        matched += len(pairs)
        total += max(na, nb)
        for (i, j) in pairs:
            max_dz = max(max_dz, abs(za[i] - zb[j]))
        for z in [za[i] for i in ua] + [zb[j] for j in ub]:
            unmatched += 1
            c = z_to_bin(z)
            f = oracle_logit[e]
            m = min(decision_margin(f, k) for k in range(max(0, c - 4), min(N_BINS, c + 5)))
            if m < eps:
                exempted += 1
    strict = matched / total if total else 1.0
    exempt = max(0.0, 1.0 - (unmatched - exempted) / total) if total else 1.0
    return dict(strict=strict, exempt=exempt, matched=matched, total=total,
                unmatched=unmatched, exempted=exempted, max_dz=max_dz)
