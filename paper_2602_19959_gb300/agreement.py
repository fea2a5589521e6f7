"""PV-list agreement between two runs of the path (host-side measurement, numpy only).

Two PV lists of an event agree on a vertex when their z positions match one to one
within `tol` (0.1 mm, one bin). Agreement = matched / sum over events of max(n_a, n_b).
With exempt vertices taken out, an event's disagreements are max(u_a - x_a, u_b - x_b)
(u: unmatched vertices of a side, x: the exempt ones among them), which equals
max(n_a, n_b) - matched when nothing is exempt.

A vertex found by one side only is *exempt* when the disagreement is explained by the
measured per-bin differences of the two sides' logits: the peak decision at bin k (the
local-maximum test against every bin j of its +-5 window and the threshold test) can
only differ between the sides when |f_k - t| <= |df_k|, or when k is above the threshold
on one side and, for some j, |f_k - f_j| <= |df_k| + |df_j|; f are the reference logits,
df = logit_b - logit_a per bin and t = ln(0.01 / 0.99) the threshold on logits. A vertex
is exempt when some bin within +-4 bins of it passes that test (its peak bin is within
2 bins of the bin of its centroid). Without the exemption the number is "strict"; both are
always reported.

The peak rule keeps two peaks of one side at least 6 bins apart and a centroid within
1.5 bins of its peak, so two vertices of one side are more than 0.2 mm apart and the
matching within 0.1 mm is unique: each vertex is matched to its nearest neighbour on
the other side when that is within tol.
"""

from __future__ import annotations

import numpy as np

N_BINS = 4000
HALF_WIN = 5
THR_LOGIT = float(np.log(0.01 / 0.99))


def ambiguous_bins(f_ref: np.ndarray, df: np.ndarray) -> np.ndarray:
    """[n, 4000] bool: bins whose peak decision the per-bin differences df could flip.

    The threshold test at k can flip when |f_k - t| <= |df_k|. A comparison with a
    neighbour j of the +-5 window can flip when |f_k - f_j| <= |df_k| + |df_j|, and it
    matters only for a bin above the threshold on at least one side."""
    f_ref = np.atleast_2d(np.asarray(f_ref, np.float64))
    df = np.atleast_2d(np.asarray(df, np.float64))
    adf = np.abs(df)
    amb = np.abs(f_ref - THR_LOGIT) <= adf
    cand = np.maximum(f_ref, f_ref + df) > THR_LOGIT
    n = f_ref.shape[1]
    for d in range(1, HALF_WIN + 1):
        # pairs (k, k + d): the decision at k involves j = k + d and the one at k + d involves k
        near = np.abs(f_ref[:, :n - d] - f_ref[:, d:]) <= adf[:, :n - d] + adf[:, d:]
        amb[:, :n - d] |= near & cand[:, :n - d]
        amb[:, d:] |= near & cand[:, d:]
    return amb


def _bins(z: np.ndarray) -> np.ndarray:
    return np.clip(np.floor((z + 100.0) / 0.1), 0, N_BINS - 1).astype(np.int64)


def pv_agreement(z_a, n_a, z_b, n_b, logit_a=None, logit_b=None, tol: float = 0.1) -> dict:
    """Agreement of side b's PV lists with side a's (a = the reference).

    z_a, z_b: [n_events, max_pv] ascending z per event (only the first min(n, max_pv)
    entries are read); n_a, n_b: [n_events] counts (-1 = bypassed: must agree).
    logit_a, logit_b: [n_events, 4000] logits of both sides, for the exemption (None:
    no exemption, exempt = strict).
    Returns dict(strict, exempt, matched, total, unmatched, exempted, max_dz)."""
    n_a = np.asarray(n_a).astype(np.int64)
    n_b = np.asarray(n_b).astype(np.int64)
    if np.any((n_a < 0) != (n_b < 0)):
        bad = int(np.nonzero((n_a < 0) != (n_b < 0))[0][0])
        raise AssertionError(f"event {bad}: bypassed on one side only ({n_a[bad]}, {n_b[bad]})")
    ok = n_a >= 0
    ka = np.minimum(np.where(ok, n_a, 0), np.shape(z_a)[1])
    kb = np.minimum(np.where(ok, n_b, 0), np.shape(z_b)[1])
    total = int(np.sum(np.maximum(ka, kb)))
    # every event's list shifted by 1000 mm per event: one sorted array per side
    ea = np.repeat(np.arange(len(ka)), ka)
    eb = np.repeat(np.arange(len(kb)), kb)
    za = np.asarray(z_a, np.float64)[ea, _ranks(ka)]
    zb = np.asarray(z_b, np.float64)[eb, _ranks(kb)]
    ga, gb = za + 1000.0 * ea, zb + 1000.0 * eb
    ia = _nearest(gb, ga)                 # for each a: index of the nearest b
    da = np.abs(ga - gb[ia]) if len(gb) else np.full(len(ga), np.inf)
    ma = da <= tol
    ib = _nearest(ga, gb)
    db = np.abs(gb - ga[ib]) if len(ga) else np.full(len(gb), np.inf)
    mb = db <= tol
    matched = int(np.sum(ma))
    assert matched == int(np.sum(mb)), "matching within tol is one to one"
    max_dz = float(np.max(da[ma])) if matched else 0.0
    # per event: unmatched vertices of each side, and how many of them are exempt
    n_ev = len(ka)
    side = np.concatenate([np.zeros(int(np.sum(~ma)), np.int64), np.ones(int(np.sum(~mb)), np.int64)])
    unm_e = np.concatenate([ea[~ma], eb[~mb]])
    unm_c = np.concatenate([_bins(za[~ma]), _bins(zb[~mb])])
    ex = np.zeros(len(unm_e), bool)
    if logit_a is not None and logit_b is not None and len(unm_e):
        la, lb = np.asarray(logit_a), np.asarray(logit_b)
        for e in np.unique(unm_e):
            amb = ambiguous_bins(la[e], lb[e].astype(np.float64) - la[e])[0]
            for i in np.nonzero(unm_e == e)[0]:
                c = unm_c[i]
                ex[i] = amb[max(0, c - 4):c + 5].any()
    ua = np.bincount(unm_e[side == 0], minlength=n_ev)
    ub = np.bincount(unm_e[side == 1], minlength=n_ev)
    xa = np.bincount(unm_e[(side == 0) & ex], minlength=n_ev)
    xb = np.bincount(unm_e[(side == 1) & ex], minlength=n_ev)
    # an event's disagreements: max(n_a, n_b) - matched = max(ua, ub); those left once the
    # exempt vertices are taken out: max(ua - xa, ub - xb)
    unexplained = int(np.sum(np.maximum(ua - xa, ub - xb)))
    unmatched = int(len(unm_e))
    exempted = int(np.sum(ex))
    strict = matched / total if total else 1.0
    exempt = 1.0 - unexplained / total if total else 1.0
    return dict(strict=strict, exempt=exempt, matched=matched, total=total,
                unmatched=unmatched, exempted=exempted, max_dz=max_dz)


def _ranks(k: np.ndarray) -> np.ndarray:
    """0, 1, ..., k[0]-1, 0, 1, ..., k[1]-1, ..."""
    if len(k) == 0 or int(np.sum(k)) == 0:
        return np.zeros(0, np.int64)
    start = np.repeat(np.cumsum(k) - k, k)
    return np.arange(int(np.sum(k))) - start


def _nearest(sorted_ref: np.ndarray, x: np.ndarray) -> np.ndarray:
    """Index into sorted_ref of the element nearest to each x (0 when sorted_ref is empty)."""
    if len(sorted_ref) == 0:
        return np.zeros(len(x), np.int64)
    j = np.searchsorted(sorted_ref, x)
    lo = np.clip(j - 1, 0, len(sorted_ref) - 1)
    hi = np.clip(j, 0, len(sorted_ref) - 1)
    return np.where(np.abs(sorted_ref[lo] - x) <= np.abs(sorted_ref[hi] - x), lo, hi)
