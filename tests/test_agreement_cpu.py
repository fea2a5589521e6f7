"""The PV-list agreement measure (paper_2602_19959_gb300.agreement) on the CPU: its
vectorised matching against the plain two-pointer matching, and its exemption rule on
hand-built logits where the answer is known."""

import numpy as np

from paper_2602_19959_gb300.agreement import THR_LOGIT, ambiguous_bins, pv_agreement
from tests.helpers import match_pvs


def _lists(rng, n_events, max_pv):
    """Ascending z lists with neighbours >= 0.3 mm apart (as the peak rule guarantees),
    and a second side with some vertices moved, dropped or added."""
    za = np.zeros((n_events, max_pv), np.float32)
    zb = np.zeros((n_events, max_pv), np.float32)
    na = np.zeros(n_events, np.int32)
    nb = np.zeros(n_events, np.int32)
    for e in range(n_events):
        k = int(rng.integers(0, max_pv - 2))
        a = np.sort(rng.choice(np.arange(-333, 999), size=k, replace=False)).astype(np.float64) * 0.3
        b = a + rng.uniform(-0.12, 0.12, size=k)             # some beyond the 0.1 mm tolerance
        keep = rng.random(k) > 0.1
        b = b[keep]
        extra = rng.uniform(-100, 300, size=int(rng.integers(0, 3)))
        b = np.sort(np.concatenate([b, extra]))
        if len(b):
            b = b[np.concatenate([[True], np.diff(b) >= 0.3])][:max_pv]
        za[e, :k] = a
        zb[e, :len(b)] = b
        na[e], nb[e] = k, len(b)
    return za, na, zb, nb


def test_vectorised_matching_equals_two_pointer():
    rng = np.random.default_rng(4)
    za, na, zb, nb = _lists(rng, 200, 40)
    a = pv_agreement(za, na, zb, nb)
    matched = total = 0
    max_dz = 0.0
    for e in range(len(na)):
        pa, pb = za[e, :na[e]].astype(np.float64), zb[e, :nb[e]].astype(np.float64)
        pairs, _, _ = match_pvs(pa, pb)
        matched += len(pairs)
        total += max(na[e], nb[e])
        for i, j in pairs:
            max_dz = max(max_dz, abs(pa[i] - pb[j]))
    assert a["matched"] == matched and a["total"] == total
    assert a["unmatched"] == (int(na.sum()) - matched) + (int(nb.sum()) - matched)
    assert abs(a["max_dz"] - max_dz) < 1e-9
    assert a["strict"] == a["exempt"] == matched / total          # no logits: no exemption


def test_bypassed_events_must_agree():
    z = np.zeros((2, 4), np.float32)
    a = pv_agreement(z, np.array([-1, 0]), z, np.array([-1, 0]))
    assert a["total"] == 0 and a["strict"] == 1.0
    try:
        pv_agreement(z, np.array([-1, 0]), z, np.array([0, 0]))
    except AssertionError:
        return
    raise AssertionError("a bypass on one side only must fail")


def _bump_logits(centres, height=5.0):
    f = np.full(4000, -20.0)
    for c in centres:
        for d in range(-3, 4):
            f[c + d] = max(f[c + d], height - abs(d))
    return f


def test_exemption_follows_the_measured_per_bin_differences():
    # a near tie: bins 1000 and 1003 both at the top of a plateau-like bump, the oracle
    # picks 1000 by 1e-3, the other side has 1003 higher by 1e-3 (a flip the per-bin
    # differences of 2e-3 explain); a far vertex at 2000 with no tie is a real disagreement
    fa = _bump_logits([1000, 2000])
    fa[1003] = fa[1000] - 1e-3
    fb = fa.copy()
    fb[1003] = fa[1000] + 1e-3
    zc = lambda b: -100.0 + (b + 0.5) * 0.1                   # bin centre
    za = np.array([[zc(1000), zc(2000)]])
    zb = np.array([[zc(1003), zc(2000), zc(2500)]])           # and an extra vertex at 2500
    a = pv_agreement(za, np.array([2]), zb, np.array([3]), fa[None], fb[None])
    assert a["matched"] == 1 and a["unmatched"] == 3
    assert a["exempted"] == 2                 # the tie flip on both sides; not the extra vertex
    assert a["total"] == 3 and abs(a["strict"] - 1 / 3) < 1e-12
    assert abs(a["exempt"] - (1 - 1 / 3)) < 1e-12      # one unexplained: the extra vertex


def test_ambiguous_bins_threshold_and_window():
    f = np.full(4000, -50.0)
    f[10] = THR_LOGIT + 1e-4                   # within 2e-4 of the threshold
    f[500] = 3.0
    f[505] = 3.0 - 1e-4                        # a neighbour 5 bins away, nearly tied
    f[700] = 3.0
    f[706] = 3.0 - 1e-4                        # 6 bins away: outside the window
    df = np.full(4000, 1e-4)
    amb = ambiguous_bins(f, df)[0]
    assert amb[10] and amb[500] and amb[505]
    assert not amb[700] and not amb[706]
    assert not ambiguous_bins(f, np.zeros(4000))[0][[10, 500, 505]].any()
