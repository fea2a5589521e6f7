"""Seeded synthetic collision events in Structure-of-Arrays form.

The paper's workload is simulated LHCb Run 3 minimum-bias crossings: on average
5.6 proton-proton collision vertices per event (§1) and nine reconstructed
VELO-track features per track (§2). Neither that simulation nor detector data is
available, so events are drawn here from a seeded toy model with that shape:

standard events (the 16-, 1000- and 20000-event workloads)
    N_PV = max(1, Poisson(5.6)); z_PV ~ N(0, 45 mm) clipped to [-100, 300] mm;
    Poisson(25) tracks per PV with poca_z = z_PV + N(0, 0.08 mm);
    Poisson(15) background tracks with poca_z ~ U[-100, 300) mm.

uneven events (the 50000-event batching workload)
    N_PV ~ U{1..12}; Poisson(25) tracks per PV as above; background count
    min(400, floor(Pareto(alpha=2, x_m=5))), uniform z.

Other features, per track: poca_x, poca_y ~ N(0, 0.05 mm); tx, ty ~ N(0, 0.15);
three POCA-ellipsoid widths ~ LogNormal(ln 0.05, 0.5); quality ~ U(0, 1).
Tracks are shuffled within each event. Features are float32, one contiguous
array per feature; ``offsets[e] .. offsets[e+1]`` are event e's tracks.

Only numpy's PCG64 generator is used, and the order of draws is fixed by this
file, so a (kind, n_events, seed) triple names one dataset on every machine.
"""

from __future__ import annotations

from dataclasses import dataclass

import numpy as np

FEATURE_NAMES = ("poca_x", "poca_y", "poca_z", "tx", "ty", "w1", "w2", "w3", "quality")
Z_MIN, Z_MAX = -100.0, 300.0


@dataclass
class EventBatch:
    features: np.ndarray      # float32 [9, n_tracks], C-contiguous, order = FEATURE_NAMES
    offsets: np.ndarray       # int32 [n_events + 1]
    n_pv: np.ndarray          # int32 [n_events], generated (true) PV count
    pv_z: np.ndarray          # float64 [sum n_pv], generated PV z positions, event-major

    @property
    def n_events(self) -> int:
        return int(self.offsets.shape[0] - 1)

    @property
    def n_tracks(self) -> int:
        return int(self.features.shape[1])

    def tracks_per_event(self) -> np.ndarray:
        return np.diff(self.offsets.astype(np.int64))

    def subset(self, start: int, stop: int) -> "EventBatch":
        """Events [start, stop) as a new batch with offsets rebased to 0."""
        a, b = int(self.offsets[start]), int(self.offsets[stop])
        pv_off = np.concatenate([[0], np.cumsum(self.n_pv)])
        return EventBatch(
            features=np.ascontiguousarray(self.features[:, a:b]),
            offsets=(self.offsets[start:stop + 1] - a).astype(np.int32),
            n_pv=self.n_pv[start:stop].copy(),
            pv_z=self.pv_z[pv_off[start]:pv_off[stop]].copy(),
        )


def _assemble(rng: np.random.Generator, n_events: int, n_pv: np.ndarray,
              n_bkg: np.ndarray) -> EventBatch:
    tot_pv = int(n_pv.sum())
    z_pv = np.clip(rng.normal(0.0, 45.0, tot_pv), Z_MIN, Z_MAX)
    n_trk_pv = rng.poisson(25.0, tot_pv)
    pv_of_track = np.repeat(np.arange(tot_pv), n_trk_pv)
    z_sig = z_pv[pv_of_track] + rng.normal(0.0, 0.08, pv_of_track.size)
    z_bkg = rng.uniform(Z_MIN, Z_MAX, int(n_bkg.sum()))

    ev_of_pv = np.repeat(np.arange(n_events), n_pv)
    ev_sig = ev_of_pv[pv_of_track]
    ev_bkg = np.repeat(np.arange(n_events), n_bkg)
    ev = np.concatenate([ev_sig, ev_bkg])
    z = np.concatenate([z_sig, z_bkg])
    # random order of tracks inside each event (events stay contiguous)
    order = np.lexsort((rng.random(ev.size), ev))
    ev, z = ev[order], z[order]
    n = z.size

    feats = np.empty((9, n), dtype=np.float32)
    feats[0] = rng.normal(0.0, 0.05, n)
    feats[1] = rng.normal(0.0, 0.05, n)
    feats[2] = z
    feats[3] = rng.normal(0.0, 0.15, n)
    feats[4] = rng.normal(0.0, 0.15, n)
    for k in (5, 6, 7):
        feats[k] = rng.lognormal(np.log(0.05), 0.5, n)
    feats[8] = rng.uniform(0.0, 1.0, n)

    counts = np.bincount(ev, minlength=n_events)
    offsets = np.zeros(n_events + 1, dtype=np.int64)
    np.cumsum(counts, out=offsets[1:])
    if offsets[-1] >= 2**31:
        raise ValueError("too many tracks for int32 offsets")
    return EventBatch(features=np.ascontiguousarray(feats), offsets=offsets.astype(np.int32),
                      n_pv=n_pv.astype(np.int32), pv_z=z_pv)


def generate_standard(n_events: int, seed: int) -> EventBatch:
    """Events with N_PV = max(1, Poisson(5.6)) and Poisson(15) uniform background tracks."""
    rng = np.random.default_rng(seed)
    n_pv = np.maximum(1, rng.poisson(5.6, n_events))
    n_bkg = rng.poisson(15.0, n_events)
    return _assemble(rng, n_events, n_pv, n_bkg)


def generate_uneven(n_events: int, seed: int) -> EventBatch:
    """Events with N_PV ~ U{1..12} and a heavy-tailed background count.

    Background = min(400, floor(X)) with X classical Pareto(alpha=2, x_m=5),
    drawn as x_m * (1 + Lomax(alpha)).
    """
    rng = np.random.default_rng(seed)
    n_pv = rng.integers(1, 13, n_events)
    x = 5.0 * (1.0 + rng.pareto(2.0, n_events))
    n_bkg = np.minimum(400, np.floor(x)).astype(np.int64)
    return _assemble(rng, n_events, n_pv, n_bkg)


def generate(kind: str, n_events: int, seed: int) -> EventBatch:
    if kind == "standard":
        return generate_standard(n_events, seed)
    if kind == "uneven":
        return generate_uneven(n_events, seed)
    raise ValueError(f"unknown event kind {kind!r}")


def concat_batches(batches) -> EventBatch:
    feats = np.concatenate([b.features for b in batches], axis=1)
    offs = [np.zeros(1, dtype=np.int64)]
    base = 0
    for b in batches:
        offs.append(b.offsets[1:].astype(np.int64) + base)
        base += b.n_tracks
    return EventBatch(features=np.ascontiguousarray(feats),
                      offsets=np.concatenate(offs).astype(np.int32),
                      n_pv=np.concatenate([b.n_pv for b in batches]),
                      pv_z=np.concatenate([b.pv_z for b in batches]))
