"""Counter-based random source and shot sampler.

SplitMix64 (Steele, Lea and Flood, "Fast splittable pseudorandom number generators",
OOPSLA 2014): output i of the stream with seed s is mix(s + (i + 1) * 0x9E3779B97F4A7C15)
where mix is the SplitMix64 finaliser.  A 53-bit uniform in [0, 1) is (z >> 11) * 2^-53.

A shot draws mechanism j of shot b from counter b * n_mech + j: x_j = [u < p_j].  The
detector outcome is m = H x mod 2 and the true class is l . x mod 2 (Sec. 2.4).
"""
from __future__ import annotations

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, counters: np.ndarray) -> np.ndarray:
    """Output `counters` (uint64 array) of the SplitMix64 stream seeded with `seed`."""
    with np.errstate(over="ignore"):
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + (counters.astype(np.uint64) + np.uint64(1)) * _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        return z ^ (z >> np.uint64(31))


def uniform53(seed: int, counters: np.ndarray) -> np.ndarray:
    return (splitmix64(seed, counters) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def sample_shots(dem, n_shots: int, seed: int, first_shot: int = 0):
    """Sample `n_shots` error patterns.  Returns (det uint8 [B, n_det], obs uint8 [B, n_obs]).

    Shot b uses counters (first_shot + b) * n_mech + j, so any block of shots can be
    regenerated on its own.
    """
    n = dem.n_mech
    det = np.zeros((n_shots, dem.n_det), dtype=np.uint8)
    obs = np.zeros((n_shots, dem.n_obs), dtype=np.uint8)
    p = np.asarray(dem.p, dtype=np.float64)
    chunk = max(1, (1 << 22) // max(n, 1))
    for b0 in range(0, n_shots, chunk):
        b1 = min(n_shots, b0 + chunk)
        shots = np.arange(first_shot + b0, first_shot + b1, dtype=np.uint64)
        ctr = shots[:, None] * np.uint64(n) + np.arange(n, dtype=np.uint64)[None, :]
        x = uniform53(seed, ctr) < p[None, :]
        for j in range(n):
            col = x[:, j]
            if not col.any():
                continue
            for i in dem.mech_dets[j]:
                det[b0:b1, i] ^= col
            for o in dem.mech_obs[j]:
                obs[b0:b1, o] ^= col
    return det, obs
