"""Counter-based batch sampler oracle (the 100 000-point uniform batch of Sec. 6
"Training", drawn from Philox4x32-10).

TEST INFRASTRUCTURE ONLY: imported by the tests; never by the product path.

Philox4x32-10 follows its published definition (Salmon, Moraes, Dror and Shaw,
"Parallel Random Numbers: As Easy as 1, 2, 3", SC'11): ten rounds of
  (c0, c1, c2, c3) <- (hi(B c2) ^ c1 ^ k0, lo(B c2), hi(A c0) ^ c3 ^ k1, lo(A c0))
with A = 0xD2511F53, B = 0xCD9E8D57, and the key bumped by the Weyl constants
(0x9E3779B9, 0xBB67AE85) between rounds.

Sampler reading (this library's own convention): point n of brick b at step s
uses counter (n, b, s, 0) and key (seed mod 2^32, seed >> 32); coordinate d is
2 * (r_d >> 8) * 2^-24 - 1, an exactly representable float32 in [-1, 1).
"""
from __future__ import annotations

import numpy as np

_A = np.uint64(0xD2511F53)
_B = np.uint64(0xCD9E8D57)
_W0 = np.uint64(0x9E3779B9)
_W1 = np.uint64(0xBB67AE85)
_MASK = np.uint64(0xFFFFFFFF)


def philox4x32_10(ctr, key):
    """ctr uint32 [..., 4], key uint32 [..., 2] -> uint32 [..., 4]."""
    c = np.asarray(ctr, dtype=np.uint64) & _MASK
    k = np.asarray(key, dtype=np.uint64) & _MASK
    c0, c1, c2, c3 = (c[..., i].copy() for i in range(4))
    k0, k1 = k[..., 0].copy(), k[..., 1].copy()
    for r in range(10):
        if r > 0:
            k0 = (k0 + _W0) & _MASK
            k1 = (k1 + _W1) & _MASK
        pa = _A * c0
        pb = _B * c2
        hi_a, lo_a = pa >> np.uint64(32), pa & _MASK
        hi_b, lo_b = pb >> np.uint64(32), pb & _MASK
        c0, c1, c2, c3 = (hi_b ^ c1 ^ k0) & _MASK, lo_b, (hi_a ^ c3 ^ k1) & _MASK, lo_a
    return np.stack([c0, c1, c2, c3], axis=-1).astype(np.uint32)


def sample_points(seed: int, step: int, brick: int, n: int) -> np.ndarray:
    """The n points of `brick` at training step `step`, float32 [n, 3], unsorted."""
    idx = np.arange(n, dtype=np.uint64)
    ctr = np.zeros((n, 4), dtype=np.uint64)
    ctr[:, 0] = idx & _MASK
    ctr[:, 1] = brick
    ctr[:, 2] = step & 0xFFFFFFFF
    key = np.array([seed & 0xFFFFFFFF, (seed >> 32) & 0xFFFFFFFF], dtype=np.uint64)
    r = philox4x32_10(ctr, np.broadcast_to(key, (n, 2)))
    u = (r[:, :3] >> np.uint32(8)).astype(np.float64) * 2.0 ** -24
    return (2.0 * u - 1.0).astype(np.float32)
