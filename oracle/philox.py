"""Philox4x32-10 counter-based generator, from its published definition (Salmon, Moraes,
Dror, Shaw, "Parallel random numbers: as easy as 1, 2, 3", SC'11).

Round: with multipliers M0 = 0xD2511F53, M1 = 0xCD9E8D57 and the 64-bit products
(hi0, lo0) = M0 * c0, (hi1, lo1) = M1 * c2, the counter becomes
(hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0). Between rounds the key is bumped by the Weyl
constants (0x9E3779B9, 0xBB67AE85). Ten rounds.

Used by spec I to draw injected particles: the CUDA path implements the same generator
independently, so both sides see identical uniforms.
"""
from __future__ import annotations

import numpy as np

M0 = np.uint64(0xD2511F53)
M1 = np.uint64(0xCD9E8D57)
W0 = np.uint32(0x9E3779B9)
W1 = np.uint32(0xBB67AE85)
MASK32 = np.uint64(0xFFFFFFFF)


def philox4x32_10(ctr, key):
    """ctr: uint32 array (..., 4); key: uint32 array (..., 2). Returns uint32 (..., 4)."""
    c = [np.asarray(ctr[..., i], dtype=np.uint32) for i in range(4)]
    k0 = np.asarray(key[..., 0], dtype=np.uint32)
    k1 = np.asarray(key[..., 1], dtype=np.uint32)
    with np.errstate(over="ignore"):
        for r in range(10):
            if r > 0:
                k0 = (k0 + W0).astype(np.uint32)
                k1 = (k1 + W1).astype(np.uint32)
            p0 = M0 * c[0].astype(np.uint64)
            p1 = M1 * c[2].astype(np.uint64)
            hi0 = (p0 >> np.uint64(32)).astype(np.uint32)
            lo0 = (p0 & MASK32).astype(np.uint32)
            hi1 = (p1 >> np.uint64(32)).astype(np.uint32)
            lo1 = (p1 & MASK32).astype(np.uint32)
            c = [hi1 ^ c[1] ^ k0, lo1, hi0 ^ c[3] ^ k1, lo0]
    return np.stack(c, axis=-1)


def uniform01(u32):
    """Map uint32 to a double in the open interval (0, 1): (u + 0.5) * 2^-32."""
    return (np.asarray(u32, dtype=np.float64) + 0.5) * (2.0 ** -32)
