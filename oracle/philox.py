"""Philox4x32-10 counter-based generator, written from its published definition
(Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy as 1, 2, 3",
SC'11, Sec. 3 and Table 2). Test infrastructure only (see package header).

One round maps counter (c0, c1, c2, c3) and key (k0, k1) to
    (hi(M1*c2) ^ c1 ^ k0,  lo(M1*c2),  hi(M0*c0) ^ c3 ^ k1,  lo(M0*c0))
with M0 = 0xD2511F53, M1 = 0xCD9E8D57. Between rounds the key is bumped by
the Weyl constants (0x9E3779B9, 0xBB67AE85). Ten rounds.

Pinned by the published known-answer vectors in tests/golden/philox4x32_10_kat.txt.
"""
from __future__ import annotations

import numpy as np

M0 = np.uint64(0xD2511F53)
M1 = np.uint64(0xCD9E8D57)
W0 = np.uint32(0x9E3779B9)
W1 = np.uint32(0xBB67AE85)
_MASK = np.uint64(0xFFFFFFFF)


def philox4x32_10(ctr: np.ndarray, key: np.ndarray) -> np.ndarray:
    """ctr: uint32 [..., 4]; key: uint32 [..., 2] (broadcast). Returns uint32 [..., 4]."""
    c = [np.asarray(ctr[..., i], dtype=np.uint32).copy() for i in range(4)]
    k0 = np.asarray(key[..., 0], dtype=np.uint32).copy()
    k1 = np.asarray(key[..., 1], dtype=np.uint32).copy()
    with np.errstate(over="ignore"):
        for rnd in range(10):
            p0 = M0 * c[0].astype(np.uint64)
            p1 = M1 * c[2].astype(np.uint64)
            hi0 = (p0 >> np.uint64(32)).astype(np.uint32)
            lo0 = (p0 & _MASK).astype(np.uint32)
            hi1 = (p1 >> np.uint64(32)).astype(np.uint32)
            lo1 = (p1 & _MASK).astype(np.uint32)
            c = [hi1 ^ c[1] ^ k0, lo1, hi0 ^ c[3] ^ k1, lo0]
            if rnd != 9:
                k0 = k0 + W0
                k1 = k1 + W1
    return np.stack(np.broadcast_arrays(*c), axis=-1).astype(np.uint32)


def noise_words(seed: int, n_dofs: int, n_samples: int) -> np.ndarray:
    """The raw uint32 stream of the sampler's noise: word j of sample s is
    word (j mod 4) of Philox4x32-10(key = (seed lo32, seed hi32),
    ctr = (q lo32, q hi32, s, 0)), q = j div 4. Returns uint32 [n_samples, n_dofs]."""
    nq = (n_dofs + 3) // 4
    q = np.arange(nq, dtype=np.uint64)
    s = np.arange(n_samples, dtype=np.uint32)
    ctr = np.zeros((n_samples, nq, 4), dtype=np.uint32)
    ctr[..., 0] = (q & _MASK).astype(np.uint32)[None, :]
    ctr[..., 1] = (q >> np.uint64(32)).astype(np.uint32)[None, :]
    ctr[..., 2] = s[:, None]
    key = np.array([seed & 0xFFFFFFFF, (seed >> 32) & 0xFFFFFFFF], dtype=np.uint32)
    out = philox4x32_10(ctr, key)
    return out.reshape(n_samples, nq * 4)[:, :n_dofs]
