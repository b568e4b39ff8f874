"""Counter-based random draws for the synthetic TBPM workloads.

Every random number a workload needs (random phases of the initial states,
Anderson onsite disorder, vacancy selection, per-bond hopping noise, the
per-sample sizes of a batch) is a pure function of (seed, stream, index), so
the same array can be regenerated independently by any consumer and no state
is carried between calls.

The mixing function is the SplitMix64 output function (Steele, Lea & Flood,
"Fast splittable pseudorandom number generators", OOPSLA 2014), used here as
a keyed hash of a counter:

    key(seed, stream)  = mix64(seed + GAMMA * (stream + 1))
    u64(seed, stream, i) = mix64(key + GAMMA * (i + 1))
    mix64(x) = z ^ (z >> 31),  z = ((y ^ (y >> 27)) * C2),  y = ((x ^ (x >> 30)) * C1)

with GAMMA = 0x9E3779B97F4A7C15, C1 = 0xBF58476D1CE4E5B9,
C2 = 0x94D049BB133111EB, all arithmetic modulo 2^64.  A uniform double in
[0, 1) takes the top 53 bits.  This module holds no arithmetic of the
propagation method itself.
"""
from __future__ import annotations

import numpy as np

GAMMA = np.uint64(0x9E3779B97F4A7C15)
C1 = np.uint64(0xBF58476D1CE4E5B9)
C2 = np.uint64(0x94D049BB133111EB)
_S30 = np.uint64(30)
_S27 = np.uint64(27)
_S31 = np.uint64(31)
_S11 = np.uint64(11)

# Stream numbers of the synthetic workloads.  Random phases of state p use
# stream PHASE0 + p.
PHASE0 = 1
ONSITE = 100
VACANCY = 101
BOND_NOISE = 102
BATCH = 103


def mix64(x: np.ndarray) -> np.ndarray:
    """SplitMix64 output function, elementwise on uint64 (wraps mod 2^64)."""
    x = np.asarray(x, dtype=np.uint64)
    with np.errstate(over="ignore"):
        y = (x ^ (x >> _S30)) * C1
        z = (y ^ (y >> _S27)) * C2
    return z ^ (z >> _S31)


def stream_key(seed: int, stream: int) -> np.uint64:
    with np.errstate(over="ignore"):
        v = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + GAMMA * np.uint64(stream + 1)
    return mix64(np.array([v], dtype=np.uint64))[0]


def u64(seed: int, stream: int, idx: np.ndarray | int) -> np.ndarray:
    """Raw 64-bit draws for counters ``idx`` of (seed, stream)."""
    k = stream_key(seed, stream)
    i = np.asarray(idx, dtype=np.uint64)
    with np.errstate(over="ignore"):
        return mix64(k + GAMMA * (i + np.uint64(1)))


def uniform(seed: int, stream: int, n: int, offset: int = 0) -> np.ndarray:
    """n doubles in [0, 1) for counters offset .. offset+n-1."""
    idx = np.arange(offset, offset + n, dtype=np.uint64)
    return (u64(seed, stream, idx) >> _S11).astype(np.float64) * (2.0 ** -53)


def uniform_range(seed: int, stream: int, n: int, lo: float, hi: float) -> np.ndarray:
    return lo + (hi - lo) * uniform(seed, stream, n)


def normal(seed: int, stream: int, n: int) -> np.ndarray:
    """n standard normal draws by Box-Muller on counters 2i and 2i+1."""
    u = uniform(seed, stream, 2 * n)
    u1 = 1.0 - u[0::2]          # (0, 1]: log is finite
    u2 = u[1::2]
    return np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * np.pi * u2)


def phases(seed: int, n_states: int, n_orb: int) -> np.ndarray:
    """Random phases theta[p, i] in [0, 2 pi) of state p, orbital i."""
    out = np.empty((n_states, n_orb), dtype=np.float64)
    for p in range(n_states):
        out[p] = 2.0 * np.pi * uniform(seed, PHASE0 + p, n_orb)
    return out


def phases_torch(seed: int, n_states: int, n_orb: int, device="cpu"):
    """:func:`phases` computed with torch on ``device`` (the same numbers: the
    mixing runs on int64 with wrap-around products and masked logical shifts)."""
    import torch

    def s64(v: int) -> int:
        v &= 0xFFFFFFFFFFFFFFFF
        return v - (1 << 64) if v >= (1 << 63) else v

    def lsr(x, k):
        return (x >> k) & ((1 << (64 - k)) - 1)

    def mix(x):
        y = (x ^ lsr(x, 30)) * s64(int(C1))
        z = (y ^ lsr(y, 27)) * s64(int(C2))
        return z ^ lsr(z, 31)

    out = torch.empty((n_states, n_orb), dtype=torch.float64, device=device)
    i1 = torch.arange(1, n_orb + 1, dtype=torch.int64, device=device)
    for p in range(n_states):
        k = s64(int(stream_key(seed, PHASE0 + p)))
        u = mix(i1 * s64(int(GAMMA)) + k)
        out[p] = lsr(u, 11).to(torch.float64) * (2.0 ** -53) * (2.0 * np.pi)
    return out
