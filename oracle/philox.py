"""Philox4x32-10 counter-based generator (Salmon, Moraes, Dror, Shaw,
"Parallel random numbers: as easy as 1, 2, 3", SC'11, Sec. 3/4).

Written from the published definition: a 4x32-bit counter and a 2x32-bit key;
each of the 10 rounds takes two 32x32->64 products of counter words with the
multipliers, XORs the high halves with the other counter words and the key,
and the key is bumped by the Weyl constants between rounds.

The paper (arXiv 2002.07109) draws its Poisson counts, partner indices and
thinning uniforms from an unspecified generator.  This project keys every
draw by (seed; slot, atom, step, stream) so that the oracle and the GPU draw
the same numbers: see ``counter`` below.

Pinned by the known-answer vectors of the Philox paper's reference
distribution (tests/test_oracle_rng.py) and, on the GPU, by the CUDA
library's Philox4_32_10 generator.
"""
import numpy as np

_M0 = np.uint64(0xD2511F53)
_M1 = np.uint64(0xCD9E8D57)
_W0 = 0x9E3779B9
_W1 = 0xBB67AE85
_MASK = np.uint64(0xFFFFFFFF)

# Stream identifiers (top byte of counter word 3).
STREAM_O = 0        # O step Gaussians
STREAM_J1 = 1       # jump half-step after the first B half-kick
STREAM_J2 = 2       # jump half-step before the last B half-kick
POISSON_SLOT = 0x80000000  # slot flag: uniforms for Poisson chunk counts


def philox4x32_10(ctr, key):
    """Philox4x32 with 10 rounds.

    ctr: uint32 array of shape (4, n) (or broadcastable); key: pair of ints.
    Returns a uint32 array of shape (4, n).
    """
    c = [np.asarray(ctr[k], dtype=np.uint64) & _MASK for k in range(4)]
    k0 = int(key[0]) & 0xFFFFFFFF
    k1 = int(key[1]) & 0xFFFFFFFF
    for rnd in range(10):
        if rnd > 0:
            k0 = (k0 + _W0) & 0xFFFFFFFF
            k1 = (k1 + _W1) & 0xFFFFFFFF
        p0 = _M0 * c[0]
        p1 = _M1 * c[2]
        hi0, lo0 = p0 >> np.uint64(32), p0 & _MASK
        hi1, lo1 = p1 >> np.uint64(32), p1 & _MASK
        c = [hi1 ^ c[1] ^ np.uint64(k0), lo1, hi0 ^ c[3] ^ np.uint64(k1), lo0]
    return np.stack([x.astype(np.uint32) for x in c])


def counter(slot, atom, step, stream):
    """Counter words for one draw: (slot, atom, step mod 2^32,
    stream << 24 | (step >> 32) mod 2^24)."""
    slot = np.asarray(slot, dtype=np.uint64)
    atom = np.asarray(atom, dtype=np.uint64)
    step = np.asarray(step, dtype=np.uint64)
    slot, atom, step = np.broadcast_arrays(slot, atom, step)
    c3 = (np.uint64(stream) << np.uint64(24)) | ((step >> np.uint64(32)) & np.uint64(0xFFFFFF))
    return np.stack([slot & _MASK, atom & _MASK, step & _MASK, c3])


def seed_key(seed):
    seed = int(seed)
    return (seed & 0xFFFFFFFF, (seed >> 32) & 0xFFFFFFFF)


def draw(seed, slot, atom, step, stream):
    """Four uint32 words per (slot, atom) for the given step and stream."""
    return philox4x32_10(counter(slot, atom, step, stream), seed_key(seed))


def u24(x):
    """Uniform on [0, 1) with 24 bits: (x >> 8) * 2^-24 (exact in float32)."""
    return (np.asarray(x, dtype=np.uint32) >> np.uint32(8)).astype(np.float64) * 2.0 ** -24


def u24_open0(x):
    """Uniform on (0, 1] with 24 bits: ((x >> 8) + 1) * 2^-24."""
    return ((np.asarray(x, dtype=np.uint32) >> np.uint32(8)).astype(np.float64) + 1.0) * 2.0 ** -24


def u53(x1, x2):
    """Uniform on [0, 1) with 53 bits from two words: ((x1>>5)*2^26 + (x2>>6)) * 2^-53."""
    a = (np.asarray(x1, dtype=np.uint64) >> np.uint64(5)).astype(np.float64)
    b = (np.asarray(x2, dtype=np.uint64) >> np.uint64(6)).astype(np.float64)
    return (a * 67108864.0 + b) * 2.0 ** -53


def index_below(x0, n):
    """Uniform integer in [0, n): high 32 bits of the 64-bit product x0 * n."""
    return ((np.asarray(x0, dtype=np.uint64) * np.asarray(n, dtype=np.uint64)) >> np.uint64(32)).astype(np.int64)
