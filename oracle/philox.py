"""Philox4x32-10 (test infrastructure; see the package docstring).

Written from the generator's published definition: J. K. Salmon, M. A. Moraes,
R. O. Dror, D. E. Shaw, "Parallel Random Numbers: As Easy as 1, 2, 3", SC'11,
Sec. 4.2 (Philox-4x32: two 32x32->64 multiplications per round, Weyl-sequence
key schedule, ten rounds).  Pinned by the authors' known-answer vectors in
``tests/golden/philox4x32_10_kat.txt``.

Draws used by the hot path (the CUDA side implements the same definition in
its own code):

* sampling uniform for (seed, step, sample b, site n):
  key = (seed & 0xffffffff, seed >> 32), counter = (n, b, step & 0xffffffff,
  step >> 32), u = (x0 >> 8) * 2**-24, which is exact in float32 and float64;
* growth noise for (seed, tensor t, row r, col c):
  key as above, counter = (c, r, t, 0x6e717367), Box-Muller on (x0, x1).
"""
import numpy as np

M0 = 0xD2511F53
M1 = 0xCD9E8D57
W0 = 0x9E3779B9
W1 = 0xBB67AE85
MASK = 0xFFFFFFFF
GROW_TAG = 0x6E717367


def _mulhilo(a, b):
    prod = (a.astype(np.uint64) * np.uint64(b))
    return (prod >> np.uint64(32)) & np.uint64(MASK), prod & np.uint64(MASK)


def philox4x32_10(ctr, key):
    """Ten Philox rounds on counters ``ctr`` (4 uint arrays) with key (k0, k1).

    Each round: (hi0, lo0) = M0 * c0, (hi1, lo1) = M1 * c2;
    c <- (hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0); then the key is bumped by the
    Weyl constants (W0, W1) before the next round.
    """
    c0, c1, c2, c3 = [np.asarray(c, dtype=np.uint64) & np.uint64(MASK) for c in ctr]
    k0 = np.asarray(key[0], dtype=np.uint64) & np.uint64(MASK)
    k1 = np.asarray(key[1], dtype=np.uint64) & np.uint64(MASK)
    for r in range(10):
        if r > 0:
            k0 = (k0 + np.uint64(W0)) & np.uint64(MASK)
            k1 = (k1 + np.uint64(W1)) & np.uint64(MASK)
        hi0, lo0 = _mulhilo(c0, M0)
        hi1, lo1 = _mulhilo(c2, M1)
        c0, c1, c2, c3 = hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0
    return c0, c1, c2, c3


def _key(seed):
    seed = int(seed)
    return (seed & MASK, (seed >> 32) & MASK)


def word_to_uniform(x):
    """Top 24 bits of a 32-bit word as a uniform in [0, 1)."""
    return (np.asarray(x, dtype=np.uint64) >> np.uint64(8)).astype(np.float64) * 2.0 ** -24


def sampling_uniforms(seed, step, B, N, sample_offset=0):
    """Uniforms u[b, n] for samples b = offset..offset+B-1 and sites n (sampling order)."""
    n = np.arange(N, dtype=np.uint64)[None, :]
    b = (np.arange(B, dtype=np.uint64) + np.uint64(sample_offset))[:, None]
    step = int(step)
    shape = (B, N)
    x0, _, _, _ = philox4x32_10(
        (np.broadcast_to(n, shape), np.broadcast_to(b, shape),
         np.full(shape, step & MASK, dtype=np.uint64),
         np.full(shape, (step >> 32) & MASK, dtype=np.uint64)),
        _key(seed))
    return word_to_uniform(x0)


def growth_normals(seed, tensor_id, rows, cols):
    """Standard normals z[r, c] for one tensor of the growth step (Box-Muller)."""
    r = np.arange(rows, dtype=np.uint64)[:, None]
    c = np.arange(cols, dtype=np.uint64)[None, :]
    shape = (rows, cols)
    x0, x1, _, _ = philox4x32_10(
        (np.broadcast_to(c, shape), np.broadcast_to(r, shape),
         np.full(shape, tensor_id, dtype=np.uint64),
         np.full(shape, GROW_TAG, dtype=np.uint64)),
        _key(seed))
    u1 = word_to_uniform(x0) + 2.0 ** -24      # (0, 1]
    u2 = word_to_uniform(x1)                   # [0, 1)
    return np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * np.pi * u2)
