"""Counter-based random numbers for the synthetic RIOT workloads.

Philox4x32-10 is the counter-based generator of Salmon, Moraes, Dror & Shaw,
"Parallel random numbers: as easy as 1, 2, 3" (SC'11): a 10-round bijection
on a 128-bit counter keyed by a 64-bit key.  Each round multiplies two of the
four 32-bit words by fixed odd constants, keeps the high and low halves of
the products and mixes them with the other two words and the round key; the
key is bumped by two Weyl constants between rounds.

Normals come from the Box-Muller transform (Box & Muller, 1958): two
uniforms u1, u2 in (0, 1) give sqrt(-2 ln u1) * (cos 2 pi u2, sin 2 pi u2).

Stream layout (the same definition is implemented independently in the CUDA
library, which draws the RIOT sketch on the device):
  key     = (seed & 0xffffffff, seed >> 32)
  counter = (c & 0xffffffff, c >> 32, stream, 0) for call number c
  one call gives words w0..w3 -> uniforms u_j = (w_j + 0.5) * 2**-32
  element i of the stream is call c = i // 4, slot r = i % 4:
      r = 0: sqrt(-2 ln u0) cos(2 pi u1)     r = 1: sqrt(-2 ln u0) sin(2 pi u1)
      r = 2: sqrt(-2 ln u2) cos(2 pi u3)     r = 3: sqrt(-2 ln u2) sin(2 pi u3)

This module holds no arithmetic of the assimilation method itself: it only
turns (seed, stream, index) into numbers.
"""
import numpy as np

PHILOX_M0 = np.uint64(0xD2511F53)
PHILOX_M1 = np.uint64(0xCD9E8D57)
PHILOX_W0 = np.uint64(0x9E3779B9)
PHILOX_W1 = np.uint64(0xBB67AE85)
MASK32 = np.uint64(0xFFFFFFFF)


def philox4x32_10(ctr, key):
    """Apply Philox4x32-10 to counters.

    ctr: uint32-valued array of shape (..., 4); key: uint32-valued array of
    shape (..., 2) broadcastable against ctr[..., :2].  Returns uint32 words
    of shape (..., 4).
    """
    c = np.asarray(ctr, dtype=np.uint64) & MASK32
    k = np.asarray(key, dtype=np.uint64) & MASK32
    c0, c1, c2, c3 = c[..., 0], c[..., 1], c[..., 2], c[..., 3]
    k0 = np.broadcast_to(k[..., 0], c0.shape).copy()
    k1 = np.broadcast_to(k[..., 1], c0.shape).copy()
    for rnd in range(10):
        if rnd > 0:
            k0 = (k0 + PHILOX_W0) & MASK32
            k1 = (k1 + PHILOX_W1) & MASK32
        p0 = PHILOX_M0 * c0          # < 2**64: exact in uint64
        p1 = PHILOX_M1 * c2
        hi0, lo0 = p0 >> np.uint64(32), p0 & MASK32
        hi1, lo1 = p1 >> np.uint64(32), p1 & MASK32
        c0, c1, c2, c3 = (hi1 ^ c1 ^ k0), lo1, (hi0 ^ c3 ^ k1), lo0
    return np.stack([c0, c1, c2, c3], axis=-1).astype(np.uint32)


def _key(seed):
    seed = int(seed) & 0xFFFFFFFFFFFFFFFF
    return np.array([seed & 0xFFFFFFFF, seed >> 32], dtype=np.uint64)


def raw_words(seed, stream, ncalls, first_call=0):
    """uint32 words of calls first_call .. first_call+ncalls-1, shape (ncalls, 4)."""
    calls = np.arange(first_call, first_call + ncalls, dtype=np.uint64)
    ctr = np.zeros((ncalls, 4), dtype=np.uint64)
    ctr[:, 0] = calls & MASK32
    ctr[:, 1] = calls >> np.uint64(32)
    ctr[:, 2] = np.uint64(int(stream) & 0xFFFFFFFF)
    return philox4x32_10(ctr, _key(seed))


def uniforms(seed, stream, count):
    """count uniforms in (0, 1) as float64 (the u_j of the stream layout)."""
    ncalls = (count + 3) // 4
    w = raw_words(seed, stream, ncalls).reshape(-1)[:count]
    return (w.astype(np.float64) + 0.5) * (2.0 ** -32)


def normals(seed, stream, count, first=0):
    """Standard normals, elements first .. first+count-1 of the stream (float64)."""
    if count <= 0:
        return np.zeros(0)
    c_lo = first // 4
    c_hi = (first + count + 3) // 4
    w = raw_words(seed, stream, c_hi - c_lo, first_call=c_lo).astype(np.float64)
    u = (w + 0.5) * (2.0 ** -32)
    r0 = np.sqrt(-2.0 * np.log(u[:, 0]))
    r1 = np.sqrt(-2.0 * np.log(u[:, 2]))
    a0 = 2.0 * np.pi * u[:, 1]
    a1 = 2.0 * np.pi * u[:, 3]
    z = np.stack([r0 * np.cos(a0), r0 * np.sin(a0), r1 * np.cos(a1), r1 * np.sin(a1)], axis=1)
    z = z.reshape(-1)
    off = first - 4 * c_lo
    return z[off:off + count]


def choose_indices(seed, stream, n, m):
    """m distinct indices of range(n), sorted, by a partial Fisher-Yates shuffle
    driven by the stream's uint32 words."""
    if m > n:
        raise ValueError("m > n")
    perm = np.arange(n, dtype=np.int64)
    w = raw_words(seed, stream, (m + 3) // 4).reshape(-1)[:m]
    for i in range(m):
        j = i + int(w[i]) % (n - i)
        perm[i], perm[j] = perm[j], perm[i]
    return np.sort(perm[:m])
