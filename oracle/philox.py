"""Counter-based random numbers: Philox4x32-10 (Salmon, Moraes, Dror, Shaw,
"Parallel random numbers: as easy as 1, 2, 3", SC 2011), written from its
published definition, and the normal draws built on it.

Used where the simulation needs more random numbers than can be passed in as
inputs (one independent phase screen per training sample): both the oracle
and the CUDA path implement this same generator, so the noise is identical
on both sides.

* state: counter (c0, c1, c2, c3), key (k0, k1), 32-bit words;
* round: with M0 = 0xD2511F53, M1 = 0xCD9E8D57,
      (hi0, lo0) = M0 * c0,  (hi1, lo1) = M1 * c2   (64-bit products)
      c <- (hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0)
  then k0 += 0x9E3779B9, k1 += 0xBB67AE85 (Weyl sequence), ten rounds
  (the key bump follows every round but the last);
* uniform in (0, 1): u = (x + 0.5) / 2^32;
* normals: Box-Muller, (sqrt(-2 ln u0) cos 2 pi u1, sqrt(-2 ln u0) sin 2 pi u1)
  and the same for (u2, u3): four normals per counter.

Counter layout used by the screen noise: c = (element pair index low 32
bits, high 32 bits, sample index, stream id), key = (seed low, seed high).
"""
import numpy as np

M0 = np.uint64(0xD2511F53)
M1 = np.uint64(0xCD9E8D57)
W0 = np.uint32(0x9E3779B9)
W1 = np.uint32(0xBB67AE85)
MASK = np.uint64(0xFFFFFFFF)


def philox4x32_10(c0, c1, c2, c3, k0, k1):
    """Vectorised Philox4x32-10; uint32 arrays in, four uint32 arrays out."""
    c0 = np.asarray(c0, dtype=np.uint32)
    c1 = np.asarray(c1, dtype=np.uint32)
    c2 = np.asarray(c2, dtype=np.uint32)
    c3 = np.asarray(c3, dtype=np.uint32)
    k0 = np.asarray(k0, dtype=np.uint32) + np.zeros_like(c0)
    k1 = np.asarray(k1, dtype=np.uint32) + np.zeros_like(c0)
    for r in range(10):
        p0 = c0.astype(np.uint64) * M0
        p1 = c2.astype(np.uint64) * M1
        hi0 = (p0 >> np.uint64(32)).astype(np.uint32)
        lo0 = (p0 & MASK).astype(np.uint32)
        hi1 = (p1 >> np.uint64(32)).astype(np.uint32)
        lo1 = (p1 & MASK).astype(np.uint32)
        c0, c1, c2, c3 = hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0
        if r < 9:
            k0 = k0 + W0
            k1 = k1 + W1
    return c0, c1, c2, c3


def uniform(x):
    return (np.asarray(x, dtype=np.float64) + 0.5) * (1.0 / 4294967296.0)


def normals4(c0, c1, c2, c3, seed):
    """Four standard normals per counter (arrays of shape c0.shape)."""
    seed = int(seed)
    x = philox4x32_10(c0, c1, c2, c3, seed & 0xFFFFFFFF, (seed >> 32) & 0xFFFFFFFF)
    u = [uniform(v) for v in x]
    r0 = np.sqrt(-2.0 * np.log(u[0]))
    r1 = np.sqrt(-2.0 * np.log(u[2]))
    t0 = 2.0 * np.pi * u[1]
    t1 = 2.0 * np.pi * u[3]
    return r0 * np.cos(t0), r0 * np.sin(t0), r1 * np.cos(t1), r1 * np.sin(t1)


def complex_noise(seed, sample, stream, n):
    """n complex values (real, imaginary standard normals) for one sample:
    counter i covers elements 2i and 2i+1 (n rounded up to even)."""
    m = (n + 1) // 2
    i = np.arange(m, dtype=np.uint64)
    lo = (i & MASK).astype(np.uint32)
    hi = (i >> np.uint64(32)).astype(np.uint32)
    g0, g1, g2, g3 = normals4(lo, hi, np.full(m, sample, np.uint32),
                              np.full(m, stream, np.uint32), seed)
    out = np.empty(2 * m, dtype=np.complex128)
    out[0::2] = g0 + 1j * g1
    out[1::2] = g2 + 1j * g3
    return out[:n]
