"""Philox4x32-10 counter-based generator and Box-Muller normals (numpy).
TEST INFRASTRUCTURE.

Written from the published definition (Salmon, Moraes, Dror, Shaw,
"Parallel random numbers: as easy as 1, 2, 3", SC'11): a 4 x 32-bit counter
and a 2 x 32-bit key; each of 10 rounds multiplies words 0 and 2 by
0xD2511F53 and 0xCD9E8D57 (64-bit products split into hi/lo halves) and
permutes/xors them with the other words and the key; the key is bumped by the
Weyl constants 0x9E3779B9, 0xBB67AE85 between rounds.

Normals used by the time steps: element e of stream `sid` for step `step`
uses counter (e // 4, step, sid, 0) and output word e % 4.  Words come in
pairs (w0, w1), (w2, w3); u = (w + 0.5) 2^-32; the pair gives
sqrt(-2 ln u_a) cos(2 pi u_b) and sqrt(-2 ln u_a) sin(2 pi u_b).
"""
import numpy as np

M0, M1 = np.uint64(0xD2511F53), np.uint64(0xCD9E8D57)
W0, W1 = np.uint32(0x9E3779B9), np.uint32(0xBB67AE85)
MASK = np.uint64(0xFFFFFFFF)


def philox4x32_10(ctr, key):
    """ctr [..., 4] uint32, key [2] uint32 -> [..., 4] uint32."""
    c = [np.asarray(ctr[..., i], dtype=np.uint32).copy() for i in range(4)]
    k0, k1 = np.uint32(key[0]), np.uint32(key[1])
    with np.errstate(over='ignore'):
        for rnd in range(10):
            p0 = c[0].astype(np.uint64) * M0
            p1 = c[2].astype(np.uint64) * M1
            hi0, lo0 = (p0 >> np.uint64(32)).astype(np.uint32), (p0 & MASK).astype(np.uint32)
            hi1, lo1 = (p1 >> np.uint64(32)).astype(np.uint32), (p1 & MASK).astype(np.uint32)
            c = [hi1 ^ c[1] ^ k0, lo1, hi0 ^ c[3] ^ k1, lo0]
            if rnd < 9:
                k0 = np.uint32(k0 + W0)
                k1 = np.uint32(k1 + W1)
    return np.stack(c, axis=-1)


def normals(n, seed, step, sid):
    """n standard normals of stream sid at time step `step` (see module doc)."""
    nctr = (n + 3) // 4
    ctr = np.zeros((nctr, 4), dtype=np.uint32)
    ctr[:, 0] = np.arange(nctr, dtype=np.uint64).astype(np.uint32)
    ctr[:, 1] = np.uint32(step)
    ctr[:, 2] = np.uint32(sid)
    key = (np.uint32(seed & 0xFFFFFFFF), np.uint32((seed >> 32) & 0xFFFFFFFF))
    w = philox4x32_10(ctr, key).astype(np.float64)
    u = (w + 0.5) * 2.0 ** -32
    rad = np.sqrt(-2.0 * np.log(u[:, 0::2]))
    ang = 2.0 * np.pi * u[:, 1::2]
    z = np.empty((nctr, 4))
    z[:, 0] = rad[:, 0] * np.cos(ang[:, 0])
    z[:, 1] = rad[:, 0] * np.sin(ang[:, 0])
    z[:, 2] = rad[:, 1] * np.cos(ang[:, 1])
    z[:, 3] = rad[:, 1] * np.sin(ang[:, 1])
    return z.reshape(-1)[:n]
