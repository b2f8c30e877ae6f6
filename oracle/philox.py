"""Philox4x32-10 counter-based generator (Salmon, Moraes, Dror and Shaw,
"Parallel random numbers: as easy as 1, 2, 3", SC'11) and the Gaussian test
vectors drawn from it. Written here from the published definition, in numpy
uint32/uint64 arithmetic; the CUDA side has its own implementation. Test
infrastructure only.

Sketch-vector recipe (shared definition, two implementations): element
e = i * M + c of the row-major n x M block uses Philox block b = e // 4 with
counter (b mod 2^32, b div 2^32, 0, 0) and key (seed mod 2^32, seed div 2^32).
The four output words x0..x3 become uniforms u = (x + 0.5) / 2^32; the pair
(x0, x1) gives the normals of slots 0, 1 and (x2, x3) those of slots 2, 3 by
Box-Muller, r = sqrt(-2 ln u_a), z = r cos(2 pi u_b), r sin(2 pi u_b),
evaluated in FP64 and rounded to bfloat16 (round to nearest even).
"""
import numpy as np

M0 = np.uint64(0xD2511F53)
M1 = np.uint64(0xCD9E8D57)
W0 = np.uint32(0x9E3779B9)
W1 = np.uint32(0xBB67AE85)
MASK = np.uint64(0xFFFFFFFF)


def philox4x32_10(ctr, key):
    """ctr: uint32 array [..., 4]; key: uint32 array [..., 2]. Returns [..., 4]."""
    c = [np.asarray(ctr[..., j], dtype=np.uint64) for j in range(4)]
    k0 = np.asarray(key[..., 0], dtype=np.uint32).copy()
    k1 = np.asarray(key[..., 1], dtype=np.uint32).copy()
    for r in range(10):
        p0 = M0 * c[0]
        p1 = M1 * c[2]
        hi0, lo0 = p0 >> np.uint64(32), p0 & MASK
        hi1, lo1 = p1 >> np.uint64(32), p1 & MASK
        c = [hi1 ^ c[1] ^ k0.astype(np.uint64), lo1, hi0 ^ c[3] ^ k1.astype(np.uint64), lo0]
        if r < 9:
            k0 = (k0 + W0).astype(np.uint32)
            k1 = (k1 + W1).astype(np.uint32)
    return np.stack([x.astype(np.uint32) for x in c], axis=-1)


def to_bf16_bits(x):
    """Round FP64 values to bfloat16 (nearest even); returns uint16 bits."""
    f = np.asarray(x, dtype=np.float64).astype(np.float32)
    # a double -> float -> bf16 double rounding would differ from direct
    # rounding only if the float rounding lands exactly on a bf16 tie; redo
    # those ties from the double value.
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> np.uint64(16)) & np.uint64(1)
    rounded = ((u + np.uint64(0x7FFF) + lsb) >> np.uint64(16)).astype(np.uint16)
    tie = (u & np.uint64(0xFFFF)) == np.uint64(0x8000)
    if tie.any():
        xd = np.asarray(x, dtype=np.float64)[tie]
        down = (u[tie] >> np.uint64(16)).astype(np.uint16)
        up = down + np.uint16(1)
        vd = bf16_bits_to_f64(down)
        vu = bf16_bits_to_f64(up)
        pick_up = np.abs(xd - vu) < np.abs(xd - vd)
        exact = np.abs(xd - vu) == np.abs(xd - vd)
        pick_up = pick_up | (exact & ((down & np.uint16(1)) == 1))
        rounded[tie] = np.where(pick_up, up, down)
    return rounded


def bf16_bits_to_f64(bits):
    b = np.asarray(bits, dtype=np.uint16).astype(np.uint32) << np.uint32(16)
    return b.view(np.float32).astype(np.float64)


def gaussian_sketch(n, M, seed):
    """n x M block of N(0, 1) test vectors rounded to bfloat16 (recipe above).
    Returns (float64 values, uint16 bf16 bits)."""
    total = n * M
    nblk = (total + 3) // 4
    b = np.arange(nblk, dtype=np.uint64)
    ctr = np.zeros((nblk, 4), dtype=np.uint32)
    ctr[:, 0] = (b & MASK).astype(np.uint32)
    ctr[:, 1] = (b >> np.uint64(32)).astype(np.uint32)
    key = np.empty((nblk, 2), dtype=np.uint32)
    key[:, 0] = np.uint32(seed & 0xFFFFFFFF)
    key[:, 1] = np.uint32((seed >> 32) & 0xFFFFFFFF)
    x = philox4x32_10(ctr, key).astype(np.float64)
    u = (x + 0.5) * (1.0 / 4294967296.0)
    r01 = np.sqrt(-2.0 * np.log(u[:, 0]))
    r23 = np.sqrt(-2.0 * np.log(u[:, 2]))
    z = np.empty((nblk, 4))
    z[:, 0] = r01 * np.cos(2.0 * np.pi * u[:, 1])
    z[:, 1] = r01 * np.sin(2.0 * np.pi * u[:, 1])
    z[:, 2] = r23 * np.cos(2.0 * np.pi * u[:, 3])
    z[:, 3] = r23 * np.sin(2.0 * np.pi * u[:, 3])
    bits = to_bf16_bits(z.ravel()[:total]).reshape(n, M)
    return bf16_bits_to_f64(bits), bits
