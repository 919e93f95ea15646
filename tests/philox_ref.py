"""Philox4x32-10 in plain Python (Salmon et al., SC 2011), for replaying GPU draws on the CPU."""

M0, M1 = 0xD2511F53, 0xCD9E8D57
W0, W1 = 0x9E3779B9, 0xBB67AE85
MASK = 0xFFFFFFFF


def philox4x32_10(ctr, key):
    x0, x1, x2, x3 = ctr
    k0, k1 = key
    for r in range(10):
        if r:
            k0, k1 = (k0 + W0) & MASK, (k1 + W1) & MASK
        p0, p1 = M0 * x0, M1 * x2
        hi0, lo0, hi1, lo1 = p0 >> 32, p0 & MASK, p1 >> 32, p1 & MASK
        x0, x1, x2, x3 = hi1 ^ x1 ^ k0, lo1, hi0 ^ x3 ^ k1, lo0
    return x0, x1, x2, x3


def uniform(seed, step, chain, j):
    """The j-th uniform double in (0, 1) of (seed; step, chain)."""
    r = philox4x32_10((step & MASK, (step >> 32) & MASK, chain & MASK, (j >> 1) & MASK),
                      (seed & MASK, (seed >> 32) & MASK))
    a, b = (r[2], r[3]) if j & 1 else (r[0], r[1])
    m = ((a >> 6) << 27) | (b >> 5)
    return (m + 0.5) * 2.0 ** -53
