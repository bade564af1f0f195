"""Test-side restatement of Philox4x32-10 (Salmon et al., SC'11) and of the GPU snapshot
generator's use of it, for checking doa_synth_ula bit-for-bit on the random words."""
import numpy as np

M0, M1, W0, W1 = 0xD2511F53, 0xCD9E8D57, 0x9E3779B9, 0xBB67AE85
MASK = 0xFFFFFFFF


def philox4x32_10(ctr, key):
    c = list(ctr)
    k = list(key)
    for _ in range(10):
        p0 = M0 * c[0]
        p1 = M1 * c[2]
        c = [(p1 >> 32) ^ c[1] ^ k[0], p1 & MASK, (p0 >> 32) ^ c[3] ^ k[1], p0 & MASK]
        k = [(k[0] + W0) & MASK, (k[1] + W1) & MASK]
    return c


def box_muller(a, b):
    u1 = np.float32((np.float32(a) + np.float32(1.0)) * np.float32(2.3283064365386963e-10))
    u2 = np.float32(np.float32(b) * np.float32(2.3283064365386963e-10))
    r = np.sqrt(np.float32(-2.0) * np.log(u1))
    return r * np.cos(2 * np.pi * np.float64(u2)), r * np.sin(2 * np.pi * np.float64(u2))


def synth_ula(d, angles, snr_db, M, N, seed, first):
    """float64 reference of the generator: same counters, same draw order."""
    B = len(d)
    X = np.zeros((B, M, N), dtype=np.complex128)
    inv2 = 1 / np.sqrt(2.0)
    for b in range(B):
        inst = first + b
        A = np.exp(1j * np.pi * np.arange(M)[:, None] * np.sin(np.radians(angles[b, :d[b]]))[None, :])
        sigma = np.sqrt(10 ** (-snr_db[b] / 10)) * inv2
        for t in range(N):
            ctr = [t, inst & MASK, (inst >> 32) & MASK, 0]
            key = [seed & MASK, (seed >> 32) & MASK]
            s = np.zeros(d[b], dtype=np.complex128)
            for i in range(0, d[b], 2):
                w = philox4x32_10(ctr, key)
                ctr[3] += 1
                g0 = box_muller(w[0], w[1])
                g1 = box_muller(w[2], w[3])
                s[i] = (g0[0] + 1j * g0[1]) * inv2
                if i + 1 < d[b]:
                    s[i + 1] = (g1[0] + 1j * g1[1]) * inv2
            for m in range(0, M, 2):
                w = philox4x32_10(ctr, key)
                ctr[3] += 1
                for h, (a, bb) in enumerate(((w[0], w[1]), (w[2], w[3]))):
                    if m + h < M:
                        g = box_muller(a, bb)
                        X[b, m + h, t] = (g[0] + 1j * g[1]) * sigma + A[m + h] @ s
    return X
