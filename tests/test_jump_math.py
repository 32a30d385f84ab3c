"""The identities behind the (+) S-DP path for long tables, checked on the CPU
against plain polynomial long division and the oracle's tables.

With (x) = + modulo 2^32, Eq. (1) is a linear recurrence over Z/2^32 with
the monic characteristic polynomial chi(x) = x^{a_1} - sum_j x^{a_1 - a_j}.
The GPU path relies on three facts (small random cases, exact integers):
  (J)  ST[N + t] = sum_s r_s ST[s + t], where sum_s r_s x^s = x^N mod chi;
  (R)  the remainder of a product c (degree <= 2 a_1 - 2) modulo chi is
       r[e] = c[e] + sum_j h[e + a_j] over a_1 <= e + a_j <= 2 a_1 - 2, with
       h[d] = sum_m g[m] c[d + m] and g the recurrence's impulse response
       (g[0] = 1, g[m] = sum_j g[m - a_j]);
  (G)  x^N mod chi = r with r[a_1 - 1 - t] = g[M + t] - sum over a_j <= t of
       g[M + t - a_j], M = N - a_1 + 1, for N >= a_1.
Nothing here imports the CUDA path; the GPU parity tests check the kernels.
"""
import random

import numpy as np

import oracle

MOD = 1 << 32


def chi(a):
    """Coefficients of chi, lowest degree first (degree a_1, monic)."""
    A = a[0]
    c = [0] * (A + 1)
    c[A] = 1
    for aj in a:
        c[A - aj] = (c[A - aj] - 1) % MOD
    return c


def poly_mod(p, a):
    """Remainder of p modulo chi by schoolbook long division (chi is monic)."""
    A = a[0]
    ch = chi(a)
    p = [x % MOD for x in p]
    for d in range(len(p) - 1, A - 1, -1):
        q = p[d]
        if q:
            for i in range(A + 1):
                p[d - A + i] = (p[d - A + i] - q * ch[i]) % MOD
    return (p + [0] * A)[:A]


def x_pow_mod(N, a):
    return poly_mod([0] * N + [1], a)


def impulse(a, count):
    g = [0] * count
    g[0] = 1
    for m in range(1, count):
        g[m] = sum(g[m - aj] for aj in a if m - aj >= 0) % MOD
    return g


def cases(seed, count):
    rng = random.Random(seed)
    for _ in range(count):
        A = rng.randint(2, 14)
        extra = rng.sample(range(1, A), min(rng.randint(0, 4), A - 1))
        yield rng, sorted(set([A] + extra), reverse=True)


def test_window_identity():
    for rng, a in cases(1, 40):
        A = a[0]
        preset = [rng.getrandbits(32) for _ in range(A)]
        n = 40 * A
        st = [int(x) for x in oracle.sdp(np.array(preset, np.uint32), n, np.array(a, np.int32), "add")]
        for _ in range(3):
            N = rng.randint(A, n - 2 * A)
            r = x_pow_mod(N, a)
            for t in range(A):
                assert sum(r[s] * st[s + t] for s in range(A)) % MOD == st[N + t], (a, N, t)


def test_reduction_through_the_impulse_response():
    for rng, a in cases(2, 60):
        A = a[0]
        c = [rng.getrandbits(32) for _ in range(2 * A - 1)]
        g = impulse(a, A - 1)
        h = [sum(g[m] * c[d + m] for m in range(A - 1) if d + m <= 2 * A - 2) % MOD for d in range(A, 2 * A - 1)]
        r = []
        for e in range(A):
            v = c[e] + sum(h[e + aj - A] for aj in a if A <= e + aj <= 2 * A - 2)
            r.append(v % MOD)
        assert r == poly_mod(c, a), a


def test_power_read_off_the_impulse_response():
    for rng, a in cases(3, 60):
        A = a[0]
        N = rng.randint(A, 20 * A)
        g = impulse(a, N + 1)
        M = N - A + 1
        r = [0] * A
        for t in range(A):
            r[A - 1 - t] = (g[M + t] - sum(g[M + t - aj] for aj in a if aj <= t)) % MOD
        assert r == x_pow_mod(N, a), (a, N)


def test_chi_reduces_the_recurrence():
    """x^m chi(x) maps to zero under x^m -> ST[m]: the recurrence itself."""
    for rng, a in cases(4, 20):
        A = a[0]
        preset = [rng.getrandbits(32) for _ in range(A)]
        st = [int(x) for x in oracle.sdp(np.array(preset, np.uint32), 6 * A, np.array(a, np.int32), "add")]
        ch = chi(a)
        for m in range(0, 5 * A):
            assert sum(ch[i] * st[m + i] for i in range(A + 1)) % MOD == 0


def middle_product(u, z):
    """out[t] = sum_s u[s] z[t + s] for t < len(u) (z has 2 len(u) - 1 values)."""
    A = len(u)
    return [sum(u[s] * z[t + s] for s in range(A)) % MOD for t in range(A)]


def test_transposed_karatsuba_middle_product():
    """(K) The windows and reductions of the (+) path are middle products
    out[t] = sum_s u[s] z[t + s]. With u = u0 | u1 and z viewed from 0, h
    and 2h (h = len(u) / 2), three half-size middle products give them:
    P1 = M(u0 + u1, z[h:]), P2 = M(u0, z[:] - z[h:]), P3 = M(u1, z[2h:] -
    z[h:]); out[:h] = P1 + P2 and out[h:] = P1 + P3. Exact over Z/2^32,
    including values near 2^32 (checked against the direct sum)."""
    rng = random.Random(11)
    for A in [2, 4, 8, 16, 64]:
        for _ in range(5):
            u = [rng.randrange(MOD) for _ in range(A)]
            z = [rng.randrange(MOD) for _ in range(2 * A - 1)]
            h = A // 2
            zz = z + [0]  # one slack value so the views below have 2h - 1 entries each
            u0, u1 = u[:h], u[h:]
            up = [(x + y) % MOD for x, y in zip(u0, u1)]
            z1 = zz[h:h + 2 * h - 1]
            d0 = [(zz[i] - zz[h + i]) % MOD for i in range(2 * h - 1)]
            d2 = [(zz[2 * h + i] - zz[h + i]) % MOD for i in range(2 * h - 1)]
            p1, p2, p3 = middle_product(up, z1), middle_product(u0, d0), middle_product(u1, d2)
            got = [(x + y) % MOD for x, y in zip(p1, p2)] + [(x + y) % MOD for x, y in zip(p1, p3)]
            assert got == middle_product(u, z), A
