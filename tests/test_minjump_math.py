"""The identities behind the (min) S-DP path for long tables, checked on the
CPU against the recursive definition and the oracle's tables.

With (x) = min, unrolling Eq. (1) down to the preset gives ST[N] = min over
s in C_N of ST[s], where C_N = {N} for N < a_1 and C_N = union_j C_{N - a_j}
otherwise.  The GPU path relies on four facts (small random cases):
  (W)  ST[N + t] = min_{s in C_N} ST[s + t] for 0 <= t < a_1;
  (P)  C_{N+M} is the sumset C_N + C_M reduced from the top down (a degree
       d >= a_1 replaced by the degrees d - a_j);
  (B)  that reduction may fold whole blocks of floor(a_k / 32) 32-bit words
       at once when a_k >= 32 (no fold lands in its own block);
  (F)  if C_N is the full set [0, a_1), so is C_{N+M} for every M >= 0.
Nothing here imports the CUDA path; the GPU parity tests check the kernels.
"""
import random

import numpy as np

import oracle


def c_sets(a, count):
    """C_N for N < count by the recursive definition, as Python ints (bit s = s in C_N)."""
    A = a[0]
    c = []
    for N in range(count):
        if N < A:
            c.append(1 << N)
        else:
            v = 0
            for aj in a:
                v |= c[N - aj]
            c.append(v)
    return c


def sumset(x, y):
    r, s = 0, 0
    while x:
        if x & 1:
            r |= y << s
        x >>= 1
        s += 1
    return r


def reduce_bits(c, a):
    """Top-down, one degree at a time."""
    A = a[0]
    for d in range(c.bit_length() - 1, A - 1, -1):
        if (c >> d) & 1:
            c &= ~(1 << d)
            for aj in a:
                c |= 1 << (d - aj)
    return c


def reduce_blocks(c, a):
    """The kernel's order: 32-bit words from the top, floor(a_k / 32) words at
    a time; each block's degrees >= a_1 are snapshotted, folded, cleared."""
    A, ak = a[0], a[-1]
    Wb = ak // 32
    nw = max((c.bit_length() + 31) // 32, 1)
    words = [(c >> (32 * i)) & 0xFFFFFFFF for i in range(2 * nw)]
    wlo = A // 32
    hi_mask = (~((1 << (A % 32)) - 1)) & 0xFFFFFFFF if A % 32 else 0xFFFFFFFF
    top = len(words) - 1
    while top >= wlo:
        bot = max(top - Wb + 1, wlo)
        blk = [(words[w] & hi_mask) if w == wlo else words[w] for w in range(bot, top + 1)]
        for wi, bits in enumerate(blk):
            if not bits:
                continue
            for aj in a:
                tb = 32 * (bot + wi) - aj
                v = bits << tb if tb >= 0 else bits >> (-tb)
                assert v < (1 << (32 * bot)), "a fold landed in its own block"
                for i in range(len(words)):
                    words[i] |= (v >> (32 * i)) & 0xFFFFFFFF
        for w in range(bot, top + 1):
            words[w] = (words[w] & ~hi_mask & 0xFFFFFFFF) if w == wlo else 0
        top -= Wb
    return sum(w << (32 * i) for i, w in enumerate(words))


def cases(seed, count, min_ak=1):
    rng = random.Random(seed)
    for _ in range(count):
        A = rng.randint(max(2, min_ak), 90)
        k = rng.randint(1, 5)
        a = sorted({A} | {rng.randint(min_ak, A) for _ in range(k - 1)}, reverse=True)
        yield a


def test_window_identity_W():
    rng = np.random.default_rng(7)
    for a in cases(1, 25):
        A = a[0]
        n = 6 * A + 40
        pre = rng.integers(0, 2 ** 32, size=A, dtype=np.uint64).astype(np.uint32)
        st = oracle.sdp(pre, n, a, "min")
        c = c_sets(a, n)
        for N in range(0, n - A, max(1, A // 3)):
            for t in range(A):
                want = min(int(st[s + t]) for s in range(A) if (c[N] >> s) & 1)
                assert want == int(st[N + t]), (a, N, t)


def test_product_rule_P():
    for a in cases(2, 25):
        c = c_sets(a, 8 * a[0] + 50)
        for N, M in [(0, 3), (a[0], a[0]), (3 * a[0] + 1, 2 * a[0] - 1), (4 * a[0], 4 * a[0] - 7)]:
            if N + M < len(c):
                assert reduce_bits(sumset(c[N], c[M]), a) == c[N + M], (a, N, M)


def test_block_reduction_B():
    rng = random.Random(3)
    for a in cases(4, 40, min_ak=32):
        A = a[0]
        for _ in range(5):
            prod = rng.getrandbits(2 * A - 1)
            assert reduce_blocks(prod, a) == reduce_bits(prod, a), a
    # the 2^26 workload's offsets and a product of two dense sets
    from paper_2008_01938_gb300 import inputs
    a = [int(x) for x in inputs.sdp_instance_big().offsets]
    prod = random.Random(5).getrandbits(2 * a[0] - 1)
    assert reduce_blocks(prod, a) == reduce_bits(prod, a)


def test_full_set_is_absorbing_F():
    seen = 0
    for a in cases(6, 40):
        A = a[0]
        full = (1 << A) - 1
        c = c_sets(a, 40 * A)
        first = next((N for N in range(A, len(c)) if c[N] == full), None)
        if first is None:
            continue
        seen += 1
        assert all(c[N] == full for N in range(first, len(c))), a
    assert seen >= 10  # the property was exercised
