"""Pins for the interval-DP oracle (Eq. (2) with f(l, r) = l + r +
p[i] p[k+1] p[j+1] + w[i][j]): brute force over every binary tree, the MCM
special case, the minimal external path length of a binary tree, and the
textbook optimal binary search tree.  A dropped weight, a weight read at the
wrong index (w[j][i], w[i][k], w[k+1][j]), a dropped rank-1 term or the wrong
tie-break fails at least one of them."""
import functools
import math
import os

import numpy as np
import pytest

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def brute_force(p, w):
    """Every full binary tree over every interval i..j, costed explicitly
    (each internal node (i, k, j) adds p[i] p[k+1] p[j+1] + w[i][j]): the
    minimum and the smallest top split achieving it."""
    n = len(p) - 1

    @functools.lru_cache(maxsize=None)
    def trees(i, j):
        if i == j:
            return [(0, -1)]
        out = []
        for k in range(i, j):
            for lc, _ in trees(i, k):
                for rc, _ in trees(k + 1, j):
                    out.append((lc + rc + int(p[i]) * int(p[k + 1]) * int(p[j + 1]) + int(w[i][j]), k))
        return out

    m = np.zeros((n, n), dtype=np.int64)
    s = np.full((n, n), -1, dtype=np.int16)
    for i in range(n):
        for j in range(i + 1, n):
            allt = trees(i, j)
            best = min(c for c, _ in allt)
            m[i, j] = best
            s[i, j] = min(k for c, k in allt if c == best)
    return m, s


@pytest.mark.parametrize("seed", range(12))
def test_brute_force(seed):
    rng = np.random.default_rng(500 + seed)
    n = int(rng.integers(1, 9))
    p = rng.integers(0, 6, n + 1).astype(np.int32)
    w = rng.integers(0, 40, (n, n)).astype(np.int64)
    if seed % 3 == 0:
        p[:] = 0                      # weight only: ties between splits are common
    m, s = oracle.interval(p, w)
    bm, bs = brute_force(p, w)
    assert np.array_equal(m, bm)
    assert np.array_equal(s, bs)


def test_lower_triangle_is_ignored():
    rng = np.random.default_rng(77)
    n = 7
    p = rng.integers(0, 6, n + 1).astype(np.int32)
    w = rng.integers(0, 40, (n, n)).astype(np.int64)
    w2 = w.copy()
    w2[np.tril_indices(n)] = -5       # never read
    assert all(np.array_equal(a, b) for a, b in zip(oracle.interval(p, w), oracle.interval(p, w2)))


def test_zero_weight_is_mcm():
    # the MCM tables (pinned separately against the textbook and brute force)
    rng = np.random.default_rng(78)
    p = rng.integers(1, 30, 41).astype(np.int32)
    m, s = oracle.interval(p, np.zeros((40, 40), dtype=np.int64))
    om, os_ = oracle.mcm(p)
    assert np.array_equal(m, om) and np.array_equal(s, os_)


def _external_path_length(leaves):
    # a complete binary tree is optimal: q = floor(log2 L) levels full, the
    # remaining L - 2^q leaves one level deeper, each adding 2 to the sum
    q = int(math.floor(math.log2(leaves)))
    return leaves * q + 2 * (leaves - 2 ** q)


def test_minimal_external_path_length():
    # p = 0 and w[i][j] = j - i + 1 (the number of leaves below a node): the
    # cost of a tree is the sum of its leaves' depths, minimal for a complete tree
    n = 150
    idx = np.arange(n)
    w = (idx[None, :] - idx[:, None] + 1).astype(np.int64)
    m, _ = oracle.interval(np.zeros(n + 1, dtype=np.int32), w)
    for i in range(0, n, 7):
        for j in range(i + 1, n, 5):
            assert m[i, j] == _external_path_length(j - i + 1), (i, j)


def test_textbook_optimal_bst():
    rows = {}
    with open(os.path.join(GOLDEN, "clrs_obst.txt")) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                key, *vals = line.split()
                rows[key] = [int(v) for v in vals]
    P, Q = rows["p"], rows["q"]
    n = len(Q)                         # gaps 0..5
    w = np.zeros((n, n), dtype=np.int64)
    for i in range(n):
        for j in range(i + 1, n):
            w[i, j] = sum(P[i:j]) + sum(Q[i:j + 1])   # p_{i+1}..p_j (P is 0-based) and q_i..q_j
    m, s = oracle.interval(np.zeros(n + 1, dtype=np.int32), w)
    assert m[0, n - 1] + sum(Q) == rows["expected_cost"][0]
    assert s[0, n - 1] + 1 == rows["root"][0]


def test_cell_from_subproblem():
    rng = np.random.default_rng(79)
    n = 30
    p = rng.integers(0, 9, n + 1).astype(np.int32)
    w = rng.integers(0, 100, (n, n)).astype(np.int64)
    m, s = oracle.interval(p, w)
    for i, j in [(0, n - 1), (3, 17), (10, 11), (12, 29)]:
        assert oracle.interval_cell(p, w, i, j) == (int(m[i, j]), int(s[i, j]))


def test_rejects_bad_input():
    with pytest.raises(oracle.OracleError):
        oracle.interval([1, -1, 2], np.zeros((2, 2), dtype=np.int64))
    w = np.zeros((2, 2), dtype=np.int64)
    w[0, 1] = -1
    with pytest.raises(oracle.OracleError):
        oracle.interval([1, 1, 2], w)
