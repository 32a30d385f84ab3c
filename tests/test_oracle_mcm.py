"""Pins for the MCM oracle: each check is independent of the oracle's own code
(textbook values, brute force over every parenthesisation, closed forms, the
paper's Eq. (2) operand lists), chosen so that a dropped term, a wrong index,
a transposed operand or the wrong tie-break fails at least one of them."""
import functools
import itertools
import os

import numpy as np
import pytest

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _read_golden(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append(line.split())
    return rows


def brute_force_tables(p):
    """Enumerate every full parenthesisation of every sub-chain A_i..A_j and
    return the minimum cost and the smallest first-split index achieving it.
    Independent of the DP: costs are summed over explicit bracketings."""
    n = len(p) - 1

    @functools.lru_cache(maxsize=None)
    def trees(i, j):
        # all bracketings of A_i..A_j as (cost, top split k)
        if i == j:
            return [(0, -1)]
        out = []
        for k in range(i, j):
            for lc, _ in trees(i, k):
                for rc, _ in trees(k + 1, j):
                    out.append((lc + rc + p[i] * p[k + 1] * p[j + 1], k))
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


def bracketing_cost(p, s, i, j):
    """Cost of the bracketing encoded by the split table s (evaluated
    recursively, without looking at m)."""
    if i == j:
        return 0
    k = int(s[i, j])
    assert i <= k < j
    return bracketing_cost(p, s, i, k) + bracketing_cost(p, s, k + 1, j) + int(p[i]) * int(p[k + 1]) * int(p[j + 1])


def test_textbook_example():
    rows = _read_golden("clrs_6matrix.txt")
    dims = [int(x) for x in rows[0][1:]]
    m, s = oracle.mcm(dims)
    for r in rows[1:]:
        tab = m if r[0] == "m" else s
        assert tab[int(r[1]), int(r[2])] == int(r[3])


@pytest.mark.parametrize("seed", range(12))
def test_brute_force_small(seed):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(1, 9))
    hi = 2 if seed % 3 == 0 else 40      # tie-heavy dims in [1, 2] for a third
    p = [int(x) for x in rng.integers(1, hi + 1, n + 1)]
    m, s = oracle.mcm(p)
    bm, bs = brute_force_tables(p)
    assert np.array_equal(m, bm)
    assert np.array_equal(s, bs)


def test_brute_force_n9_ties():
    p = [1, 2, 1, 2, 1, 2, 1, 2, 1, 2]
    m, s = oracle.mcm(p)
    bm, bs = brute_force_tables(p)
    assert np.array_equal(m, bm) and np.array_equal(s, bs)


@pytest.mark.parametrize("c", [1, 3, 32])
def test_equal_dims_closed_form(c):
    # every bracketing of k+1 equal square matrices costs k * c^3, so every
    # split ties and the smallest one, i, must be chosen
    n = 40
    m, s = oracle.mcm([c] * (n + 1))
    for i in range(n):
        for j in range(i + 1, n):
            assert m[i, j] == (j - i) * c ** 3
            assert s[i, j] == i


def test_adjacent_pairs_closed_form():
    rng = np.random.default_rng(5)
    p = rng.integers(1, 1000, 61).astype(np.int32)
    m, s = oracle.mcm(p)
    for i in range(59):
        assert m[i, i + 1] == int(p[i]) * int(p[i + 1]) * int(p[i + 2])
        assert s[i, i + 1] == i


def test_split_table_reproduces_cost():
    rng = np.random.default_rng(11)
    p = rng.integers(1, 33, 201).astype(np.int32)
    m, s = oracle.mcm(p)
    for (i, j) in [(0, 199), (3, 150), (50, 51), (17, 180)]:
        assert bracketing_cost(p, s, i, j) == m[i, j]


def test_diagonal_and_lower_triangle():
    m, s = oracle.mcm([3, 4, 5, 6])
    assert np.all(np.tril(m) == 0)
    assert np.all(s[np.tril_indices(3)] == -1)
    m1, s1 = oracle.mcm([7, 9])
    assert m1.shape == (1, 1) and m1[0, 0] == 0 and s1[0, 0] == -1


def test_cell_by_subchain_matches_full_table():
    rng = np.random.default_rng(2)
    p = rng.integers(1, 33, 101).astype(np.int32)
    m, s = oracle.mcm(p)
    for (i, j) in [(0, 99), (10, 20), (40, 99), (5, 6)]:
        assert oracle.mcm_cell(p, i, j) == (m[i, j], s[i, j])


def test_invalid_dims_rejected():
    with pytest.raises(oracle.OracleError):
        oracle.mcm([3, 0, 5])


def test_eq2_operand_lists():
    # Section IV-B: the diagonal-major linearisation and split order
    for row in _read_golden("eq2_n5_operands.txt"):
        tgt = int(row[0])
        vals = [int(x) for x in row[1:]]
        pairs = list(zip(vals[0::2], vals[1::2]))
        assert oracle.mcm_operand_pairs(5, tgt) == pairs
    # the first n entries of the linear table are the diagonal
    assert [oracle.diag_major_index(5, r, r) for r in range(1, 6)] == [1, 2, 3, 4, 5]
    assert oracle.diag_major_index(5, 1, 5) == 15


# --- the pins above must reject plausible mistakes -------------------------

def _mutant_mcm(p, mutation):
    n = len(p) - 1
    m = np.zeros((n, n), dtype=np.int64)
    s = np.full((n, n), -1, dtype=np.int16)
    for d in range(1, n):
        for i in range(n - d):
            j = i + d
            best, bk = None, -1
            for k in range(i, j):
                if mutation == "p_k_index":
                    w = p[i] * p[k] * p[j + 1]
                elif mutation == "dropped_weight":
                    w = 0
                elif mutation == "transposed_operand":
                    w = p[i] * p[k + 1] * p[j + 1]
                else:
                    w = p[i] * p[k + 1] * p[j + 1]
                left = m[i, k]
                right = m[k + 1, j] if mutation != "transposed_operand" else m[j, k + 1] if k + 1 != j else 0
                cand = left + right + w
                if best is None or (cand < best if mutation != "ties_largest" else cand <= best):
                    best, bk = cand, k
            m[i, j], s[i, j] = best, bk
    return m, s


@pytest.mark.parametrize("mutation", ["p_k_index", "dropped_weight", "transposed_operand", "ties_largest"])
def test_pins_catch_mutants(mutation):
    rows = _read_golden("clrs_6matrix.txt")
    dims = [int(x) for x in rows[0][1:]]
    caught = False
    mm, ms = _mutant_mcm(dims, mutation)
    for r in rows[1:]:
        tab = mm if r[0] == "m" else ms
        caught |= tab[int(r[1]), int(r[2])] != int(r[3])
    c = 2
    em, es = _mutant_mcm([c] * 9, mutation)
    for i, j in itertools.combinations(range(8), 2):
        caught |= em[i, j] != (j - i) * c ** 3 or es[i, j] != i
    assert caught, mutation
