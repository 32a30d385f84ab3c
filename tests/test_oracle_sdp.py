"""Pins for the S-DP oracle (Definition 1 / Fig. 1): Fibonacci by fast
doubling, top-down recursion, the Fig. 3 instance worked by hand, the Fig. 2
pipeline schedule simulated step by step, the k = 1 periodic copy and the
algebraic invariants of min and wrapping +."""
import functools
import os

import numpy as np
import pytest

import oracle
from paper_2008_01938_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
M32 = (1 << 32) - 1


def fib_pair(i):
    """(F(i), F(i+1)) mod 2^32 by fast doubling."""
    if i == 0:
        return 0, 1
    a, b = fib_pair(i >> 1)
    c = (a * ((2 * b - a) & M32)) & M32
    d = (a * a + b * b) & M32
    return (d, (c + d) & M32) if i & 1 else (c, d)


def test_fibonacci_both_presets():
    n = 5000
    f = oracle.sdp([0, 1], n, [2, 1], "add")
    for i in [0, 1, 2, 10, 47, 48, 93, 1000, 4999]:
        assert int(f[i]) == fib_pair(i)[0]
    # the paper's preset ST[0] = ST[1] = 1 gives F(i + 1)
    g = oracle.sdp([1, 1], n, [2, 1], "add")
    for i in [0, 1, 5, 100, 4999]:
        assert int(g[i]) == fib_pair(i + 1)[0]


def test_fibonacci_large_index():
    n = 1 << 20
    f = oracle.sdp([0, 1], n, [2, 1], "add")
    for i in [n - 1, n - 2, 123457]:
        assert int(f[i]) == fib_pair(i)[0]


def _topdown(preset, n, a, op):
    a1 = a[0]

    @functools.lru_cache(maxsize=None)
    def st(i):
        if i < a1:
            return int(preset[i])
        vals = [st(i - aj) for aj in a]
        if op == "min":
            return min(vals)
        return sum(vals) & M32

    return [st(i) for i in range(n)]


@pytest.mark.parametrize("seed", range(8))
@pytest.mark.parametrize("op", ["min", "add"])
def test_topdown_recursion(seed, op):
    rng = np.random.default_rng(seed)
    k = int(rng.integers(1, 6))
    a = sorted(rng.choice(np.arange(1, 12), size=k, replace=False).tolist(), reverse=True)
    n = int(rng.integers(0, 80))
    preset = rng.integers(0, 1 << 32, a[0], dtype=np.uint64).astype(np.uint32)
    got = oracle.sdp(preset, n, a, op)
    assert got.tolist() == _topdown(preset, n, a, op)


def test_fig3_instance_by_hand():
    rows = {}
    with open(os.path.join(GOLDEN, "fig3_k3.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                key, *vals = line.split()
                rows[key] = [int(v) for v in vals]
    for op in ("min", "add"):
        got = oracle.sdp(rows["preset"], 10, rows["offsets"], op)
        assert got.tolist() == rows[op]


def _pipeline_fig2(preset, n, a, op):
    """Step-by-step simulation of the paper's pipeline algorithm (Fig. 2):
    for head i = a_1 .. n+k-2, thread j works on ST[i-j+1] when
    a_1 <= i-j+1 < n, assigning ST[i_j - a_1] (j = 1) or combining
    ST[i_j - a_j] into it (j > 1).  Threads of one step read before any of
    them writes."""
    k = len(a)
    st = [0] * max(n, a[0])
    st[:a[0]] = [int(x) for x in preset[:a[0]]]
    for i in range(a[0], n + k - 1):
        updates = []
        for j in range(1, k + 1):
            ij = i - j + 1
            if a[0] <= ij < n:
                src = st[ij - a[j - 1]]
                if j == 1:
                    updates.append((ij, src))
                else:
                    cur = st[ij]
                    updates.append((ij, min(cur, src) if op == "min" else (cur + src) & M32))
        for idx, v in updates:
            st[idx] = v
    return st[:n]


@pytest.mark.parametrize("seed", range(6))
def test_fig2_pipeline_schedule_agrees(seed):
    rng = np.random.default_rng(100 + seed)
    k = int(rng.integers(2, 6))
    a = sorted(rng.choice(np.arange(1, 14), size=k, replace=False).tolist(), reverse=True)
    n = 120
    preset = rng.integers(0, 1000, a[0]).astype(np.uint32)
    for op in ("min", "add"):
        assert oracle.sdp(preset, n, a, op).tolist() == _pipeline_fig2(preset, n, a, op)


def test_k1_periodic_copy():
    preset = np.arange(7, dtype=np.uint32) * 3 + 1
    for op in ("min", "add"):
        st = oracle.sdp(preset, 100, [7], op)
        assert all(int(st[i]) == int(preset[i % 7]) for i in range(100))


def test_invariants():
    inst = inputs.sdp_random(n=30000, k=9, amin=40, amax=700, seed=8, preset_hi=1 << 20)
    x = inst.preset.astype(np.uint32)
    y = inputs.SplitMix64(77).randint(0, 1 << 20, x.size).astype(np.uint32)
    n, a = inst.n, inst.offsets
    # (+): linear modulo 2^32
    sx, sy = oracle.sdp(x, n, a, "add"), oracle.sdp(y, n, a, "add")
    assert np.array_equal(oracle.sdp((x + y).astype(np.uint32), n, a, "add"), (sx + sy).astype(np.uint32))
    # (min): distributes over elementwise min; values come from the preset; shift
    mx, my = oracle.sdp(x, n, a, "min"), oracle.sdp(y, n, a, "min")
    assert np.array_equal(oracle.sdp(np.minimum(x, y), n, a, "min"), np.minimum(mx, my))
    assert set(np.unique(mx).tolist()) <= set(x.tolist())
    assert np.array_equal(oracle.sdp(x + 1000, n, a, "min"), mx + 1000)


def test_short_tables_and_validation():
    st = oracle.sdp([5, 6, 7], 2, [3, 1], "min")     # n <= a_1: nothing to compute
    assert st.tolist() == [5, 6]
    with pytest.raises(oracle.OracleError):
        oracle.sdp([1, 2, 3], 10, [2, 3], "min")       # not strictly decreasing
    with pytest.raises(oracle.OracleError):
        oracle.sdp([1, 2, 3], 10, [3, 0], "min")       # offset must be > 0


# --- planted mistakes must be caught ----------------------------------------

def _mutant_sdp(preset, n, a, op, mutation):
    st = [int(v) for v in preset[:a[0]]] + [0] * max(0, n - a[0])
    for i in range(a[0], n):
        offs = a[:-1] if mutation == "dropped_offset" else a
        vals = [st[i - aj + (1 if mutation == "off_by_one" else 0)] for aj in offs]
        st[i] = min(vals) if op == "min" else sum(vals) & M32
    return st[:n]


@pytest.mark.parametrize("mutation", ["dropped_offset", "off_by_one"])
def test_pins_catch_mutants(mutation):
    n = 200
    got = _mutant_sdp([0, 1], n, [2, 1], "add", mutation)
    assert any(got[i] != fib_pair(i)[0] for i in range(n))
