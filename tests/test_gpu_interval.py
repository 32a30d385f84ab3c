"""GPU parity for the interval DP with a per-cell weight (Eq. (2) with
f(l, r) = l + r + p[i] p[k+1] p[j+1] + w[i][j]): the CUDA path through the C
ABI against the CPU oracle, m and s element by element, bit-exact.  The
interval DP is built for int32 costs only; the host refusal of int64 is
checked without a GPU in test_abi.py."""
import hashlib
import json
import os

import numpy as np
import pytest

import oracle
from paper_2008_01938_gb300 import inputs

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "fullsize.json")


@pytest.fixture(scope="module")
def dp():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2008_01938_gb300 as dp
    return dp


def _solve(dp, p, w, cost):
    import torch
    wt = torch.from_numpy(np.ascontiguousarray(w, dtype=np.int32)).cuda()
    m, s = dp.interval_dp_solve(torch.from_numpy(np.asarray(p, np.int32)).cuda(), wt, cost=cost)
    dp.sync_status()
    return m.cpu().numpy(), s.cpu().numpy()


def _check(dp, inst, cost):
    m, s = _solve(dp, inst.p, inst.w, cost)
    om, os_ = oracle.interval(inst.p, inst.w)
    bad = np.argwhere((m.astype(np.int64) != om) | (s != os_))
    assert bad.size == 0, f"{len(bad)} cells differ, first {bad[:5].tolist()}"


@pytest.mark.parametrize("n", [1, 2, 3, 31, 32, 33, 64, 65, 97, 200, 257, 400])
def test_parity_int32_random(dp, n):
    _check(dp, inputs.interval_random(n, 8, 200, seed=4000 + n), "i32")


@pytest.mark.parametrize("n", [2, 33, 129, 500])
def test_parity_optimal_bst(dp, n):
    # no rank-1 term: every candidate of a cell differs only in its two operands
    _check(dp, inputs.interval_obst(n, 9, seed=6000 + n), "i32")


@pytest.mark.parametrize("wmax", [1 << 16, 1 << 20, 5_000_000])
def test_large_weights_small_packing_chunks(dp, wmax):
    # cost bounds of about 2^24, 2^28 and 2^30.5 leave 5, 3 and 1 packing bits
    inst = inputs.interval_random(300, 4, wmax, seed=wmax % 1000)
    _check(dp, inst, "i32")


def test_ties_everywhere(dp):
    # constant weight, no rank-1 term: the cost of a cell is w times the
    # number of products, the same for every tree, so every split ties
    n = 150
    w = np.triu(np.full((n, n), 3, dtype=np.int64), 1)
    _check(dp, inputs.IntervalInstance(np.zeros(n + 1, dtype=np.int32), w), "i32")


def test_zero_weight_is_mcm(dp):
    import torch
    p = inputs.mcm_dims(300, 1, 32, seed=61)
    m, s = _solve(dp, p, np.zeros((300, 300), dtype=np.int32), "i32")
    mm, ms = dp.mcm_solve(torch.from_numpy(p).cuda(), cost="i32")
    dp.sync_status()
    assert np.array_equal(m, mm.cpu().numpy()) and np.array_equal(s, ms.cpu().numpy())


def test_lower_triangle_is_not_read(dp):
    inst = inputs.interval_random(130, 6, 500, seed=62)
    w = inst.w.copy()
    w[np.tril_indices(130)] = -7
    m, s = _solve(dp, inst.p, w, "i32")
    om, os_ = oracle.interval(inst.p, inst.w)
    assert np.array_equal(m.astype(np.int64), om) and np.array_equal(s, os_)


def test_invalid_and_overflow_reported(dp):
    import torch
    from paper_2008_01938_gb300.native import DP_EINVAL, DP_EOVERFLOW, DpError
    inst = inputs.interval_random(70, 5, 100, seed=63)
    p = torch.from_numpy(inst.p).cuda()
    w = torch.from_numpy(inst.w.astype(np.int32)).cuda()
    w[3, 40] = -1
    dp.interval_dp_solve(p, w)
    with pytest.raises(DpError) as e:
        dp.sync_status()
    assert e.value.code == DP_EINVAL
    w[3, 40] = 1 << 25                                 # 69 * 2^25 >= 2^31
    dp.interval_dp_solve(p, w)
    with pytest.raises(DpError) as e:
        dp.sync_status()
    assert e.value.code == DP_EOVERFLOW
    w[3, 40] = 5
    p[9] = -2
    dp.interval_dp_solve(p, w)
    with pytest.raises(DpError) as e:
        dp.sync_status()
    assert e.value.code == DP_EINVAL
    # the context stays usable
    _check(dp, inputs.interval_random(90, 5, 100, seed=64), "i32")


def _sha(a):
    return hashlib.sha256(np.ascontiguousarray(a).tobytes()).hexdigest()


def _bellman_ok(inst, m, i, j):
    """The recurrence holds at (i, j) on the GPU table itself."""
    if i == j:
        return m[i, j] == 0
    p = inst.p.astype(np.int64)
    k = np.arange(i, j)
    cand = m[i, i:j].astype(np.int64) + m[i + 1:j + 1, j].astype(np.int64) + p[i] * p[k + 1] * p[j + 1]
    return int(cand.min()) + int(inst.w[i, j]) == int(m[i, j])


def test_full_size_optimal_bst_4096(dp):
    """The 4096-cell optimal-BST instance (frequencies U[1,4] / U[0,4], seed 5)
    the benchmark runs: whole-table SHA-256 against the oracle's (written by
    tests/golden/make_golden.py), oracle cells, and the recurrence on samples."""
    g = json.load(open(GOLDEN)).get("interval_obst_n4096_seed5") if os.path.exists(GOLDEN) else None
    if g is None:
        pytest.skip("golden entry not generated")
    inst = inputs.interval_obst(4096, 4, seed=5)
    m, s = _solve(dp, inst.p, inst.w, "i32")
    for i, j, mv, sv in g["cells"]:
        assert (int(m[i, j]), int(s[i, j])) == (mv, sv)
    assert _sha(m.astype("<i4")) == g["m_sha256"]
    assert _sha(s.astype("<i2")) == g["s_sha256"]
    rng = np.random.default_rng(1)
    for _ in range(200):
        i, j = sorted(rng.integers(0, 4096, 2).tolist())
        assert _bellman_ok(inst, m, i, j)
    for _ in range(5):
        i = int(rng.integers(0, 3500))
        j = i + int(rng.integers(1, 400))
        assert oracle.interval_cell(inst.p, inst.w, i, j) == (int(m[i, j]), int(s[i, j]))
