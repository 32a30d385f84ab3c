"""Device traceback of the optimal parenthesisation: a valid post-order of
n-1 products whose evaluated cost is the oracle's m[0][n-1], equal to a plain
recursive traceback of the oracle's split table."""
import numpy as np
import pytest

import oracle
from paper_2008_01938_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dp():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2008_01938_gb300 as dp
    return dp


def _cpu_postorder(s, i, j, out):
    # explicit stack (the chain can be n-1 levels deep)
    stack = [(i, j, False)]
    while stack:
        a, b, done = stack.pop()
        if a == b:
            continue
        k = int(s[a, b])
        if done:
            out.append((a, k, b))
        else:
            stack.append((a, b, True))
            stack.append((k + 1, b, False))
            stack.append((a, k, False))
    return out


def _check(dp, p, cost="i32"):
    import torch
    n = len(p) - 1
    m, s = dp.mcm_solve(torch.from_numpy(np.asarray(p, np.int32)).cuda(), cost=cost)
    steps = dp.mcm_traceback(s)
    dp.sync_status()
    st = steps.cpu().numpy().astype(np.int64)
    om, os_ = oracle.mcm(p)
    assert st.shape == (n - 1, 3)
    if n == 1:
        return
    # a valid post-order: operands are single matrices or earlier results
    ready = {(t, t) for t in range(n)}
    cost_sum = 0
    for i, k, j in st:
        assert i <= k < j and (i, k) in ready and (k + 1, j) in ready
        ready.discard((i, k))
        ready.discard((k + 1, j))
        ready.add((i, j))
        cost_sum += int(p[i]) * int(p[k + 1]) * int(p[j + 1])
    assert ready == {(0, n - 1)}
    assert cost_sum == int(om[0, n - 1])                     # the bracketing achieves the optimum
    assert [tuple(r) for r in st] == _cpu_postorder(os_, 0, n - 1, [])


@pytest.mark.parametrize("n", [1, 2, 3, 10, 33, 100, 257, 700])
def test_traceback_random(dp, n):
    _check(dp, inputs.mcm_dims(n, 1, 32, seed=3000 + n))


def test_traceback_textbook(dp):
    # the textbook 6-matrix chain: ((A1 (A2 A3)) ((A4 A5) A6))
    import torch
    p = [30, 35, 15, 5, 10, 20, 25]
    _check(dp, p)
    _, s = dp.mcm_solve(torch.tensor(p, dtype=torch.int32, device="cuda"))
    st = [tuple(r) for r in dp.mcm_traceback(s).cpu().numpy()]
    assert st == [(1, 1, 2), (0, 0, 2), (3, 3, 4), (3, 4, 5), (0, 2, 5)]


def test_traceback_deep_chain_and_int64(dp):
    # increasing dims make the optimal tree a left comb (depth n-1)
    _check(dp, list(range(1, 302)), cost="i64")
    _check(dp, inputs.mcm_dims(500, 1, 1000, seed=3999), cost="i64")
