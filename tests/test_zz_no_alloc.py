"""The allocation-free MCM entry point (mcm_solve_noalloc) against mcm_solve:
two calls in a row, through the C ABI, bit-exact on m and s.  Collected last,
so it also runs after every other GPU test has used the device."""
import ctypes

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


def _noalloc(dp, p_dev):
    import torch
    n = p_dev.numel() - 1
    m = torch.full((n, n), -7, dtype=torch.int32, device=p_dev.device)
    s = torch.full((n, n), -7, dtype=torch.int16, device=p_dev.device)
    status = torch.zeros(1, dtype=torch.int32, device=p_dev.device)
    from paper_2008_01938_gb300 import api
    api.mcm_solve_noalloc(p_dev, m, s, status)
    dp.sync_status(status=status)
    return m.cpu().numpy(), s.cpu().numpy()


def _reference(dp, p_dev):
    m, s = dp.mcm_solve(p_dev, cost="i32")
    dp.sync_status()
    return m.cpu().numpy(), s.cpu().numpy()


def test_two_calls_in_a_row_match_mcm_solve(dp):
    import torch
    # the largest chain the static scratch holds, then a ragged smaller one:
    # the second call must not see anything the first one left behind
    cases = [inputs.mcm_dims(1024, 1, 32, seed=7001), inputs.mcm_dims(517, 1, 32, seed=7002)]
    outs = []
    for p in cases:
        p_dev = torch.from_numpy(np.asarray(p, np.int32)).cuda()
        outs.append((_noalloc(dp, p_dev), p_dev))
    for ((m, s), p_dev), p in zip(outs, cases):
        rm, rs = _reference(dp, p_dev)
        assert m.dtype == np.int32 and s.dtype == np.int16
        assert np.array_equal(m, rm), f"m differs in {(m != rm).sum()} cells"
        assert np.array_equal(s, rs), f"s differs in {(s != rs).sum()} cells"
    # and the ragged one against the oracle
    om, os_ = oracle.mcm(cases[1])
    (m, s), _ = outs[1]
    assert np.array_equal(m.astype(np.int64), om) and np.array_equal(s, os_)


def test_same_size_twice_and_tiny(dp):
    import torch
    for p in ([3, 9, 4, 7, 2, 5, 8, 6], inputs.mcm_dims(300, 1, 32, seed=7003), inputs.mcm_dims(300, 1, 32, seed=7004)):
        p_dev = torch.from_numpy(np.asarray(p, np.int32)).cuda()
        m, s = _noalloc(dp, p_dev)
        rm, rs = _reference(dp, p_dev)
        assert np.array_equal(m, rm) and np.array_equal(s, rs)


def test_rejects_sizes_beyond_the_scratch(dp):
    import torch
    from paper_2008_01938_gb300 import native
    p_dev = torch.ones(1026, dtype=torch.int32, device="cuda")
    m = torch.empty(1025 * 1025, dtype=torch.int32, device="cuda")
    s = torch.empty(1025 * 1025, dtype=torch.int16, device="cuda")
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    from paper_2008_01938_gb300 import api
    with pytest.raises(native.DpError) as ei:
        api.mcm_solve_noalloc(p_dev, m, s, status)
    assert ei.value.code == native.DP_EINVAL and "1024" in str(ei.value)
    lib = native.load()
    vp = ctypes.c_void_p
    rc = lib.mcm_solve_noalloc(vp(p_dev.data_ptr()), 8, vp(m.data_ptr()), vp(s.data_ptr()), None, None)
    assert rc == native.DP_EINVAL  # the status word is required
    assert int(status.item()) == 0
