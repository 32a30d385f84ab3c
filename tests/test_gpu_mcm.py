"""GPU parity for the MCM table fill: the CUDA path through the C ABI against
the CPU oracle, element by element (m and s), bit-exact."""
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


def _solve(dp, p, cost):
    import torch
    m, s = dp.mcm_solve(torch.from_numpy(np.asarray(p, np.int32)).cuda(), cost=cost)
    dp.sync_status()
    return m.cpu().numpy(), s.cpu().numpy()


def _check(dp, p, cost):
    m, s = _solve(dp, p, cost)
    om, os_ = oracle.mcm(p)
    if cost == "i32":
        assert m.dtype == np.int32
    bad = np.argwhere((m.astype(np.int64) != om) | (s != os_))
    assert bad.size == 0, f"{len(bad)} cells differ, first {bad[:5].tolist()}"


@pytest.mark.parametrize("n", [1, 2, 3, 5, 31, 32, 33, 63, 64, 65, 97, 128, 200, 257, 400])
def test_parity_int32_random(dp, n):
    _check(dp, inputs.mcm_dims(n, 1, 32, seed=1000 + n), "i32")


@pytest.mark.parametrize("n", [1, 7, 32, 70, 161, 300])
def test_parity_int64_random(dp, n):
    _check(dp, inputs.mcm_dims(n, 1, 1000, seed=2000 + n), "i64")


def test_parity_small_config(dp):
    _check(dp, inputs.mcm_small(), "i32")   # 128 matrices, dims U[1,32], seed 0


@pytest.mark.parametrize("cost", ["i32", "i64"])
def test_ties_everywhere(dp, cost):
    # equal dims: every split ties, s must be the smallest k everywhere
    _check(dp, [5] * 151, cost)
    # dims in [1, 2]: heavy ties across segments and tiles
    _check(dp, inputs.mcm_dims(333, 1, 2, seed=7), cost)


@pytest.mark.parametrize("n,hi", [(100, 200), (100, 240), (64, 256), (40, 300)])
def test_large_dims_small_packing_chunks(dp, n, hi):
    # cost bounds close to 2^31 force packing chunks smaller than a tile
    p = inputs.mcm_dims(n, 1, hi, seed=n + hi)
    p[0] = hi
    _check(dp, p, "i32")


def test_overflow_and_invalid_dims_reported(dp):
    import torch
    from paper_2008_01938_gb300.native import DP_EINVAL, DP_EOVERFLOW, DpError
    p = torch.full((301,), 2000, dtype=torch.int32, device="cuda")  # 299 * 2000^3 >= 2^31
    dp.mcm_solve(p, cost="i32")
    with pytest.raises(DpError) as e:
        dp.sync_status()
    assert e.value.code == DP_EOVERFLOW
    q = torch.from_numpy(inputs.mcm_dims(50, 1, 9, seed=3)).cuda()
    q[17] = 0
    dp.mcm_solve(q, cost="i64")
    with pytest.raises(DpError) as e:
        dp.sync_status()
    assert e.value.code == DP_EINVAL
    # the context stays usable after device-reported errors
    _check(dp, inputs.mcm_dims(70, 1, 32, seed=4), "i32")


def test_host_buffer_entry_point(dp):
    p = inputs.mcm_dims(150, 1, 32, seed=9)
    m, s = dp.mcm_solve_host(p, cost="i32")
    om, os_ = oracle.mcm(p)
    assert np.array_equal(m, om.astype(np.int32)) and np.array_equal(s, os_)


def _host_address(dp, x, writable):
    import ctypes
    from paper_2008_01938_gb300 import native
    lib = native.load()
    nbytes = x.numel() * x.element_size() if hasattr(x, "numel") else x.nbytes
    ptr = x.data_ptr() if hasattr(x, "data_ptr") else x.ctypes.data
    return lib.dp_test_host_range_device_address(ctypes.c_void_p(ptr), nbytes, int(writable))


@pytest.mark.parametrize("cost,n", [("i32", 1), ("i32", 33), ("i32", 97), ("i32", 150), ("i64", 70), ("i64", 129)])
def test_host_entry_point_pinned_tables(dp, cost, n):
    """Page-locked m and s: the kernel writes them in place (no copy after the
    solve); the tables match the oracle exactly."""
    import torch
    hi = 32 if cost == "i32" else 1000
    p_np = inputs.mcm_dims(n, 1, hi, seed=40 + n)
    p = torch.from_numpy(p_np).pin_memory()
    tdt = torch.int32 if cost == "i32" else torch.int64
    m = torch.full((n, n), 7, dtype=tdt).pin_memory()
    s = torch.full((n, n), 7, dtype=torch.int16).pin_memory()
    assert _host_address(dp, m, True) and _host_address(dp, s, True) and _host_address(dp, p, False)
    dp.mcm_solve_host(p, cost=cost, m=m, s=s)
    om, os_ = oracle.mcm(p_np)
    assert np.array_equal(m.numpy(), om.astype(m.numpy().dtype)) and np.array_equal(s.numpy(), os_)


def test_host_entry_point_mixed_buffers(dp):
    """Pinned m with pageable s (and pageable dims) goes through the copy path."""
    import torch
    p_np = inputs.mcm_dims(120, 1, 32, seed=12)
    m = torch.zeros((120, 120), dtype=torch.int32).pin_memory()
    s = np.zeros((120, 120), np.int16)
    assert not _host_address(dp, s, True) and not _host_address(dp, p_np, False)
    dp.mcm_solve_host(p_np, cost="i32", m=m, s=s)
    om, os_ = oracle.mcm(p_np)
    assert np.array_equal(m.numpy(), om.astype(np.int32)) and np.array_equal(s, os_)


def test_host_range_outside_allocation(dp):
    """A range that runs past its page-locked allocation is not used in place."""
    import torch
    from paper_2008_01938_gb300 import native
    import ctypes
    x = torch.zeros(1 << 20, dtype=torch.uint8).pin_memory()
    lib = native.load()
    assert lib.dp_test_host_range_device_address(ctypes.c_void_p(x.data_ptr()), 1 << 20, 1)
    assert not lib.dp_test_host_range_device_address(ctypes.c_void_p(x.data_ptr()), 1 << 40, 1)


def test_status_word_argument(dp):
    import torch
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    p = torch.from_numpy(inputs.mcm_dims(90, 1, 32, seed=5)).cuda()
    m, s = dp.mcm_solve(p, cost="i32", status=st)
    dp.sync_status(status=st)
    assert int(st.item()) == 0


def test_bounded_wait_timeout_is_reported(dp):
    """Fault injection on the host: one queue entry is dropped, so the tiles
    that depend on it hit their bounded waits; the kernel returns and reports
    DP_ETIMEOUT instead of hanging, and the context stays usable."""
    import ctypes

    import torch
    from paper_2008_01938_gb300 import native
    lib = native.load()
    n = 200
    p = torch.from_numpy(inputs.mcm_dims(n, 1, 32, seed=11)).cuda()
    m = torch.empty((n, n), dtype=torch.int32, device="cuda")
    s = torch.empty((n, n), dtype=torch.int16, device="cuda")
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = lib.dp_test_mcm_drop_task(ctypes.c_void_p(p.data_ptr()), n, 0, ctypes.c_void_p(m.data_ptr()),
                                   ctypes.c_void_p(s.data_ptr()), ctypes.c_void_p(status.data_ptr()), stream,
                                   3, 2_000_000)
    assert rc == 0
    torch.cuda.synchronize()
    assert int(status.item()) == native.DP_ETIMEOUT
    status.zero_()
    _check(dp, inputs.mcm_dims(120, 1, 32, seed=12), "i32")


def _sha(a):
    return hashlib.sha256(np.ascontiguousarray(a).tobytes()).hexdigest()


def _bellman_ok(p, m, i, j):
    """The recurrence holds at (i, j) on the GPU table itself."""
    if i == j:
        return m[i, j] == 0
    k = np.arange(i, j)
    cand = m[i, i:j].astype(np.int64) + m[i + 1:j + 1, j].astype(np.int64) + \
        int(p[i]) * p[k + 1].astype(np.int64) * int(p[j + 1])
    return int(cand.min()) == int(m[i, j])


def test_full_size_4096(dp):
    """The 4096-matrix chain (dims U[1,32], seed 1) as the benchmark runs it:
    whole-table SHA-256 against the oracle's (written by
    tests/golden/make_golden.py), oracle cells, and the recurrence on samples."""
    if not os.path.exists(GOLDEN):
        pytest.skip("golden file not generated")
    g = json.load(open(GOLDEN))["mcm_n4096_seed1"]
    p = inputs.mcm_big()
    m, s = _solve(dp, p, "i32")
    for i, j, mv, sv in g["cells"]:
        assert (int(m[i, j]), int(s[i, j])) == (mv, sv)
    assert _sha(m.astype("<i4")) == g["m_sha256"]
    assert _sha(s.astype("<i2")) == g["s_sha256"]
    rng = np.random.default_rng(0)
    for _ in range(200):
        i, j = sorted(rng.integers(0, 4096, 2).tolist())
        assert _bellman_ok(p, m, i, j)
    # exact oracle on sub-chains for short spans
    for _ in range(5):
        i = int(rng.integers(0, 3500))
        j = i + int(rng.integers(1, 400))
        assert oracle.mcm_cell(p, i, j) == (int(m[i, j]), int(s[i, j]))


# ---------------------------------------------------------------------------
# batched plans
# ---------------------------------------------------------------------------

def _batch_tensors(b, cost):
    import torch
    dt = torch.int64 if cost == "i64" else torch.int32
    p_all = torch.from_numpy(b.p_all).cuda()
    p_off = torch.from_numpy(b.p_off[:-1].copy()).cuda()
    tab_off = torch.from_numpy(b.tab_off[:-1].copy()).cuda()
    m_all = torch.empty(int(b.tab_off[-1]), dtype=dt, device="cuda")
    s_all = torch.empty(int(b.tab_off[-1]), dtype=torch.int16, device="cuda")
    return p_all, p_off, tab_off, m_all, s_all


@pytest.mark.parametrize("cost", ["i64", "i32"])
def test_batched_parity(dp, cost):
    hi = 1000 if cost == "i64" else 32
    b = inputs.mcm_batch(count=150, nlo=1, nhi=300, dlo=1, dhi=hi, seed=21)
    plan = dp.McmPlan(b.ns, cost=cost)
    t = _batch_tensors(b, cost)
    plan.solve(*t)
    dp.sync_status()
    m_all, s_all = t[3].cpu().numpy(), t[4].cpu().numpy()
    for i in range(b.ns.size):
        n = int(b.ns[i])
        o = int(b.tab_off[i])
        om, os_ = oracle.mcm(b.dims(i))
        assert np.array_equal(m_all[o:o + n * n].reshape(n, n).astype(np.int64), om), i
        assert np.array_equal(s_all[o:o + n * n].reshape(n, n), os_), i
    plan.destroy()


@pytest.mark.parametrize("cost", ["i64", "i32"])
def test_batched_autotune(dp, cost):
    """The autotuner picks one of its candidate configurations, leaves the
    tables solved, and later solves under the chosen configuration (also
    captured in a graph) agree with the oracle."""
    import torch
    hi = 1000 if cost == "i64" else 32
    b = inputs.mcm_batch(count=80, nlo=8, nhi=400, dlo=1, dhi=hi, seed=23)
    plan = dp.McmPlan(b.ns, cost=cost)
    assert plan.config() == (8, 0)                    # defaults before tuning
    t = _batch_tensors(b, cost)
    lpp, bps = plan.autotune(*t)
    dp.sync_status()
    assert lpp in (4, 8, 16) and bps >= 1
    assert plan.config() == (lpp, bps)

    def check_all():
        m_all, s_all = t[3].cpu().numpy(), t[4].cpu().numpy()
        for i in range(b.ns.size):
            n, o = int(b.ns[i]), int(b.tab_off[i])
            om, os_ = oracle.mcm(b.dims(i))
            assert np.array_equal(m_all[o:o + n * n].reshape(n, n).astype(np.int64), om), i
            assert np.array_equal(s_all[o:o + n * n].reshape(n, n), os_), i

    check_all()                                       # left solved by the tuner
    t[3].fill_(-1)
    t[4].fill_(-1)
    s = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        plan.solve(*t, stream=s)
    g.replay()
    torch.cuda.synchronize()
    dp.sync_status()
    check_all()
    plan.destroy()


def test_batched_graph_capture_replay(dp):
    import torch
    b = inputs.mcm_batch(count=60, nlo=8, nhi=200, seed=22)
    plan = dp.McmPlan(b.ns, cost="i64")
    t = _batch_tensors(b, "i64")
    s = torch.cuda.Stream()
    plan.solve(*t, stream=s)       # warm-up outside capture (first-use setup)
    s.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        plan.solve(*t, stream=s)
    for _ in range(2):
        t[3].fill_(-1)
        g.replay()
        torch.cuda.synchronize()
        dp.sync_status()
        m_all = t[3].cpu().numpy()
        for i in range(0, b.ns.size, 7):
            n, o = int(b.ns[i]), int(b.tab_off[i])
            om, _ = oracle.mcm(b.dims(i))
            assert np.array_equal(m_all[o:o + n * n].reshape(n, n), om)
    plan.destroy()


def test_batched_full_config(dp):
    """10,000 chains, n log-uniform in [8, 512], dims U[1,1000], int64 costs:
    concatenated tables against the oracle's digests."""
    if not os.path.exists(GOLDEN) or "mcm_batch10000_seed3" not in json.load(open(GOLDEN)):
        pytest.skip("golden batch digest not generated")
    g = json.load(open(GOLDEN))["mcm_batch10000_seed3"]
    b = inputs.mcm_batch()
    plan = dp.McmPlan(b.ns, cost="i64")
    t = _batch_tensors(b, "i64")
    plan.solve(*t)
    dp.sync_status()
    m_all, s_all = t[3].cpu().numpy(), t[4].cpu().numpy()
    finals = [int(m_all[int(b.tab_off[i]) + int(b.ns[i]) - 1]) for i in range(100)]
    assert finals == g["final_costs_first100"]
    assert _sha(m_all.astype("<i8")) == g["m_sha256_concat"]
    assert _sha(s_all.astype("<i2")) == g["s_sha256_concat"]
    plan.destroy()


def test_int32_rate_probe(dp):
    """The roofline's measured denominators: every rate positive and below
    the issue limit of the SM (4 warp instructions per clock, 128 lanes), the
    SM count that of the device, the int64 bulk loop only with room for it,
    and DP_EINVAL for a buffer of fewer than 9 values."""
    import ctypes
    import torch
    from paper_2008_01938_gb300 import native
    lib = native.load()
    st = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    out = (ctypes.c_double * 10)(*([-1.0] * 10))
    native.check(lib.dp_measure_int32_rates(out, 10, st))
    assert int(out[6]) == torch.cuda.get_device_properties(0).multi_processor_count
    for i in [0, 1, 2, 3, 4]:
        assert 0 < out[i] <= 130, (i, out[i])
    assert 0 < out[5] <= 64 and 0 < out[9] < out[5], (out[5], out[9])
    assert out[7] > 0 and out[8] > 0
    nine = (ctypes.c_double * 10)(*([-1.0] * 10))
    native.check(lib.dp_measure_int32_rates(nine, 9, st))
    assert nine[9] == -1.0 and nine[5] > 0
    assert lib.dp_measure_int32_rates(nine, 8, st) == 1


@pytest.mark.parametrize("n, hi", [(129, 101), (97, 111), (129, 102), (65, 160)])
def test_diagonal_tile_keys_at_the_packing_limit(dp, n, hi):
    """The diagonal tiles keep 32-bit (value << 5) + split keys when the
    cost bound (n - 1) max(p)^3 is below 2^27 (packing shift 5), and 64-bit
    keys otherwise. Chains just below the limit (127 * 101^3 and 96 * 111^3
    below 2^27, keys near 2^32) and just above it (127 * 102^3, 64 * 160^3),
    with dims at the maximum in every tile, against the oracle."""
    bound = (n - 1) * hi ** 3
    p = inputs.mcm_dims(n, hi - 3, hi, seed=7 * n + hi)
    p[::5] = hi
    assert (bound < (1 << 27)) == ((n, hi) in [(129, 101), (97, 111)])
    _check(dp, p, "i32")
