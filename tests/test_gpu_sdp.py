"""GPU parity for the simplified DP (Definition 1): the CUDA path through the
C ABI against the CPU oracle, bit-exact, plus full-size closed forms and
invariants."""
import hashlib
import json
import os

import numpy as np
import pytest

import oracle
from paper_2008_01938_gb300 import inputs

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "fullsize.json")
M32 = (1 << 32) - 1


@pytest.fixture(scope="module")
def dp():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2008_01938_gb300 as dp
    return dp


def _gpu(dp, preset, n, offsets, op):
    import torch
    st = np.zeros(max(n, int(offsets[0])), dtype=np.uint32)
    st[:offsets[0]] = np.asarray(preset, dtype=np.uint32)[:offsets[0]]
    t = torch.from_numpy(st.view(np.int32)).cuda()
    dp.sdp_solve(t, offsets, op=op, n=n)
    dp.sync_status()
    return t.cpu().numpy().view(np.uint32)[:n]


CASES = [
    # (n, k, amin, amax, seed): a_k >= 1024 (1024-wide steps), a_k small,
    # single offset, k > 32 (offsets in shared memory), large a_1 (no ring)
    (200000, 32, 1024, 8192, 1),
    (50000, 8, 40, 700, 2),
    (30000, 3, 1, 9, 3),
    (12345, 1, 5, 5, 4),
    (40000, 48, 100, 3000, 5),
    (120000, 6, 20000, 40000, 6),
    (3000, 5, 2000, 2999, 7),
]


@pytest.mark.parametrize("case", CASES)
@pytest.mark.parametrize("op", ["min", "add"])
def test_parity_random(dp, case, op):
    n, k, amin, amax, seed = case
    inst = inputs.sdp_random(n=n, k=k, amin=amin, amax=amax, seed=seed)
    got = _gpu(dp, inst.preset, n, inst.offsets, op)
    ref = oracle.sdp(inst.preset, n, inst.offsets, op)
    bad = np.flatnonzero(got != ref)
    assert bad.size == 0, f"{bad.size} cells differ, first {bad[:5].tolist()}"


def test_consecutive_offsets_worst_case(dp):
    # Section III-A, Fig. 4: a run of consecutive offsets makes the paper's
    # pipeline threads collide; here it is just another offset set
    offs = [40, 39, 38, 37, 36, 35, 10, 9, 8]
    pre = inputs.SplitMix64(5).u32(40)
    for op in ("min", "add"):
        assert np.array_equal(_gpu(dp, pre, 100000, offs, op), oracle.sdp(pre, 100000, offs, op))


def test_short_tables(dp):
    for n in (0, 1, 5, 8, 9):
        got = _gpu(dp, [3, 1, 4, 1, 5, 9, 2, 6], n, [8, 3], "add")
        assert np.array_equal(got, oracle.sdp([3, 1, 4, 1, 5, 9, 2, 6], n, [8, 3], "add"))


# (x) = + by chunks from jumped windows (the jump of Fiduccia's method for
# linear recurrences), forced to a given number of chunks through the test
# hook: (n, offsets, chunks).  Offsets are a list, or (k, amin, amax, seed)
# for inputs.sdp_random.
JUMP_CASES = [
    (100000, [2, 1], 2),
    (100003, [2, 1], 152),                  # as many chunks as SMs, ragged tail
    (50000, [5], 7),                        # one offset: a periodic table
    (70000, (8, 40, 700, 2), 13),
    (20000, [9, 8, 7, 6, 5, 4, 3, 2, 1], 9),  # consecutive offsets down to a_k = 1
    (300000, (32, 1024, 8192, 1), 5),       # the 2^26 workload's offsets: 3 squarings, a tree of 3 products
    (962, [40, 33, 17, 2], 12),             # last chunk (38 cells) shorter than the window
    (165, [9, 4, 3], 5),                    # last chunk of 5 cells
    (400000, (16, 64, 4096, 9), 40),
    (1000000, (32, 1024, 8192, 3), 40),     # a_1 = 8192: windows by the transposed Karatsuba step
    (400000, (32, 1024, 8192, 4), 20),      # the same, chunks of the least length (2 a_1)
]


def _jump(dp, preset, n, offsets, chunks):
    import ctypes
    import torch
    from paper_2008_01938_gb300 import native
    lib = native.load()
    a = np.ascontiguousarray(np.asarray(offsets, dtype=np.int32))
    st = np.zeros(n, dtype=np.uint32)
    st[:a[0]] = np.asarray(preset, dtype=np.uint32)[:a[0]]
    t = torch.from_numpy(st.view(np.int32)).cuda()
    native.check(lib.dp_test_sdp_jump(ctypes.c_void_p(t.data_ptr()), n, ctypes.c_void_p(a.ctypes.data),
                                      int(a.size), int(chunks), None, None))
    dp.sync_status()
    return t.cpu().numpy().view(np.uint32)


@pytest.mark.parametrize("case", JUMP_CASES)
def test_add_by_jumped_chunks(dp, case):
    n, offs, chunks = case
    if isinstance(offs, tuple):
        k, amin, amax, seed = offs
        inst = inputs.sdp_random(n=n, k=k, amin=amin, amax=amax, seed=seed)
        offs, pre = inst.offsets, inst.preset
    else:
        pre = inputs.SplitMix64(n + chunks).u32(offs[0])
    got = _jump(dp, pre, n, offs, chunks)
    ref = oracle.sdp(pre, n, offs, "add")
    bad = np.flatnonzero(got != ref)
    assert bad.size == 0, f"{bad.size} cells differ, first {bad[:5].tolist()}"


# (x) = min by chunks whose windows come from Boolean products modulo the
# characteristic polynomial (Kitamasa's method over the Boolean semiring),
# forced to a given number of chunks: (n, offsets, chunks, preset kind).
# The path needs a_k >= 32 and a_1 <= 8192.  "planted": a large constant
# with a few small values planted, so that windows are not simply the
# preset's minimum.
MIN_JUMP_CASES = [
    (100000, [64, 33], 2, "random"),
    (100003, [64, 33], 152, "planted"),              # as many chunks as SMs, ragged tail
    (50000, [40], 7, "random"),                       # one offset: a periodic table
    (70000, (8, 40, 700, 2), 13, "planted"),
    (40000, [40, 39, 38, 37, 36, 35, 34, 33, 32], 9, "planted"),  # consecutive offsets, a_k = 32
    (300000, (32, 1024, 8192, 1), 5, "planted"),     # the 2^26 workload's offsets
    (962, [40, 33], 12, "random"),                    # last chunk shorter than the window
    (400000, (16, 64, 4096, 9), 40, "planted"),      # the serving mix's offset recipe
    (200000, [1024, 768, 512], 20, "planted"),       # common factor 256: C never fills, many runs
    (120000, [300, 144, 96], 30, "planted"),          # common factor 12, a_1 not a multiple of 32
    (500000, [8192, 4096 + 2048 + 32], 20, "planted"),  # common factor 32: 256 runs per set
]


def _min_preset(n, a1, kind, seed):
    rng = inputs.SplitMix64(seed)
    if kind == "random":
        return rng.u32(a1)
    pre = (rng.u32(a1) | np.uint32(0x80000000))
    pos = rng.randint(0, a1 - 1, 7)
    pre[pos] = rng.u32(7) >> np.uint32(4)
    return pre


def _min_jump(dp, preset, n, offsets, chunks):
    import ctypes
    import torch
    from paper_2008_01938_gb300 import native
    lib = native.load()
    a = np.ascontiguousarray(np.asarray(offsets, dtype=np.int32))
    st = np.zeros(n, dtype=np.uint32)
    st[:a[0]] = np.asarray(preset, dtype=np.uint32)[:a[0]]
    t = torch.from_numpy(st.view(np.int32)).cuda()
    native.check(lib.dp_test_sdp_min_jump(ctypes.c_void_p(t.data_ptr()), n, ctypes.c_void_p(a.ctypes.data),
                                          int(a.size), int(chunks), None, None))
    dp.sync_status()
    return t.cpu().numpy().view(np.uint32)


@pytest.mark.parametrize("case", MIN_JUMP_CASES)
def test_min_by_jumped_chunks(dp, case):
    n, offs, chunks, kind = case
    if isinstance(offs, tuple):
        k, amin, amax, seed = offs
        offs = inputs.sdp_random(n=n, k=k, amin=amin, amax=amax, seed=seed).offsets
    pre = _min_preset(n, int(offs[0]), kind, n + chunks)
    got = _min_jump(dp, pre, n, offs, chunks)
    ref = oracle.sdp(pre, n, offs, "min")
    bad = np.flatnonzero(got != ref)
    assert bad.size == 0, f"{bad.size} cells differ, first {bad[:5].tolist()}"


def test_min_jump_path_choice_and_refusal(dp):
    """sdp_solve takes the min jump path for the 2^26-cell workload and not
    for a short table or a_k < 32; a forced jump outside its range is
    refused on the host."""
    import ctypes
    from paper_2008_01938_gb300 import native
    from paper_2008_01938_gb300.native import DpError
    lib = native.load()
    big = inputs.sdp_instance_big()
    a = np.ascontiguousarray(big.offsets.astype(np.int32))
    assert lib.dp_test_sdp_min_jump_chunks(big.n, ctypes.c_void_p(a.ctypes.data), int(a.size)) >= 2
    assert lib.dp_test_sdp_min_jump_chunks(30000, ctypes.c_void_p(a.ctypes.data), int(a.size)) == 0
    small_ak = np.ascontiguousarray(np.array([64, 31], dtype=np.int32))
    assert lib.dp_test_sdp_min_jump_chunks(1 << 22, ctypes.c_void_p(small_ak.ctypes.data), 2) == 0
    with pytest.raises(DpError):
        _min_jump(dp, big.preset, 40000, big.offsets, 3)     # chunks of 13334 < 2 a_1 cells
    with pytest.raises(DpError):
        _min_jump(dp, [1] * 64, 100000, [64, 31], 4)         # a_k < 32


def test_min_planted_2p24(dp):
    """2^24 cells with the 2^26 workload's offsets and a planted preset (large
    values with seven small ones), through sdp_solve (the min jump path):
    every cell against the oracle.  With a uniform preset the table settles
    at the preset's minimum early; planted minima keep the windows varied."""
    big = inputs.sdp_instance_big(n=1 << 24)
    pre = _min_preset(big.n, int(big.offsets[0]), "planted", 24)
    got = _gpu(dp, pre, big.n, big.offsets, "min")
    ref = oracle.sdp(pre, big.n, big.offsets, "min")
    bad = np.flatnonzero(got != ref)
    assert bad.size == 0, f"{bad.size} cells differ, first {bad[:5].tolist()}"


def test_host_entry_point_pinned_jump(dp):
    """(+) on a page-locked host table long enough for the jump path: its
    kernels read and write the table in host memory, in place."""
    import ctypes
    import torch
    from paper_2008_01938_gb300 import native
    big = inputs.sdp_instance_big(n=1 << 22)
    a = np.ascontiguousarray(big.offsets.astype(np.int32))
    lib = native.load()
    assert lib.dp_test_sdp_jump_chunks(big.n, ctypes.c_void_p(a.ctypes.data), int(a.size)) >= 2
    st = torch.zeros(big.n, dtype=torch.int32).pin_memory()
    st.numpy().view(np.uint32)[:a[0]] = big.preset
    dp.sdp_solve_host(st, big.offsets, op="add")
    ref = oracle.sdp(big.preset, big.n, big.offsets, "add")
    bad = np.flatnonzero(st.numpy().view(np.uint32) != ref)
    assert bad.size == 0, f"{bad.size} cells differ, first {bad[:5].tolist()}"


def test_jump_path_choice_and_refusal(dp):
    """sdp_solve takes the jump path for the 2^26-cell workload and not for a
    short table; chunks too short for two windows are refused on the host."""
    import ctypes
    from paper_2008_01938_gb300 import native
    from paper_2008_01938_gb300.native import DpError
    lib = native.load()
    big = inputs.sdp_instance_big()
    a = np.ascontiguousarray(big.offsets.astype(np.int32))
    assert lib.dp_test_sdp_jump_chunks(big.n, ctypes.c_void_p(a.ctypes.data), int(a.size)) >= 2
    assert lib.dp_test_sdp_jump_chunks(30000, ctypes.c_void_p(a.ctypes.data), int(a.size)) == 0
    with pytest.raises(DpError):
        _jump(dp, big.preset, 40000, big.offsets, 3)   # chunks of 13334 < 2 a_1 cells


def fib_pair(i):
    if i == 0:
        return 0, 1
    a, b = fib_pair(i >> 1)
    c = (a * ((2 * b - a) & M32)) & M32
    d = (a * a + b * b) & M32
    return (d, (c + d) & M32) if i & 1 else (c, d)


def test_fibonacci_full_length(dp):
    n = 1 << 22
    got = _gpu(dp, [0, 1], n, [2, 1], "add")
    for i in [0, 1, 2, 3, 1000, 123456, n // 2, n - 2, n - 1]:
        assert int(got[i]) == fib_pair(i)[0]
    got1 = _gpu(dp, [1, 1], 4096, [2, 1], "add")   # the paper's preset: F(i+1)
    assert all(int(got1[i]) == fib_pair(i + 1)[0] for i in (0, 1, 50, 4095))


def _sha(a):
    return hashlib.sha256(np.ascontiguousarray(a).tobytes()).hexdigest()


@pytest.mark.parametrize("op", ["min", "add"])
def test_full_size_2p26(dp, op):
    """2^26 cells, 32 offsets in [1024, 8192], uniform uint32 preset (seed 2):
    whole-table SHA-256 against the oracle's, plus sampled values."""
    if not os.path.exists(GOLDEN):
        pytest.skip("golden file not generated")
    g = json.load(open(GOLDEN))[f"sdp_n2p26_seed2_{op}"]
    big = inputs.sdp_instance_big()
    got = _gpu(dp, big.preset, big.n, big.offsets, op)
    for i, v in g["samples"]:
        assert int(got[i]) == v
    assert _sha(got.astype("<u4")) == g["st_sha256"]


def test_full_size_invariants(dp):
    """Properties that hold at any size, checked on 2^24-cell GPU tables:
    (+) is linear mod 2^32; (min) distributes over elementwise min, never
    leaves the preset's values, and commutes with adding a constant."""
    big = inputs.sdp_instance_big(n=1 << 24)
    x = big.preset
    y = inputs.SplitMix64(99).u32(x.size)
    n, a = big.n, big.offsets
    sx, sy = _gpu(dp, x, n, a, "add"), _gpu(dp, y, n, a, "add")
    assert np.array_equal(_gpu(dp, (x + y).astype(np.uint32), n, a, "add"), (sx + sy).astype(np.uint32))
    xs, ys = x >> np.uint32(1), y >> np.uint32(1)
    mx, my = _gpu(dp, xs, n, a, "min"), _gpu(dp, ys, n, a, "min")
    assert np.array_equal(_gpu(dp, np.minimum(xs, ys), n, a, "min"), np.minimum(mx, my))
    assert np.isin(mx, xs).all()
    assert np.array_equal(_gpu(dp, xs + np.uint32(7), n, a, "min"), mx + np.uint32(7))


def test_host_entry_point(dp):
    inst = inputs.sdp_random(n=70000, k=10, amin=300, amax=2000, seed=12)
    st = np.zeros(inst.n, dtype=np.uint32)
    st[:inst.offsets[0]] = inst.preset
    dp.sdp_solve_host(st, inst.offsets, op="min")
    assert np.array_equal(st, oracle.sdp(inst.preset, inst.n, inst.offsets, "min"))


@pytest.mark.parametrize("op,amax", [("min", 2000), ("add", 2000), ("min", 40000)])
def test_host_entry_point_pinned(dp, op, amax):
    """Page-locked table: solved in place when the window fits the on-chip
    ring (a_1 <= 2000 here), staged through device memory when it does not
    (a_1 near 40000); either way identical to the oracle."""
    import ctypes
    import torch
    from paper_2008_01938_gb300 import native
    inst = inputs.sdp_random(n=90001, k=12, amin=300, amax=amax, seed=13 + amax)
    st = torch.zeros(inst.n, dtype=torch.int32).pin_memory()
    st.numpy().view(np.uint32)[:inst.offsets[0]] = inst.preset
    lib = native.load()
    assert lib.dp_test_host_range_device_address(ctypes.c_void_p(st.data_ptr()), inst.n * 4, 1)
    dp.sdp_solve_host(st, inst.offsets, op=op)
    assert np.array_equal(st.numpy().view(np.uint32), oracle.sdp(inst.preset, inst.n, inst.offsets, op))


@pytest.mark.parametrize("op", ["min", "add"])
def test_batched_parity(dp, op):
    import torch
    insts = [inputs.sdp_random(n=int(n), k=int(k), amin=16, amax=amax, seed=40 + i)
             for i, (n, k, amax) in enumerate([(5000, 4, 100), (70000, 16, 4096), (1, 3, 50), (33333, 1, 64),
                                               (200000, 20, 2000), (9000, 40, 900)])]
    ns = [x.n for x in insts]
    offs = [x.offsets for x in insts]
    st_off = np.zeros(len(insts), dtype=np.int64)
    tot = 0
    for i, x in enumerate(insts):
        st_off[i] = tot
        tot += max(x.n, int(x.offsets[0]))
    host = np.zeros(tot, dtype=np.uint32)
    for i, x in enumerate(insts):
        host[st_off[i]:st_off[i] + x.offsets[0]] = x.preset
    t = torch.from_numpy(host.view(np.int32)).cuda()
    plan = dp.SdpPlan(ns, offs, op=op)
    plan.solve(t, torch.from_numpy(st_off).cuda())
    dp.sync_status()
    got = t.cpu().numpy().view(np.uint32)
    for i, x in enumerate(insts):
        ref = oracle.sdp(x.preset, x.n, x.offsets, op)
        assert np.array_equal(got[st_off[i]:st_off[i] + x.n], ref), i
    plan.destroy()
