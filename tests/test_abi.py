"""The native library builds, loads without a GPU, and exports every function
declared in include/dpgpu.h (no compute calls here)."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def header_functions():
    src = open(os.path.join(ROOT, "include", "dpgpu.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\*?\s*([a-z_][a-z0-9_]*)\s*\(", src, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_2008_01938_gb300 import build, native
    build.build()
    return ctypes.CDLL(native.LIB_PATH)


def test_header_lists_the_boundary():
    names = header_functions()
    for expected in ["mcm_solve", "mcm_solve_batched", "mcm_plan_create", "sdp_solve", "sdp_solve_batched",
                     "serve_submit", "serve_poll", "dp_sync_status", "dp_last_error"]:
        assert expected in names


def test_library_exports_every_header_symbol(lib):
    missing = [n for n in header_functions() if not hasattr(lib, n)]
    assert not missing, f"symbols declared in dpgpu.h but not exported: {missing}"


def test_binding_symbol_list_matches_header():
    from paper_2008_01938_gb300 import native
    assert sorted(native.HEADER_SYMBOLS) == header_functions()


def test_version_and_error_text_without_gpu(lib):
    lib.dp_version.restype = ctypes.c_char_p
    lib.dp_last_error.restype = ctypes.c_char_p
    assert b"sm_103a" in lib.dp_version()
    assert isinstance(lib.dp_last_error(), bytes)


def test_host_validation_without_gpu(lib):
    # offsets that are not strictly decreasing are rejected on the host,
    # before any CUDA call
    lib.sdp_solve.restype = ctypes.c_int
    a = (ctypes.c_int32 * 3)(5, 5, 1)
    rc = lib.sdp_solve(ctypes.c_void_p(1), ctypes.c_int64(100), a, 3, 0, None, None)
    assert rc == 1  # DP_EINVAL
    lib.dp_last_error.restype = ctypes.c_char_p
    assert b"strictly decreasing" in lib.dp_last_error()
    lib.mcm_solve.restype = ctypes.c_int
    assert lib.mcm_solve(ctypes.c_void_p(1), 0, 0, ctypes.c_void_p(1), ctypes.c_void_p(1), None, None) == 1
    # the interval DP is built for int32 costs only: int64 is refused on the host
    lib.interval_dp_solve.restype = ctypes.c_int
    one = ctypes.c_void_p(1)
    assert lib.interval_dp_solve(one, one, 40, 1, one, one, None, None) == 1
    assert b"DP_COST_I32" in lib.dp_last_error()
    assert lib.interval_dp_solve(one, None, 40, 0, one, one, None, None) == 1


def test_host_wrappers_check_buffers_without_gpu(lib):
    """The host-buffer wrappers refuse tables of the wrong size, dtype or
    layout before any library call: a page-locked table is written by the
    kernel in place, so a short one must never reach it."""
    import numpy as np
    import torch
    from paper_2008_01938_gb300 import api
    p = np.arange(1, 7, dtype=np.int32)  # 5 matrices
    with pytest.raises(ValueError, match="m must be"):
        api.mcm_solve_host(p, m=np.empty((4, 4), np.int32))
    with pytest.raises(ValueError, match="m must be"):
        api.mcm_solve_host(p, cost="i64", m=np.empty((5, 5), np.int32))
    with pytest.raises(ValueError, match="s must be"):
        api.mcm_solve_host(p, m=torch.empty((5, 5), dtype=torch.int32), s=torch.empty((5, 5), dtype=torch.int32))
    with pytest.raises(ValueError, match="m must be"):
        api.mcm_solve_host(p, m=torch.empty((5, 10), dtype=torch.int32)[:, ::2])
    with pytest.raises(TypeError):
        api.sdp_solve_host(np.zeros(100, np.int32), [3, 1])
    with pytest.raises(TypeError):
        api.sdp_solve_host(torch.zeros(100, dtype=torch.float32), [3, 1])


def _jump_plan(lib, n, offs, sms):
    import numpy as np
    lib.dp_test_sdp_jump_plan.restype = ctypes.c_int32
    lib.dp_test_sdp_jump_plan.argtypes = [ctypes.c_int64, ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32,
                                          ctypes.c_void_p]
    a = np.ascontiguousarray(np.asarray(offs, dtype=np.int32))
    out = np.zeros(8, dtype=np.int64)
    rc = lib.dp_test_sdp_jump_plan(n, ctypes.c_void_p(a.ctypes.data), int(a.size), sms,
                                   ctypes.c_void_p(out.ctypes.data))
    return rc, dict(zip(["P", "L", "L0", "s", "Gm", "P2", "P1e", "chunks"], (int(x) for x in out)))


def test_jump_plan_without_gpu(lib):
    """The plan of the (+) jump path (host arithmetic only): chunks of at
    least two windows that cover the table, x^L0 within the reach of the
    impulse response, and major windows that cover every chunk."""
    from paper_2008_01938_gb300 import inputs
    big = inputs.sdp_instance_big()
    for n, offs, sms in [(big.n, big.offsets, 152), (1 << 22, [2, 1], 152), (1 << 24, big.offsets, 152),
                         (10 ** 7, [900, 700, 64], 40)]:
        rc, p = _jump_plan(lib, n, offs, sms)
        A = int(offs[0])
        assert rc >= 2 and p["chunks"] == rc, (n, rc, p)
        assert 2 <= p["P"] <= sms and p["L"] >= 2 * A
        assert (p["P"] - 1) * p["L"] < n <= p["P"] * p["L"]
        assert p["L"] == p["L0"] << p["s"] and 1 <= p["L0"] <= p["Gm"] and p["Gm"] >= A - 1
        assert p["P1e"] == -(-n // (p["P2"] * p["L"])) and p["P1e"] * p["P2"] >= p["P"]
    # a short table keeps the step-by-step path; bad offsets are refused
    assert _jump_plan(lib, 30000, big.offsets, 152)[0] == 0
    assert _jump_plan(lib, 1 << 26, [5, 5, 1], 152)[0] == -1


def test_min_jump_plan_without_gpu(lib):
    """The plan of the (min) jump path (host arithmetic only): chunks of at
    least two windows that cover the table, L = L0 2^s with C_L0 = {L0} (so
    L0 < a_1); tables with a_k < 32 or a_1 > 8192 keep the step-by-step
    path."""
    import ctypes
    from paper_2008_01938_gb300 import inputs
    big = inputs.sdp_instance_big()

    def plan(n, offs, sms):
        a = np.ascontiguousarray(np.asarray(offs, dtype=np.int32))
        out = np.zeros(5, dtype=np.int64)
        rc = lib.dp_test_sdp_min_jump_plan(n, ctypes.c_void_p(a.ctypes.data), int(a.size), sms,
                                           ctypes.c_void_p(out.ctypes.data))
        return rc, dict(zip(["P", "L", "L0", "s", "chunks"], out.tolist()))

    for n, offs, sms in [(big.n, big.offsets, 152), (1 << 24, [64, 33], 152), (10 ** 7, [900, 700, 64], 40)]:
        rc, p = plan(n, offs, sms)
        A = int(offs[0])
        assert rc >= 2 and p["chunks"] == rc, (n, rc, p)
        assert 2 <= p["P"] <= sms and p["L"] >= 2 * A
        assert (p["P"] - 1) * p["L"] < n <= p["P"] * p["L"]
        assert p["L"] == p["L0"] << p["s"] and 1 <= p["L0"] < A
    assert plan(30000, big.offsets, 152)[0] == 0          # too short
    assert plan(1 << 24, [64, 31], 152)[0] == 0            # a_k < 32
    assert plan(1 << 26, [9000, 4000], 152)[0] == 0       # a_1 > 8192
    assert plan(1 << 26, [5, 5, 1], 152)[0] == -1         # not strictly decreasing


def test_missing_library_fails_loudly(tmp_path, monkeypatch):
    from paper_2008_01938_gb300 import native
    monkeypatch.setattr(native, "_lib", None)
    with pytest.raises(RuntimeError, match="missing"):
        native.load(str(tmp_path / "nope.so"))


def test_mcm_queue_orders_every_dependency_first(lib):
    """The MCM work queue (host only): every tile has one finisher; its bulk
    parts and the finisher cover the external levels (D+1)/2 .. D-1 exactly
    once; and every task comes after the finishers of all tiles it reads and
    a finisher after its own parts. Blocks pop tasks in queue order and wait
    only for what they read, so this order is what keeps the persistent
    kernel free of deadlock at any number of resident blocks (Section IV-B's
    diagonal order at tile granularity, with bulk parts deferred towards the
    finisher that needs them)."""
    import ctypes
    T = 32
    for ns, i64 in [([4096], 0), ([33, 70, 161, 300, 1000, 2], 0), ([33, 70, 161, 300, 1000, 2], 1), ([512, 9], 1)]:
        arr = np.asarray(ns, dtype=np.int32)
        nt_total = lib.dp_test_mcm_queue(ctypes.c_void_p(arr.ctypes.data), len(ns), i64, None, 0)
        assert nt_total > 0
        out = np.zeros(6 * nt_total, dtype=np.int32)
        assert lib.dp_test_mcm_queue(ctypes.c_void_p(arr.ctypes.data), len(ns), i64,
                                     ctypes.c_void_p(out.ctypes.data), nt_total) == nt_total
        q = out.reshape(-1, 6).tolist()
        fin_pos, parts = {}, {}
        for x, (c, I, J, kind, lo, hi) in enumerate(q):
            if kind == 0:
                assert (c, I, J) not in fin_pos
                fin_pos[(c, I, J)] = x
            else:
                parts.setdefault((c, I, J), []).append((x, lo, hi))
        for c, n in enumerate(ns):
            nt = (n + T - 1) // T
            assert sum(1 for key in fin_pos if key[0] == c) == nt * (nt + 1) // 2
        for x, (c, I, J, kind, lo, hi) in enumerate(q):
            D = J - I
            for r in range(lo, hi + 1):
                for K in {I + r, J - r}:
                    if I < K < J:
                        for tile in [(c, I, K), (c, K, J), (c, K + 1, J)]:
                            assert fin_pos[tile] < x, (ns, i64, q[x], tile)
            if kind == 0:
                if D >= 1:
                    for tile in [(c, I, I), (c, J, J), (c, I + 1, J)]:
                        assert fin_pos[tile] < x, (ns, i64, q[x], tile)
                levels = list(range(lo, hi + 1)) if D >= 2 else []
                for (y, plo, phi) in parts.get((c, I, J), []):
                    assert y < x
                    levels += list(range(plo, phi + 1))
                want = list(range((D + 1) // 2, D)) if D >= 2 else []
                assert sorted(levels) == want, (ns, i64, q[x], sorted(levels))
