"""CPU oracle for the MCM table fill and the simplified DP (S-DP) recurrence.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  The library in
``paper_2008_01938_gb300`` never does; it shares no code with this package.

The arithmetic lives in ``dp_oracle.c`` (plain C, single thread, int64 / uint32,
no blocking or reordering); this module compiles it with gcc and calls it
through ctypes.

  mcm(p)                   -> (m int64[n, n], s int16[n, n])   paper Section IV-A
                              (problem from Cormen et al., cited there)
  mcm_cell(p, i, j)        -> (m[i][j], s[i][j]) by solving the sub-chain
                              A_i..A_j alone (the sub-problem is self-contained)
  interval(p, w)           -> (m int64[n, n], s int16[n, n])   Eq. (2) with
                              f(l, r) = l + r + p[i] p[k+1] p[j+1] + w[i][j]
  sdp(preset, n, a, op)    -> uint32[n]                        Definition 1, Fig. 1
  diag_major_index(n,r,c)  -> the 1-based position of CLRS cell (r, c) in the
                              paper's linearised table (Section IV-B)

Every function is pinned by tests against facts the paper or mathematics fix
(textbook example, brute force, closed forms, Fibonacci) -- see tests/.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "dp_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile dp_oracle.c into liboracle.so next to it (gcc, -O2, no
    architecture-specific flags so it behaves the same on x86 and Arm)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-o", tmp, _SRC])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB)
            lib.dp_oracle_mcm.argtypes = [ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p]
            lib.dp_oracle_mcm.restype = ctypes.c_int
            lib.dp_oracle_interval.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p,
                                               ctypes.c_void_p]
            lib.dp_oracle_interval.restype = ctypes.c_int
            lib.dp_oracle_sdp.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32]
            lib.dp_oracle_sdp.restype = ctypes.c_int
            _lib = lib
    return _lib


class OracleError(RuntimeError):
    pass


def mcm(p) -> tuple[np.ndarray, np.ndarray]:
    """Full MCM tables for dims p[0..n]: m (int64, n x n) and s (int16, n x n),
    m = 0 and s = -1 on and below the diagonal, ties to the smallest k."""
    lib = _load()
    p = np.ascontiguousarray(np.asarray(p, dtype=np.int32))
    n = int(p.size) - 1
    m = np.empty((max(n, 0), max(n, 0)), dtype=np.int64)
    s = np.empty((max(n, 0), max(n, 0)), dtype=np.int16)
    rc = lib.dp_oracle_mcm(p.ctypes.data, n, m.ctypes.data, s.ctypes.data)
    if rc != 0:
        raise OracleError(f"dp_oracle_mcm failed with status {rc}")
    return m, s


def mcm_cell(p, i: int, j: int) -> tuple[int, int]:
    """m[i][j] and s[i][j] of the chain p, computed from the sub-chain
    A_i..A_j only (dims p[i..j+1])."""
    sub = np.asarray(p, dtype=np.int32)[i:j + 2]
    m, s = mcm(sub)
    kk = int(s[0, j - i])
    return int(m[0, j - i]), (kk + i if kk >= 0 else -1)


def interval(p, w) -> tuple[np.ndarray, np.ndarray]:
    """Interval-DP tables for rank-1 factors p[0..n] (>= 0) and the per-cell
    weight w (n x n, entries with i < j read, >= 0): m (int64) and s (int16),
    m = 0 and s = -1 on and below the diagonal, ties to the smallest k."""
    lib = _load()
    p = np.ascontiguousarray(np.asarray(p, dtype=np.int32))
    n = int(p.size) - 1
    w = np.ascontiguousarray(np.asarray(w, dtype=np.int64))
    if w.shape != (n, n):
        raise ValueError(f"w must be {n} x {n}, got {w.shape}")
    m = np.empty((max(n, 0), max(n, 0)), dtype=np.int64)
    s = np.empty((max(n, 0), max(n, 0)), dtype=np.int16)
    rc = lib.dp_oracle_interval(p.ctypes.data, w.ctypes.data, n, m.ctypes.data, s.ctypes.data)
    if rc != 0:
        raise OracleError(f"dp_oracle_interval failed with status {rc}")
    return m, s


def interval_cell(p, w, i: int, j: int) -> tuple[int, int]:
    """m[i][j] and s[i][j] of the interval DP, from the sub-problem on
    i..j alone (p[i..j+1] and the block w[i..j, i..j])."""
    sub_p = np.asarray(p, dtype=np.int32)[i:j + 2]
    sub_w = np.asarray(w, dtype=np.int64)[i:j + 1, i:j + 1]
    m, s = interval(sub_p, sub_w)
    kk = int(s[0, j - i])
    return int(m[0, j - i]), (kk + i if kk >= 0 else -1)


def sdp(preset, n: int, a, op: str | int) -> np.ndarray:
    """S-DP table of length n: ST[0..a_1-1] = preset, the rest by Fig. 1.
    op is "min" / 0 or "add" / 1 (addition modulo 2^32)."""
    lib = _load()
    opc = {"min": 0, "add": 1}.get(op, op)
    a = np.ascontiguousarray(np.asarray(a, dtype=np.int32))
    preset = np.asarray(preset, dtype=np.uint32)
    a1 = int(a[0])
    st = np.zeros(max(n, a1), dtype=np.uint32)
    st[:a1] = preset[:a1]
    rc = lib.dp_oracle_sdp(st.ctypes.data, int(n), a.ctypes.data, int(a.size), int(opc))
    if rc != 0:
        raise OracleError(f"dp_oracle_sdp failed with status {rc}")
    return st[:n].copy()


def diag_major_index(n: int, r: int, c: int) -> int:
    """1-based position of CLRS cell (r, c) (1 <= r <= c <= n) in the linear
    table of Section IV-B: diagonals in computation order (d = c - r from 0),
    rows ascending inside a diagonal.  Diagonal d starts after
    sum_{e<d} (n - e) = d*n - d(d-1)/2 earlier cells."""
    d = c - r
    return d * n - d * (d - 1) // 2 + r


def mcm_operand_pairs(n: int, idx: int) -> list[tuple[int, int]]:
    """For linear position idx (CLRS cell (r, c) with c > r), the pairs
    (l, r) of linear positions combined by f in Eq. (2), in split order
    k = r .. c-1: l = cell (r, k), r = cell (k+1, c)."""
    for d in range(n):
        for r in range(1, n - d + 1):
            if diag_major_index(n, r, r + d) == idx:
                c = r + d
                return [(diag_major_index(n, r, k), diag_major_index(n, k + 1, c)) for k in range(r, c)]
    raise ValueError(idx)
