"""Seeded synthetic inputs for the MCM and S-DP workloads.

This module is the only code shared by the CUDA path's callers and the CPU
oracle's callers: it draws random numbers and arranges them into problem
instances, and it holds none of the dynamic-programming arithmetic.

Generator: splitmix64 (S. Vigna, "Further scramblings of Marsaglia's xorshift
generators", the public splitmix64 finaliser).  The state starts at the seed;
draw number t (t = 1, 2, ...) is the finaliser applied to seed + t * GAMMA
(mod 2^64), GAMMA = 0x9E3779B97F4A7C15.  Because the state only advances by
GAMMA, draws can be produced in vectorised blocks.

Bounded integers use Lemire's multiply-shift method on the upper 32 bits of a
draw (D. Lemire, "Fast random integer generation in an interval", 2019), with
rejection, so every value in [lo, hi] is equally likely.  Rejected draws are
skipped in order, which keeps the stream identical however it is blocked.

Log-uniform integers: n = min(hi, floor(exp(u))) with u uniform in
[ln lo, ln(hi + 1)), u built from the top 53 bits of one draw.

Workloads (the matrix-chain problem of the paper's Section IV-A and the
simplified DP problem of Definition 1):
  * ``mcm_dims(n, lo, hi, seed)``: the n+1 dimensions p[0..n] of one chain.
  * ``sdp_offsets_32(seed)`` / ``sdp_instance_big(seed)``: 32 distinct offsets
    in [1024, 8192] with 8192 and 1024 always present, sorted descending, and
    8192 preset values, for a 2^26-cell table.
  * ``mcm_batch(...)``: many chains with log-uniform lengths.
  * ``serve_trace(...)``: a Poisson arrival trace of mixed MCM / S-DP requests.
  * ``interval_random(n, pmax, wmax, seed)`` / ``interval_obst(n, fmax, seed)``:
    instances of the interval DP with a per-cell weight (the triangular-table
    DP of Section IV with a more general combining function): uniform factors
    and weights, or the optimal-binary-search-tree shape (no rank-1 factors;
    the weight of cell (i, j) is the total frequency of keys i+1..j and gaps
    i..j).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

MASK64 = (1 << 64) - 1
GAMMA = 0x9E3779B97F4A7C15
_M1 = 0xBF58476D1CE4E5B9
_M2 = 0x94D049BB133111EB


def _mix(z: np.ndarray) -> np.ndarray:
    """splitmix64 output finaliser on a uint64 array (wrapping arithmetic)."""
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * np.uint64(_M1)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(_M2)
        return z ^ (z >> np.uint64(31))


def _mix_int(z: int) -> int:
    """The same finaliser on one Python int (wrapping to 64 bits)."""
    z = ((z ^ (z >> 30)) * _M1) & MASK64
    z = ((z ^ (z >> 27)) * _M2) & MASK64
    return z ^ (z >> 31)


class SplitMix64:
    """Counter-style splitmix64 stream: draw t is mix(seed + t * GAMMA).
    Single draws take a scalar path with the same arithmetic (no arrays)."""

    def __init__(self, seed: int):
        self.seed = int(seed) & MASK64
        self.count = 0  # draws consumed so far

    def _raw1(self) -> int:
        self.count += 1
        return _mix_int((self.seed + self.count * GAMMA) & MASK64)

    def raw(self, count: int) -> np.ndarray:
        """The next ``count`` 64-bit draws as a uint64 array."""
        t = np.arange(self.count + 1, self.count + 1 + count, dtype=np.uint64)
        with np.errstate(over="ignore"):
            z = np.uint64(self.seed) + t * np.uint64(GAMMA)
        self.count += count
        return _mix(z)

    def next_u64(self) -> int:
        return self._raw1()

    def randint1(self, lo: int, hi: int) -> int:
        """One integer uniform in [lo, hi]: the draws randint(lo, hi, 1) uses."""
        span = hi - lo + 1
        assert 1 <= span <= (1 << 32)
        if span == (1 << 32):
            return (self._raw1() >> 32) + lo
        thresh = ((1 << 32) - span) % span
        while True:
            prod = (self._raw1() >> 32) * span
            if (prod & 0xFFFFFFFF) >= thresh:
                return (prod >> 32) + lo

    def uniform1(self) -> float:
        """One double uniform in [0, 1): the draw uniform(1) uses."""
        return (self._raw1() >> 11) * (1.0 / (1 << 53))

    def randint(self, lo: int, hi: int, count: int) -> np.ndarray:
        """``count`` integers uniform in [lo, hi] (inclusive), int64 array."""
        span = hi - lo + 1
        assert 1 <= span <= (1 << 32)
        if span == (1 << 32):
            return (self.raw(count) >> np.uint64(32)).astype(np.int64) + lo
        thresh = ((1 << 32) - span) % span
        out = np.empty(count, dtype=np.int64)
        got = 0
        while got < count:
            need = count - got
            block = need + need // 16 + 8
            start = self.count
            x = self.raw(block) >> np.uint64(32)
            prod = x * np.uint64(span)
            low = prod & np.uint64(0xFFFFFFFF)
            ok = low >= np.uint64(thresh)
            idx = np.flatnonzero(ok)
            take = idx[:need]
            out[got:got + take.size] = (prod[take] >> np.uint64(32)).astype(np.int64) + lo
            got += take.size
            # rewind the stream to just after the last draw actually used
            self.count = start + (int(take[-1]) + 1 if take.size == need else block)
        return out

    def uniform(self, count: int) -> np.ndarray:
        """``count`` doubles uniform in [0, 1) from the top 53 bits of a draw."""
        return (self.raw(count) >> np.uint64(11)).astype(np.float64) * (1.0 / (1 << 53))

    def u32(self, count: int) -> np.ndarray:
        """``count`` uint32 values (top 32 bits of each draw)."""
        return (self.raw(count) >> np.uint64(32)).astype(np.uint32)

    def log_uniform_int(self, lo: int, hi: int) -> int:
        u = self.uniform1()
        a, b = math.log(lo), math.log(hi + 1)
        return min(hi, int(math.floor(math.exp(a + u * (b - a)))))

    def distinct_sorted_desc(self, lo: int, hi: int, count: int) -> list[int]:
        """``count`` distinct integers from [lo, hi], drawn one by one (repeats
        re-drawn), returned in descending order."""
        seen: list[int] = []
        have = set()
        while len(seen) < count:
            v = self.randint1(lo, hi)
            if v not in have:
                have.add(v)
                seen.append(v)
        return sorted(seen, reverse=True)


# ----------------------------------------------------------------------------
# matrix-chain workloads
# ----------------------------------------------------------------------------

def mcm_dims(n: int, lo: int, hi: int, seed: int) -> np.ndarray:
    """Dimensions p[0..n] (int32) of an n-matrix chain, uniform in [lo, hi]."""
    return SplitMix64(seed).randint(lo, hi, n + 1).astype(np.int32)


def mcm_small(seed: int = 0) -> np.ndarray:
    """128-matrix chain, dims uniform in [1, 32], seed 0."""
    return mcm_dims(128, 1, 32, seed)


def mcm_big(seed: int = 1) -> np.ndarray:
    """4096-matrix chain, dims uniform in [1, 32], seed 1."""
    return mcm_dims(4096, 1, 32, seed)


@dataclass
class McmBatch:
    ns: np.ndarray                  # int32[B] chain lengths
    p_all: np.ndarray               # int32[sum(n_b + 1)] concatenated dims
    p_off: np.ndarray               # int64[B + 1] prefix offsets into p_all
    tab_off: np.ndarray             # int64[B + 1] element offsets of each n_b*n_b table

    def dims(self, b: int) -> np.ndarray:
        return self.p_all[self.p_off[b]:self.p_off[b + 1]]


def mcm_batch(count: int = 10000, nlo: int = 8, nhi: int = 512, dlo: int = 1,
              dhi: int = 1000, seed: int = 3) -> McmBatch:
    """``count`` chains; per chain one log-uniform length n in [nlo, nhi], then
    its n+1 dims uniform in [dlo, dhi], all from one stream."""
    rng = SplitMix64(seed)
    ns = np.empty(count, dtype=np.int32)
    parts = []
    for b in range(count):
        n = rng.log_uniform_int(nlo, nhi)
        ns[b] = n
        parts.append(rng.randint(dlo, dhi, n + 1).astype(np.int32))
    p_all = np.concatenate(parts) if parts else np.zeros(0, np.int32)
    p_off = np.zeros(count + 1, dtype=np.int64)
    p_off[1:] = np.cumsum(ns.astype(np.int64) + 1)
    tab_off = np.zeros(count + 1, dtype=np.int64)
    tab_off[1:] = np.cumsum(ns.astype(np.int64) ** 2)
    return McmBatch(ns=ns, p_all=p_all, p_off=p_off, tab_off=tab_off)


# ----------------------------------------------------------------------------
# simplified-DP (Definition 1) workloads
# ----------------------------------------------------------------------------

@dataclass
class SdpInstance:
    n: int
    offsets: np.ndarray   # int32[k], strictly decreasing, offsets[0] = a_1
    preset: np.ndarray    # uint32[a_1], the values ST[0 .. a_1 - 1]


def sdp_instance_big(seed: int = 2, n: int = 1 << 26) -> SdpInstance:
    """k = 32 offsets: 30 distinct draws from [1025, 8191] plus 8192 and 1024,
    sorted descending; preset ST[0..8191] uniform uint32."""
    rng = SplitMix64(seed)
    mids = rng.distinct_sorted_desc(1025, 8191, 30)
    offs = np.array(sorted(mids + [8192, 1024], reverse=True), dtype=np.int32)
    preset = rng.u32(int(offs[0]))
    return SdpInstance(n=n, offsets=offs, preset=preset)


def sdp_random(n: int, k: int, amin: int, amax: int, seed: int,
               preset_hi: int | None = None) -> SdpInstance:
    """k distinct offsets from [amin, amax] (descending) and a uniform preset
    of length a_1 (uint32, or uniform in [0, preset_hi] when given)."""
    rng = SplitMix64(seed)
    offs = np.array(rng.distinct_sorted_desc(amin, amax, k), dtype=np.int32)
    a1 = int(offs[0])
    if preset_hi is None:
        preset = rng.u32(a1)
    else:
        preset = rng.randint(0, preset_hi, a1).astype(np.uint32)
    return SdpInstance(n=n, offsets=offs, preset=preset)


# ----------------------------------------------------------------------------
# serving trace
# ----------------------------------------------------------------------------

@dataclass
class Request:
    t_arrival: float          # seconds from trace start
    kind: str                 # "mcm" or "sdp"
    n: int
    dims: np.ndarray | None = None       # MCM: int32[n + 1]
    offsets: np.ndarray | None = None    # S-DP: int32[k]
    preset: np.ndarray | None = None     # S-DP: uint32[a_1]


def serve_trace(rate: float = 2000.0, duration: float = 60.0, seed: int = 4,
                mcm_frac: float = 0.8, mcm_n=(16, 2048), mcm_d=(1, 1000),
                sdp_n=(1 << 16, 1 << 24), sdp_k: int = 16, sdp_a=(64, 4096),
                max_requests: int | None = None) -> list[Request]:
    """Open-loop Poisson trace.  Per request, in draw order: exponential gap,
    kind (MCM with probability ``mcm_frac``), length, then dims (MCM) or
    offsets and preset (S-DP)."""
    rng = SplitMix64(seed)
    out: list[Request] = []
    t = 0.0
    while True:
        u = rng.uniform1()
        t += -math.log(1.0 - u) / rate
        if t >= duration or (max_requests is not None and len(out) >= max_requests):
            break
        kind = "mcm" if rng.uniform1() < mcm_frac else "sdp"
        if kind == "mcm":
            n = rng.log_uniform_int(*mcm_n)
            dims = rng.randint(mcm_d[0], mcm_d[1], n + 1).astype(np.int32)
            out.append(Request(t, kind, n, dims=dims))
        else:
            n = rng.log_uniform_int(*sdp_n)
            offs = np.array(rng.distinct_sorted_desc(sdp_a[0], sdp_a[1], sdp_k), dtype=np.int32)
            preset = rng.u32(int(offs[0]))
            out.append(Request(t, kind, n, offsets=offs, preset=preset))
    return out


# ----------------------------------------------------------------------------
# interval DP with a per-cell weight
# ----------------------------------------------------------------------------

@dataclass
class IntervalInstance:
    p: np.ndarray                   # int32[n+1] rank-1 factors (zeros: no rank-1 term)
    w: np.ndarray                   # int64[n, n] weights, zero on and below the diagonal

    @property
    def n(self) -> int:
        return int(self.p.size) - 1


def interval_random(n: int, pmax: int, wmax: int, seed: int) -> IntervalInstance:
    """Factors uniform in [0, pmax] and weights uniform in [0, wmax] above the
    diagonal (drawn row by row)."""
    g = SplitMix64(seed)
    p = g.randint(0, pmax, n + 1).astype(np.int32)
    w = np.zeros((n, n), dtype=np.int64)
    iu = np.triu_indices(n, 1)
    w[iu] = g.randint(0, wmax, iu[0].size)
    return IntervalInstance(p, w)


def interval_obst(n: int, fmax: int, seed: int) -> IntervalInstance:
    """Optimal-BST shape over n gaps (n - 1 keys): key frequencies uniform in
    [1, fmax], gap frequencies uniform in [0, fmax]; no rank-1 factors; the
    weight of cell (i, j), i < j, is the frequency of keys i+1..j plus that of
    gaps i..j."""
    g = SplitMix64(seed)
    key = np.concatenate([[0], g.randint(1, fmax, n - 1)]) if n > 1 else np.zeros(1, np.int64)
    gap = g.randint(0, fmax, n)
    kc = np.cumsum(key)                          # kc[j] = keys 1..j
    gc = np.concatenate([[0], np.cumsum(gap)])   # gc[t] = gaps 0..t-1
    w = (kc[None, :] - kc[:, None]) + (gc[None, 1:] - gc[:n, None])
    w = np.triu(w, 1).astype(np.int64)
    return IntervalInstance(np.zeros(n + 1, dtype=np.int32), w)
