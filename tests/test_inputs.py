"""The seeded input generator: published splitmix64 vectors, Lemire bounds,
stream identity under blocking, and the workload shapes."""
import numpy as np

from paper_2008_01938_gb300 import inputs
from paper_2008_01938_gb300.inputs import SplitMix64


def test_splitmix64_published_vectors():
    # Reference outputs of Vigna's splitmix64 (seed 0 and seed 1234567).
    assert [int(x) for x in SplitMix64(0).raw(3)] == [
        0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]
    assert [int(x) for x in SplitMix64(1234567).raw(3)] == [
        6457827717110365317, 3203168211198807973, 9817491932198370423]


def test_randint_bounds_and_blocking():
    a = SplitMix64(7).randint(1, 32, 5000)
    assert a.min() == 1 and a.max() == 32
    # drawing in pieces gives the same stream as drawing at once
    r = SplitMix64(7)
    b = np.concatenate([r.randint(1, 32, 1), r.randint(1, 32, 999), r.randint(1, 32, 4000)])
    assert np.array_equal(a, b)
    # roughly uniform
    counts = np.bincount(a, minlength=33)[1:]
    assert counts.min() > 100 and counts.max() < 220


def test_randint_rejection_path():
    # span 3 has a non-zero rejection threshold; values stay in range and the
    # stream is identical however it is blocked
    r1 = SplitMix64(99).randint(0, 2, 3000)
    r = SplitMix64(99)
    r2 = np.concatenate([r.randint(0, 2, 17), r.randint(0, 2, 2983)])
    assert np.array_equal(r1, r2)
    assert set(np.unique(r1)) == {0, 1, 2}


def test_workload_shapes():
    p = inputs.mcm_small()
    assert p.dtype == np.int32 and p.size == 129 and p.min() >= 1 and p.max() <= 32
    big = inputs.sdp_instance_big(n=1 << 20)
    a = big.offsets
    assert a.size == 32 and a[0] == 8192 and a[-1] == 1024
    assert np.all(np.diff(a) < 0) and len(set(a.tolist())) == 32
    assert big.preset.size == 8192 and big.preset.dtype == np.uint32
    b = inputs.mcm_batch(count=200, seed=3)
    assert b.ns.min() >= 8 and b.ns.max() <= 512
    assert b.p_off[-1] == b.p_all.size
    assert all(b.dims(i).size == b.ns[i] + 1 for i in range(200))
    # log-uniform: small n are much more common than large n
    assert np.median(b.ns) < 150


def test_serve_trace_shape():
    tr = inputs.serve_trace(rate=2000.0, duration=0.25, seed=4)
    assert 350 < len(tr) < 650
    ts = [r.t_arrival for r in tr]
    assert ts == sorted(ts)
    kinds = [r.kind for r in tr]
    frac = kinds.count("mcm") / len(kinds)
    assert 0.7 < frac < 0.9
    for r in tr:
        if r.kind == "mcm":
            assert 16 <= r.n <= 2048 and r.dims.size == r.n + 1
        else:
            assert (1 << 16) <= r.n <= (1 << 24)
            assert r.offsets.size == 16 and np.all(np.diff(r.offsets) < 0)
            assert r.preset.size == r.offsets[0]


def test_interval_instances():
    a = inputs.interval_random(40, 7, 99, seed=9)
    b = inputs.interval_random(40, 7, 99, seed=9)
    assert np.array_equal(a.p, b.p) and np.array_equal(a.w, b.w)
    assert a.p.dtype == np.int32 and a.p.min() >= 0 and a.p.max() <= 7
    assert a.w.dtype == np.int64 and a.w.min() >= 0 and a.w.max() <= 99
    assert not np.any(np.tril(a.w))                  # nothing on or below the diagonal
    assert a.p.min() == 0 and a.w[np.triu_indices(40, 1)].min() == 0
    # the OBST weight, summed key by key and gap by gap
    o = inputs.interval_obst(30, 5, seed=10)
    assert not np.any(o.p)
    g = inputs.SplitMix64(10)
    key = [0] + g.randint(1, 5, 29).tolist()          # keys 1..29
    gap = g.randint(0, 5, 30).tolist()                # gaps 0..29
    for i in range(30):
        for j in range(i + 1, 30):
            assert o.w[i, j] == sum(key[i + 1:j + 1]) + sum(gap[i:j + 1])
