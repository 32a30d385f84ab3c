"""Write full-size expected values for the parity tests.

Calls only the CPU oracle (``oracle/``) and the seeded input generator; never
the CUDA path.  Output: ``tests/golden/fullsize.json`` holding SHA-256 digests
of whole tables (little-endian, the cost type each workload is stated in) and
a few sampled cells, so the GPU tests can check full-size results bit for bit
without re-running the single-threaded oracle on the GPU host.

Run:  python tests/golden/make_golden.py [--skip-batch] [--only NAME,NAME]
(The 4096-matrix chain takes a few minutes on one core.  --only recomputes
the named entries and keeps the others.)
"""
import argparse
import hashlib
import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_2008_01938_gb300 import inputs  # noqa: E402

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "fullsize.json")


def sha(a: np.ndarray) -> str:
    return hashlib.sha256(np.ascontiguousarray(a).tobytes()).hexdigest()


def mcm_entry(p, cost_dtype):
    t = time.time()
    m, s = oracle.mcm(p)
    n = p.size - 1
    rng = np.random.default_rng(n)
    cells = []
    for _ in range(16):
        i, j = sorted(rng.integers(0, n, 2).tolist())
        cells.append([i, j, int(m[i, j]), int(s[i, j])])
    cells.append([0, n - 1, int(m[0, n - 1]), int(s[0, n - 1])])
    return {
        "n": int(n),
        "m_dtype": cost_dtype,
        "m_sha256": sha(m.astype(cost_dtype).astype(np.dtype(cost_dtype).newbyteorder("<"))),
        "s_sha256": sha(s.astype("<i2")),
        "cells": cells,
        "oracle_seconds": round(time.time() - t, 2),
    }


def interval_entry(inst, cost_dtype):
    t = time.time()
    m, s = oracle.interval(inst.p, inst.w)
    n = inst.n
    rng = np.random.default_rng(n + 1)
    cells = []
    for _ in range(16):
        i, j = sorted(rng.integers(0, n, 2).tolist())
        cells.append([i, j, int(m[i, j]), int(s[i, j])])
    cells.append([0, n - 1, int(m[0, n - 1]), int(s[0, n - 1])])
    return {
        "n": int(n),
        "m_dtype": cost_dtype,
        "m_sha256": sha(m.astype(cost_dtype).astype(np.dtype(cost_dtype).newbyteorder("<"))),
        "s_sha256": sha(s.astype("<i2")),
        "cells": cells,
        "oracle_seconds": round(time.time() - t, 2),
    }


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--skip-batch", action="store_true")
    ap.add_argument("--only", default="")
    args = ap.parse_args()
    out = json.load(open(OUT)) if os.path.exists(OUT) else {}
    only = set(x for x in args.only.split(",") if x)

    def want(name):
        return not only or name in only

    if want("mcm_n128_seed0"):
        out["mcm_n128_seed0"] = mcm_entry(inputs.mcm_small(), "int32")
        print("n=128 done", flush=True)
    if want("mcm_n4096_seed1"):
        out["mcm_n4096_seed1"] = mcm_entry(inputs.mcm_big(), "int32")
        print("n=4096 done", out["mcm_n4096_seed1"]["oracle_seconds"], flush=True)
    if want("interval_obst_n4096_seed5"):
        out["interval_obst_n4096_seed5"] = interval_entry(inputs.interval_obst(4096, 4, seed=5), "int32")
        print("interval n=4096 done", out["interval_obst_n4096_seed5"]["oracle_seconds"], flush=True)

    big = inputs.sdp_instance_big()
    for op in ("min", "add"):
        if not want(f"sdp_n2p26_seed2_{op}"):
            continue
        t = time.time()
        st = oracle.sdp(big.preset, big.n, big.offsets, op)
        idx = [8192, 8193, 10000, 1 << 20, (1 << 26) - 1]
        out[f"sdp_n2p26_seed2_{op}"] = {
            "n": big.n,
            "st_sha256": sha(st.astype("<u4")),
            "samples": [[i, int(st[i])] for i in idx],
            "oracle_seconds": round(time.time() - t, 2),
        }
        print("sdp", op, "done", flush=True)

    if not args.skip_batch and want("mcm_batch10000_seed3"):
        b = inputs.mcm_batch()
        t = time.time()
        hm, hs = hashlib.sha256(), hashlib.sha256()
        finals = []
        for i in range(b.ns.size):
            m, s = oracle.mcm(b.dims(i))
            hm.update(m.astype("<i8").tobytes())
            hs.update(s.astype("<i2").tobytes())
            finals.append(int(m[0, -1]))
        out["mcm_batch10000_seed3"] = {
            "count": int(b.ns.size),
            "total_split_evals": int(sum((int(n) ** 3 - int(n)) // 6 for n in b.ns)),
            "m_sha256_concat": hm.hexdigest(),
            "s_sha256_concat": hs.hexdigest(),
            "final_costs_first100": finals[:100],
            "oracle_seconds": round(time.time() - t, 2),
        }
        print("batch done", flush=True)

    with open(OUT, "w") as f:
        json.dump(out, f, indent=1)
    print("wrote", OUT)


if __name__ == "__main__":
    main()
