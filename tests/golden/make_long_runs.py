"""Write ``long_runs.json``: fingerprints of the whole state after long runs of
the CPU oracle, for the long-horizon GPU parity tests.

The oracle's compact step (``oracle.Fractal.step``) is too slow to run
thousands of generations at multi-tile sizes inside a test, so this script
runs it once and stores, per workload and checkpoint generation, the live-cell
count and the SHA-256 of the whole state (one byte per compact cell in omega
order).  A GPU state with the same digest is the same state, byte for byte.

Only ``oracle/`` computes here: the initial states come from the oracle's own
Bernoulli initialiser (SplitMix64), and ``workloads`` only supplies the
offset tables, rules and the seeded instance mix.

Run: ``python tests/golden/make_long_runs.py [--only NAME ...]``
(about an hour of 8-core CPU time for the whole list).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import oracle  # noqa: E402
from paper_2110_12952_gb300 import workloads as W  # noqa: E402

OUT = os.path.join(HERE, "long_runs.json")

# name: (family, r, p, seed, checkpoints, tile depth the GPU test pins).  The
# tile depths are the ones the benchmark's autotuner picks at the full sizes
# (triangle 9, carpet 4, Vicsek 6, Menger 3) plus shallower ones, at levels
# where each launch has more tiles than CTAs, so that every CTA streams many
# tiles through its pipeline stages.
SINGLE = {
    "triangle_r16_L9": (W.TRIANGLE, 16, 0.3, 21, (1, 10, 50, 100), 9),
    "triangle_r13_L7": (W.TRIANGLE, 13, 0.3, 22, (1, 10, 100, 1000), 7),
    "triangle_r12_L5": (W.TRIANGLE, 12, 0.5, 23, (1, 100, 1000), 5),
    "carpet_r8_L4": (W.CARPET, 8, 0.5, 24, (1, 10, 100), 4),
    "carpet_r7_L2": (W.CARPET, 7, 0.5, 25, (1, 100, 500), 2),
    "vicsek_r11_L6": (W.VICSEK, 11, 0.5, 26, (1, 10, 50), 6),
    "vicsek_r9_L3": (W.VICSEK, 9, 0.5, 27, (1, 100, 500), 3),
    "menger_r6_L3": (W.MENGER, 6, 0.5, 28, (1, 5, 20), 3),
    "menger_r5_L2": (W.MENGER, 5, 0.5, 29, (1, 100, 200), 2),
}

# a mix of independent instances, as the batched workload draws them, at
# smaller levels; every instance runs BATCH_STEPS generations
BATCH_COUNT, BATCH_SEED, BATCH_STEPS = 100, 71, 200
BATCH_LEVELS = {"triangle": (6, 11), "carpet": (3, 6), "vicsek": (3, 7)}


def rule_of(fam):
    b, s = W.default_rule(fam)
    return oracle.Rule(b, s)


def digest(state: np.ndarray) -> str:
    return hashlib.sha256(np.ascontiguousarray(state).tobytes()).hexdigest()


def run_single(name):
    fam, r, p, seed, checkpoints, L = SINGLE[name]
    o = oracle.Fractal(fam.k, fam.s, r, fam.dim, fam.table())
    x = o.init_bernoulli(seed, p)
    rec = {"family": fam.name, "r": r, "p": p, "seed": seed, "tile_levels": L,
           "init_sha256": digest(x), "checkpoints": []}
    done = 0
    for t in checkpoints:
        x = o.step(x, rule=rule_of(fam), steps=t - done)
        done = t
        rec["checkpoints"].append({"generation": t, "live": int(np.count_nonzero(x)),
                                   "sha256": digest(x)})
    return rec


def batch_mix():
    return W.batched_mix(BATCH_COUNT, master_seed=BATCH_SEED, steps=BATCH_STEPS,
                         level_ranges=BATCH_LEVELS)


def run_batch():
    out = []
    for inst in batch_mix():
        fam = inst.family
        o = oracle.Fractal(fam.k, fam.s, inst.r, fam.dim, fam.table())
        x = o.init_bernoulli(inst.seed, inst.p)
        y = o.step(x, rule=rule_of(fam), steps=inst.steps)
        out.append({"family": fam.name, "r": inst.r, "seed": inst.seed, "p": inst.p,
                    "steps": inst.steps, "live": int(np.count_nonzero(y)), "sha256": digest(y)})
    return {"count": BATCH_COUNT, "master_seed": BATCH_SEED, "steps": BATCH_STEPS,
            "levels": BATCH_LEVELS, "instances": out}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--only", nargs="*", default=None)
    args = ap.parse_args()
    data = {}
    if os.path.exists(OUT):
        with open(OUT) as fh:
            data = json.load(fh)
    data["_about"] = ("whole-state fingerprints of oracle runs (live cells, SHA-256 of the "
                      "k^r state bytes in omega order); written by make_long_runs.py")
    names = list(SINGLE) + ["batch_mix"]
    for name in names:
        if args.only is not None and name not in args.only:
            continue
        t0 = time.time()
        data[name] = run_batch() if name == "batch_mix" else run_single(name)
        print(f"{name}: {time.time() - t0:.0f} s", flush=True)
        with open(OUT + ".tmp", "w") as fh:
            json.dump(data, fh, indent=1, sort_keys=True)
        os.replace(OUT + ".tmp", OUT)


if __name__ == "__main__":
    main()
