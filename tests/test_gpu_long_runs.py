"""Long runs and whole states against the oracle.

* Hundreds to a thousand generations at levels where a launch has thousands
  of tiles (and, at the benchmark's tile depths, more tiles than CTAs, so each
  CTA streams several tiles through its pipeline stages and reuses their
  barrier phases): the whole final state is compared with the oracle's, via
  the SHA-256 of its k^r bytes and its live-cell count, at several
  checkpoint generations.  The expected fingerprints were written by
  ``tests/golden/make_long_runs.py``, which runs the oracle only.
* A mix of 100 uneven instances advanced 200 generations by one batched run.
* The triangle at r = 20 under the benchmark's own plan: the whole initial
  state is made by the oracle on the host, one generation runs on the GPU,
  and whole contiguous ranges of 3^16 cells (start, middle, end, and one
  offset across tile boundaries) are compared with the oracle's step of
  those ranges.
"""
import hashlib
import json
import os

import numpy as np
import pytest
import torch

import oracle
from paper_2110_12952_gb300 import workloads as W

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "long_runs.json")
RUNS = {}
if os.path.exists(GOLDEN):
    with open(GOLDEN) as _fh:
        RUNS = json.load(_fh)

# cases at the benchmark's tile depth whose launch has more tiles than CTAs
MANY_TILES_PER_CTA = {"triangle_r16_L9", "carpet_r8_L4", "vicsek_r11_L6", "menger_r6_L3"}


@pytest.fixture(scope="module")
def P():
    from paper_2110_12952_gb300 import build
    build.build()
    import paper_2110_12952_gb300 as pkg
    return pkg


def digest(t: torch.Tensor) -> str:
    return hashlib.sha256(t.cpu().numpy().tobytes()).hexdigest()


def ora(fam, r):
    return oracle.Fractal(fam.k, fam.s, r, fam.dim, fam.table())


SINGLE = sorted(k for k in RUNS if not k.startswith("_") and k != "batch_mix")


@pytest.mark.parametrize("name", SINGLE)
def test_long_run_whole_state(P, name):
    rec = RUNS[name]
    fam = W.FAMILIES[rec["family"]]
    r, L = rec["r"], rec["tile_levels"]
    g = P.Fractal.from_family(fam, r)
    g.tile_levels = L
    plan = g.plan_info()
    assert plan["tile_levels"] == L
    if name in MANY_TILES_PER_CTA:
        tiles = fam.k ** (r - L)
        assert tiles >= 2 * plan["grid"], (tiles, plan)
    init = ora(fam, r).init_bernoulli(rec["seed"], rec["p"])
    assert hashlib.sha256(init.tobytes()).hexdigest() == rec["init_sha256"]
    a = torch.from_numpy(init).cuda()
    b = torch.empty_like(a)
    rule = W.default_rule(fam)
    done = 0
    for cp in rec["checkpoints"]:
        t = cp["generation"]
        g.step(a, out=b, steps=t - done, rule=rule)
        a, b = b, a
        done = t
        assert int(torch.count_nonzero(a).item()) == cp["live"], f"{name}: live cells at generation {t}"
        assert digest(a) == cp["sha256"], f"{name}: state at generation {t}"
    assert g._lib.fractal_check(g._h) == 0
    del a, b
    g.close()
    torch.cuda.empty_cache()


def test_batch_mix_200_generations(P):
    assert "batch_mix" in RUNS, "tests/golden/long_runs.json lacks the batch mix"
    rec = RUNS["batch_mix"]
    mix = W.batched_mix(rec["count"], master_seed=rec["master_seed"], steps=rec["steps"],
                        level_ranges={k: tuple(v) for k, v in rec["levels"].items()})
    assert len(mix) == len(rec["instances"])
    handles, outs = {}, []
    batch = P.Batch()
    for inst, want in zip(mix, rec["instances"]):
        assert (inst.family.name, inst.r, inst.seed) == (want["family"], want["r"], want["seed"])
        key = (inst.family.name, inst.r)
        if key not in handles:
            handles[key] = P.Fractal.from_family(inst.family, inst.r)
        g = handles[key]
        x = torch.from_numpy(ora(inst.family, inst.r).init_bernoulli(inst.seed, inst.p)).cuda()
        y = torch.empty_like(x)
        batch.add(g, x, y, inst.steps, rule=W.default_rule(inst.family))
        outs.append((x, y))
    for run in range(2):   # the first run builds the graph, the second replays it
        batch.run()
        torch.cuda.synchronize()
        for i, ((_, y), want) in enumerate(zip(outs, rec["instances"])):
            assert int(torch.count_nonzero(y).item()) == want["live"], (run, i)
            assert digest(y) == want["sha256"], (run, i)
    batch.close()
    for g in handles.values():
        g.close()


def test_triangle_r20_whole_ranges_bench_plan(P):
    inst = W.TRI_R20
    fam, r = inst.family, inst.r
    o = ora(fam, r)
    cells = fam.k ** r
    init = o.init_bernoulli(inst.seed, inst.p)          # the whole state, by the oracle
    g = P.Fractal.from_family(fam, r)
    a = torch.from_numpy(init).cuda()
    b = torch.empty_like(a)
    g.autotune(a, b)                                    # the bench's own plan
    g.step(a, out=b, steps=1)
    torch.cuda.synchronize()
    n = 3 ** 16
    tile = 3 ** g.tile_levels
    starts = [0, cells // 2 - n // 2, cells - n, 7 * n + 5 * tile + 4321]
    ref = np.zeros(cells, dtype=np.uint8)
    assert starts[3] % tile != 0     # this one starts inside a tile
    for w0 in starts:
        o.step_range(init, w0, w0 + n, out=ref)
        got = b[w0:w0 + n].cpu().numpy()
        assert np.array_equal(got, ref[w0:w0 + n]), f"range starting at {w0}"
    del a, b
    g.close()
    torch.cuda.empty_cache()
