"""Temporal blocking (fractal_set_temporal_blocking): passes of up to g
generations over bitmap boxes must give exactly the oracle's generations.

* every tile depth and g = 1..9 against the oracle at small levels, with step
  counts that are and are not multiples of g, and with non-binary input;
* thousands of tiles per launch, and the long-run oracle fingerprints (500
  generations of the carpet and the Vicsek fractal);
* the full carpet at r = 10: 18 generations in two passes equal 18 single
  generations of the ordinary step (itself checked against the oracle).
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


@pytest.fixture(scope="module")
def P():
    from paper_2110_12952_gb300 import build
    build.build()
    import paper_2110_12952_gb300 as pkg
    return pkg


def ora(fam, r):
    return oracle.Fractal(fam.k, fam.s, r, fam.dim, fam.table())


@pytest.mark.parametrize("fam,r,L", [(W.CARPET, 4, 2), (W.CARPET, 4, 4), (W.CARPET, 5, 3), (W.VICSEK, 5, 2),
                                     (W.VICSEK, 5, 4), (W.VICSEK, 6, 3), (W.CARPET, 2, 2)],
                         ids=lambda v: getattr(v, "name", str(v)))
def test_temporal_every_pass_length(P, fam, r, L):
    g, o = P.Fractal.from_family(fam, r), ora(fam, r)
    init = o.init_bernoulli(300 + r + L, 0.45)
    x = torch.from_numpy(init).cuda()
    for gens in range(1, 10):
        g.set_temporal_blocking(gens, L)
        for steps in sorted({1, gens, gens + 1, 2 * gens + 3}):
            out = g.step(x, steps=steps)
            assert np.array_equal(out.cpu().numpy(), o.step(init, steps=steps)), (gens, steps)
    g.set_temporal_blocking(0)
    assert np.array_equal(g.step(x, steps=4).cpu().numpy(), o.step(init, steps=4))


@pytest.mark.parametrize("fam,r,L", [(W.CARPET, 5, 3), (W.VICSEK, 5, 3)], ids=lambda v: getattr(v, "name", str(v)))
def test_temporal_nonbinary_input_and_rules(P, fam, r, L):
    g, o = P.Fractal.from_family(fam, r), ora(fam, r)
    rng = np.random.default_rng(r)
    raw = (rng.integers(0, 2, size=g.cells) * rng.integers(1, 256, size=g.cells)).astype(np.uint8)
    g.set_temporal_blocking(9, L)
    for birth, survive in [([3], [2, 3]), ([3, 6], [2, 3]), ([1], [0, 8]), ([0, 2, 8], [1, 4, 5, 7])]:
        rule = W.rule_masks(birth, survive)
        out = g.step(torch.from_numpy(raw).cuda(), steps=11, rule=rule)
        assert np.array_equal(out.cpu().numpy(), o.step(raw, rule=oracle.Rule(*rule), steps=11)), (birth, survive)


@pytest.mark.parametrize("name,gens", [("carpet_r7_L2", 9), ("vicsek_r9_L3", 9), ("carpet_r8_L4", 7)])
def test_temporal_long_runs(P, name, gens):
    with open(os.path.join(os.path.dirname(__file__), "golden", "long_runs.json")) as fh:
        rec = json.load(fh)[name]
    fam = W.FAMILIES[rec["family"]]
    g = P.Fractal.from_family(fam, rec["r"])
    g.set_temporal_blocking(gens)
    a = torch.from_numpy(ora(fam, rec["r"]).init_bernoulli(rec["seed"], rec["p"])).cuda()
    done = 0
    for cp in rec["checkpoints"]:
        a = g.step(a, steps=cp["generation"] - done)
        done = cp["generation"]
        assert int(torch.count_nonzero(a).item()) == cp["live"], (name, done)
        assert hashlib.sha256(a.cpu().numpy().tobytes()).hexdigest() == cp["sha256"], (name, done)


def test_temporal_full_size_carpet_matches_single_generations(P):
    inst = W.CARPET_R10
    g = P.Fractal.from_family(inst.family, inst.r)
    x = g.init_bernoulli(inst.seed, inst.p)
    want = g.step(x, steps=18)
    g.set_temporal_blocking(9)
    got = g.step(x, steps=18)
    assert torch.equal(got, want)
    assert g._lib.fractal_check(g._h) == 0
    del x, want, got
    torch.cuda.empty_cache()


def test_temporal_refused_elsewhere(P):
    from paper_2110_12952_gb300.capi import FractalError
    g = P.Fractal.from_family(W.TRIANGLE, 8)
    with pytest.raises(FractalError, match="EINVAL"):
        g.set_temporal_blocking(4)
    c = P.Fractal.from_family(W.CARPET, 4)
    with pytest.raises(FractalError, match="EINVAL"):
        c.set_temporal_blocking(10)
    with pytest.raises(FractalError, match="EINVAL"):
        c.set_temporal_blocking(3, 1)
