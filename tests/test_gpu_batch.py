"""Batched execution (fractal_batch_*) against the oracle and against the
one-instance path: every instance's result must be the same alone and in the
mix, bit for bit, whatever the other instances are."""
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


def test_batch_mix_matches_oracle_and_alone(P):
    rng = np.random.default_rng(2024)
    specs = []
    fams = [(W.TRIANGLE, (0, 9)), (W.CARPET, (0, 5)), (W.VICSEK, (0, 5)), (W.MENGER, (0, 3)),
            (W.TRIANGLE_MIRRORED, (2, 7))]
    for _ in range(60):
        fam, (lo, hi) = fams[int(rng.integers(0, len(fams)))]
        r = int(rng.integers(lo, hi + 1))
        steps = int(rng.integers(0, 9))
        specs.append((fam, r, steps, int(rng.integers(0, 2**62)), float(rng.uniform(0.2, 0.6))))
    handles = {}
    batch = P.Batch()
    bufs = []
    for fam, r, steps, seed, p in specs:
        key = (fam.name, r)
        if key not in handles:
            handles[key] = P.Fractal.from_family(fam, r)
        g = handles[key]
        x = g.init_bernoulli(seed, p)
        y = torch.full_like(x, 0x55)
        batch.add(g, x, y, steps, rule=W.default_rule(fam))
        bufs.append((x, y))
    batch.run()
    torch.cuda.synchronize()
    updates, launches = batch.stats()
    assert updates == sum(f.k ** r * st for f, r, st, _, _ in specs)
    for (fam, r, steps, seed, p), (x, y) in zip(specs, bufs):
        o = ora(fam, r)
        init = o.init_bernoulli(seed, p)
        assert np.array_equal(x.cpu().numpy(), init)           # input untouched
        ref = o.step(init, rule=oracle.Rule(*W.default_rule(fam)), steps=steps)
        assert np.array_equal(y.cpu().numpy(), ref), (fam.name, r, steps)
        alone = handles[(fam.name, r)].step(x, steps=steps, rule=W.default_rule(fam))
        assert torch.equal(alone, y)
    # replay: new inputs in the same buffers, same graph
    for (fam, r, steps, seed, p), (x, y) in zip(specs, bufs):
        handles[(fam.name, r)].init_bernoulli(seed + 1, p, out=x)
    batch.run()
    torch.cuda.synchronize()
    for (fam, r, steps, seed, p), (x, y) in zip(specs[:20], bufs[:20]):
        o = ora(fam, r)
        ref = o.step(o.init_bernoulli(seed + 1, p), rule=oracle.Rule(*W.default_rule(fam)), steps=steps)
        assert np.array_equal(y.cpu().numpy(), ref)
    batch.close()


def test_batch_large_instances_match_alone(P):
    specs = [(W.TRIANGLE, 12, 5), (W.TRIANGLE, 12, 4), (W.CARPET, 6, 3), (W.VICSEK, 7, 6),
             (W.TRIANGLE, 9, 7), (W.MENGER, 4, 2)]
    batch = P.Batch()
    hs, bufs = [], []
    for i, (fam, r, steps) in enumerate(specs):
        g = P.Fractal.from_family(fam, r)
        x = g.init_bernoulli(100 + i, 0.35)
        y = torch.empty_like(x)
        batch.add(g, x, y, steps, rule=W.default_rule(fam))
        hs.append(g)
        bufs.append((x, y))
    batch.run()
    torch.cuda.synchronize()
    for (fam, r, steps), g, (x, y) in zip(specs, hs, bufs):
        assert torch.equal(g.step(x, steps=steps, rule=W.default_rule(fam)), y), (fam.name, r)
    # one mid-size instance fully against the oracle
    fam, r, steps = specs[4]
    o = ora(fam, r)
    assert np.array_equal(bufs[4][1].cpu().numpy(), o.step(o.init_bernoulli(104, 0.35), steps=steps))
    batch.close()
