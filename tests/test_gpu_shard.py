"""The sharded step on one GPU: 2 or 3 shards of one instance, each with its
own buffer (own tiles + halo), advanced generation by generation with the
halo exchange done by device copies, must give exactly the oracle's state
once the shards' own parts are put back together.  The policies of the
triangle, carpet, Vicsek fractal and Menger sponge are all covered, and one
case runs the benchmark's tile depth (9) at r = 16 for 50 generations against
the oracle fingerprint of the long-run tests."""
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


def run_sharded(P, fam, r, L, nshards, init, gens):
    from paper_2110_12952_gb300.shard import ShardPlan, exchange_local
    g = P.Fractal.from_family(fam, r)
    plans = [ShardPlan.from_family(fam, r, L, nshards, i) for i in range(nshards)]
    for p in plans:
        p.attach(g)
    x = torch.from_numpy(init).cuda()
    a = [torch.zeros(p.buffer_cells, dtype=torch.uint8, device="cuda") for p in plans]
    b = [torch.zeros_like(t) for t in a]
    for p, t in zip(plans, a):
        t[: p.local_cells].copy_(x[p.first_cell: p.first_cell + p.local_cells])
    rule = W.default_rule(fam)
    for _ in range(gens):
        exchange_local(plans, a)
        for p, i, o in zip(plans, a, b):
            p.step(i, o, rule=rule)
        a, b = b, a
    out = torch.empty_like(x)
    for p, t in zip(plans, a):
        out[p.first_cell: p.first_cell + p.local_cells].copy_(t[: p.local_cells])
    assert g._lib.fractal_check(g._h) == 0
    for p in plans:
        p.close()
    return out


@pytest.mark.parametrize("fam,r,L,n,gens", [
    (W.TRIANGLE, 12, 5, 2, 12), (W.TRIANGLE, 12, 9, 3, 12), (W.TRIANGLE, 11, 3, 3, 6),
    (W.CARPET, 6, 2, 3, 8), (W.CARPET, 6, 4, 2, 8), (W.VICSEK, 7, 3, 2, 8), (W.VICSEK, 8, 6, 3, 5),
    (W.MENGER, 4, 2, 2, 4), (W.MENGER, 4, 3, 3, 3)], ids=lambda v: getattr(v, "name", str(v)))
def test_sharded_matches_oracle(P, fam, r, L, n, gens):
    o = oracle.Fractal(fam.k, fam.s, r, fam.dim, fam.table())
    init = o.init_bernoulli(70 + r + n, 0.45)
    got = run_sharded(P, fam, r, L, n, init, gens)
    want = o.step(init, rule=oracle.Rule(*W.default_rule(fam)), steps=gens)
    assert np.array_equal(got.cpu().numpy(), want)


def test_sharded_bench_depth_long_run(P):
    path = os.path.join(os.path.dirname(__file__), "golden", "long_runs.json")
    with open(path) as fh:
        rec = json.load(fh)["triangle_r16_L9"]
    init = oracle.Fractal(3, 2, 16, 2, W.TRIANGLE.table()).init_bernoulli(rec["seed"], rec["p"])
    cp = next(c for c in rec["checkpoints"] if c["generation"] == 50)
    got = run_sharded(P, W.TRIANGLE, 16, rec["tile_levels"], 3, init, 50)
    assert int(torch.count_nonzero(got).item()) == cp["live"]
    assert hashlib.sha256(got.cpu().numpy().tobytes()).hexdigest() == cp["sha256"]
