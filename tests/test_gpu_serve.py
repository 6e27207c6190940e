"""Continuous-batching server (fractal_server_*): every served result must be
the same as the request run alone (and as the oracle), whatever else was
resident, queued or admitted meanwhile; admission respects the HBM budget."""
import threading
import time

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


def test_served_results_match_alone_and_oracle(P):
    rng = np.random.default_rng(77)
    fams = [(W.TRIANGLE, (0, 10)), (W.CARPET, (1, 5)), (W.VICSEK, (1, 6)), (W.MENGER, (1, 3))]
    handles = {}
    reqs = []
    for _ in range(48):
        fam, (lo, hi) = fams[int(rng.integers(0, len(fams)))]
        r = int(rng.integers(lo, hi + 1))
        key = (fam.name, r)
        if key not in handles:
            handles[key] = P.Fractal.from_family(fam, r)
        steps = int(rng.integers(0, 30))
        reqs.append((fam, r, steps, int(rng.integers(0, 2**62)), float(rng.uniform(0.2, 0.6)),
                     bool(rng.integers(0, 4) == 0)))
    # a small budget forces queueing and admission as memory frees up
    srv = P.Server(hbm_budget_bytes=400_000, chunk=4)
    outs, ids = [], []

    def submit_all():
        for fam, r, steps, seed, p, popmode in reqs:
            g = handles[(fam.name, r)]
            host = None if popmode else torch.zeros(g.cells, dtype=torch.uint8).pin_memory()
            outs.append(host)
            ids.append(srv.submit(g, seed, p, steps, rule=W.default_rule(fam), host_out=host))
            time.sleep(float(rng.uniform(0, 0.002)))   # arrivals while others run

    th = threading.Thread(target=submit_all)
    th.start()
    th.join()
    srv.wait_all()
    st = srv.stats()
    assert st["completed"] == len(reqs) and st["queued"] == 0 and st["hbm_used"] == 0
    for (fam, r, steps, seed, p, popmode), host, rid in zip(reqs, outs, ids):
        done, lat, pop = srv.poll(rid)
        assert done and lat > 0
        o = ora(fam, r)
        ref = o.step(o.init_bernoulli(seed, p), rule=oracle.Rule(*W.default_rule(fam)), steps=steps)
        if popmode:
            assert pop == int(ref.sum())
        else:
            assert np.array_equal(host.numpy(), ref), (fam.name, r, steps)
            g = handles[(fam.name, r)]
            alone = g.step(g.init_bernoulli(seed, p), steps=steps, rule=W.default_rule(fam))
            assert np.array_equal(alone.cpu().numpy(), host.numpy())
    srv.close()


def test_server_rejects_request_over_budget(P):
    from paper_2110_12952_gb300.capi import FractalError
    srv = P.Server(hbm_budget_bytes=10_000, chunk=2)
    big = P.Fractal.from_family(W.TRIANGLE, 9)   # 2 x 19683 bytes > budget
    with pytest.raises(FractalError, match="EBUSY"):
        srv.submit(big, 1, 0.5, 3)
    small = P.Fractal.from_family(W.TRIANGLE, 4)
    rid = srv.submit(small, 1, 0.5, 3)
    srv.wait_all()
    assert srv.poll(rid)[0]
    with pytest.raises(FractalError, match="ENOTFOUND"):
        srv.poll(rid + 100)
    srv.close()


def test_handle_not_replanned_while_served(P):
    # a handle with a request still on a server keeps its plan: a new tile
    # depth and the autotuner are refused until the request is done
    from paper_2110_12952_gb300.capi import FractalError
    g = P.Fractal.from_family(W.TRIANGLE, 12)
    L = g.tile_levels
    g.tile_levels = L            # an explicit depth (the automatic choice is -1)
    srv = P.Server(hbm_budget_bytes=0, chunk=1)
    rid = srv.submit(g, 5, 0.4, 400)
    if not srv.poll(rid)[0]:
        with pytest.raises(FractalError, match="EBUSY"):
            g.tile_levels = L - 1
        x = g.init_bernoulli(1, 0.5)
        with pytest.raises(FractalError, match="EBUSY"):
            g.autotune(x, torch.empty_like(x))
    g.tile_levels = L            # the same depth is always accepted
    srv.wait_all()
    assert srv.poll(rid)[0]
    g.tile_levels = L - 1        # done: re-planning is allowed again
    assert g.tile_levels == L - 1
    o = ora(W.TRIANGLE, 12)
    init = o.init_bernoulli(6, 0.4)
    assert np.array_equal(g.step(torch.from_numpy(init).cuda(), steps=3).cpu().numpy(), o.step(init, steps=3))
    srv.close()
