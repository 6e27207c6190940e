"""Fractals with a different transition table per level
(fractal_create_mixed) on the GPU against the oracle's per-level definition:
the maps exhaustively, the compact step at every tile depth (and on
non-binary input), the bounding-box step, the box views, a batch mixing them
with ordinary instances, and the calls that refuse them."""
import numpy as np
import pytest
import torch

import oracle
from paper_2110_12952_gb300 import workloads as W

pytestmark = pytest.mark.gpu

CORNERS3 = W.Family("corners3", 9, 3, 3, tuple((x, y, z) for z in range(3) for y in range(3) for x in range(3)
                                               if (x != 1 and y != 1 and z != 1) or (x, y, z) == (1, 1, 1)))
MIXES = {
    "tri_square": (2, 2, [W.TRIANGLE, W.FULL_SQUARE, W.TRIANGLE, W.TRIANGLE_MIRRORED, W.FULL_SQUARE, W.TRIANGLE,
                          W.TRIANGLE]),
    "carpet_vicsek_h": (3, 2, [W.CARPET, W.VICSEK, W.H_FRACTAL, W.CARPET]),
    "vicsek_x_chandelier": (3, 2, [W.VICSEK, W.X_FRACTAL, W.CHANDELIER, W.EMPTY_BOTTLES, W.VICSEK]),
    "menger_corners_3d": (3, 3, [W.MENGER, CORNERS3, W.MENGER]),
}


@pytest.fixture(scope="module")
def P():
    from paper_2110_12952_gb300 import build
    build.build()
    import paper_2110_12952_gb300 as pkg
    return pkg


def pair(P, name):
    s, dim, fams = MIXES[name]
    tabs = [f.table() for f in fams]
    return P.Fractal.mixed(s, dim, tabs), oracle.MixedFractal(s, len(tabs), dim, tabs), dim


def rule_of(dim):
    return W.MENGER_B5S45 if dim == 3 else W.LIFE_B3S23


def all_coords(side, dim, margin=0):
    ax = np.arange(-margin, side + margin, dtype=np.int64)
    g = np.meshgrid(*([ax] * dim), indexing="ij")
    return np.stack([x.reshape(-1) for x in g[::-1]], axis=1)


@pytest.mark.parametrize("name", sorted(MIXES))
def test_mixed_maps_exhaustive(P, name):
    g, o, dim = pair(P, name)
    assert g.cells == o.cells
    w = torch.arange(g.cells, dtype=torch.int64, device="cuda")
    assert np.array_equal(g.lam(w).cpu().numpy(), o.lam(np.arange(g.cells)))
    c = all_coords(g.side, dim, margin=1)
    ct = torch.from_numpy(c.astype(np.int32)).cuda()
    assert np.array_equal(g.nu(ct).cpu().numpy(), o.nu(c))
    assert np.array_equal(g.nu2d(ct).cpu().numpy(), o.nu2d(c))


@pytest.mark.parametrize("name", sorted(MIXES))
def test_mixed_step_every_tile_depth(P, name):
    g, o, dim = pair(P, name)
    rule = rule_of(dim)
    init = o.init_bernoulli(len(name), 0.45)
    want = o.step(init, rule=oracle.Rule(*rule), steps=4)
    x = torch.from_numpy(init).cuda()
    for L in range(0, g.r + 1):
        g.tile_levels = L
        out = g.step(x, steps=4, rule=rule)
        assert np.array_equal(out.cpu().numpy(), want), f"L={L}"
    rng = np.random.default_rng(3)
    raw = (rng.integers(0, 2, size=g.cells) * rng.integers(1, 256, size=g.cells)).astype(np.uint8)
    g.tile_levels = -1
    assert np.array_equal(g.step(torch.from_numpy(raw).cuda(), steps=1, rule=rule).cpu().numpy(),
                          o.step(raw, rule=oracle.Rule(*rule), steps=1))


@pytest.mark.parametrize("name", sorted(MIXES))
def test_mixed_box_views_and_bb_step(P, name):
    g, o, dim = pair(P, name)
    rule = rule_of(dim)
    init = o.init_bernoulli(7, 0.5)
    x = torch.from_numpy(init).cuda()
    box = g.scatter(x)
    assert np.array_equal(box.cpu().numpy(), o.scatter(init))
    assert np.array_equal(g.gather(box).cpu().numpy(), init)
    rng = np.random.default_rng(5)
    garbage = rng.integers(0, 3, size=g.box_cells).astype(np.uint8)
    bt = torch.from_numpy(garbage).cuda()
    for steps in (0, 1, 3):
        got = g.bb_step(bt, steps=steps, rule=rule)
        assert np.array_equal(got.cpu().numpy(), o.bb_step(garbage, rule=oracle.Rule(*rule), steps=steps)), steps


def test_mixed_many_tiles(P):
    # carpet and Vicsek levels alternating, 2.56e6 cells, thousands of tiles
    fams = [W.CARPET, W.VICSEK] * 4
    tabs = [f.table() for f in fams]
    g, o = P.Fractal.mixed(3, 2, tabs), oracle.MixedFractal(3, 8, 2, tabs)
    init = o.init_bernoulli(11, 0.4)
    want = o.step(init, steps=3)
    for L in (2, 4):
        g.tile_levels = L
        assert np.array_equal(g.step(torch.from_numpy(init).cuda(), steps=3).cpu().numpy(), want), L


def test_mixed_in_a_batch(P):
    g, o, dim = pair(P, "carpet_vicsek_h")
    u = P.Fractal.from_family(W.CARPET, 4)
    ou = oracle.Fractal(8, 3, 4, 2, W.CARPET.table())
    a, b = o.init_bernoulli(21, 0.5), ou.init_bernoulli(22, 0.5)
    xa, xb = torch.from_numpy(a).cuda(), torch.from_numpy(b).cuda()
    ya, yb = torch.empty_like(xa), torch.empty_like(xb)
    batch = P.Batch()
    batch.add(g, xa, ya, 6)
    batch.add(u, xb, yb, 6)
    batch.run()
    torch.cuda.synchronize()
    assert np.array_equal(ya.cpu().numpy(), o.step(a, steps=6))
    assert np.array_equal(yb.cpu().numpy(), ou.step(b, steps=6))
    batch.close()


def test_mixed_refused_where_unsupported(P):
    from paper_2110_12952_gb300.capi import FractalError
    g, _, _ = pair(P, "carpet_vicsek_h")
    w = torch.zeros(4, dtype=torch.int64, device="cuda")
    with pytest.raises(FractalError, match="EINVAL"):
        g.lam_tc(w)
    with pytest.raises(FractalError, match="EINVAL"):
        g.blocked_bytes(1)
    with pytest.raises(FractalError, match="EINVAL"):
        g.set_temporal_blocking(3)
    with pytest.raises(FractalError, match="EINVAL"):
        P.Fractal.mixed(3, 2, [W.CARPET.table(), [[0, 0], [0, 0]]])   # duplicate rows in a level
