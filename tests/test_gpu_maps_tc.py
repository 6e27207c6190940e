"""The tensor-core maps (fractal_lambda_tc, fractal_nu_tc) against the oracle
and the CUDA-core maps: exhaustively at small levels (every omega, every box
coordinate with a margin outside the box), and on seeded samples plus every
single-nonzero-digit omega at the full workload sizes, where the level
weights are far above 2048 (3^19 for the triangle at r = 20, 8^9 for the
carpet at r = 10), the range in which fp16 alone is not exact."""
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


def all_coords(side, dim, margin):
    ax = np.arange(-margin, side + margin, dtype=np.int64)
    g = np.meshgrid(*([ax] * dim), indexing="ij")
    return np.stack([x.reshape(-1) for x in g[::-1]], axis=1)


def boundary_omegas(k, r):
    out = [0, k ** r - 1]
    for mu in range(r):
        for j in range(1, k):
            out += [j * k ** mu, k ** r - 1 - j * k ** mu]
    return np.unique(np.array(out, dtype=np.int64))


@pytest.mark.parametrize("fam,r", [(W.TRIANGLE, 7), (W.CARPET, 4), (W.VICSEK, 4), (W.MENGER, 3),
                                   (W.H_FRACTAL, 4), (W.CANDY, 3), (W.TRIANGLE, 0), (W.TRIANGLE, 1)],
                         ids=lambda v: getattr(v, "name", str(v)))
def test_tc_maps_exhaustive(P, fam, r):
    g, o = P.Fractal.from_family(fam, r), ora(fam, r)
    w = torch.arange(-2, g.cells + 3, dtype=torch.int64, device="cuda")
    lam = g.lam_tc(w).cpu().numpy()
    wn = w.cpu().numpy()
    inside = (wn >= 0) & (wn < g.cells)
    assert np.array_equal(lam[inside], o.lam(wn[inside]))
    assert (lam[~inside] == -1).all()
    c = all_coords(g.side, fam.dim, margin=2)
    ct = torch.from_numpy(c.astype(np.int32)).cuda()
    om, c2 = g.nu_tc(ct, compact=True)
    assert np.array_equal(om.cpu().numpy(), o.nu(c))
    assert np.array_equal(c2.cpu().numpy(), o.nu2d(c))


@pytest.mark.parametrize("fam,r", [(W.TRIANGLE, 20), (W.TRIANGLE, 16), (W.CARPET, 10), (W.VICSEK, 12),
                                   (W.MENGER, 6)], ids=lambda v: getattr(v, "name", str(v)))
def test_tc_maps_full_size_weights_above_2048(P, fam, r):
    g, o = P.Fractal.from_family(fam, r), ora(fam, r)
    assert fam.k ** (r - 1) > 2048
    w = np.concatenate([boundary_omegas(fam.k, r), W.sample_omegas(g.cells, 300_000, 31 + r)])
    wt = torch.from_numpy(w).cuda()
    lam = g.lam_tc(wt)
    ref = o.lam(w)
    assert np.array_equal(lam.cpu().numpy(), ref)
    assert torch.equal(lam, g.lam(wt))
    c = np.concatenate([ref, W.sample_coords(g.side, fam.dim, 300_000, 41 + r, margin=1)])
    ct = torch.from_numpy(c.astype(np.int32)).cuda()
    om, c2 = g.nu_tc(ct, compact=True)
    assert np.array_equal(om.cpu().numpy(), o.nu(c))
    assert np.array_equal(c2.cpu().numpy(), o.nu2d(c))
    assert torch.equal(om, g.nu(ct)) and torch.equal(c2, g.nu2d(ct))


def test_tc_maps_limits(P):
    from paper_2110_12952_gb300.capi import FractalError
    # a 3D fractal with s = 2 at r = 22: dim * r = 66 levels x axes > 64
    cube = [(x, y, z) for z in range(2) for y in range(2) for x in range(2) if x + y + z != 3]
    g = P.Fractal(len(cube), 2, 22, 3, cube)
    with pytest.raises(FractalError, match="EINVAL"):
        g.lam_tc(torch.zeros(4, dtype=torch.int64, device="cuda"))
    empty = torch.zeros(0, dtype=torch.int64, device="cuda")
    assert g.lam(empty).shape == (0, 3)
