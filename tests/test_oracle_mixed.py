"""Pins of the oracle's fractals with a different transition table per level
(``oracle.MixedFractal``; the paper's conclusions propose combining NBB
fractals across scale levels as future work), tied to facts outside it:

* with the same table at every level it is the ordinary fractal, whose own
  oracle is pinned in ``test_oracle_pins.py``;
* closed forms: triangle levels alternating with full-square levels keep the
  cells with no shared 1 bit at the triangle levels; the member count is the
  product of the per-level replica counts;
* lambda is a bijection onto the members, nu inverts it, nu is -1 off the
  fractal and outside the box; the compact coordinate is a bijection onto a
  rectangle whose sides are the products of the per-axis replica counts;
* hand-worked lambda / nu / compact-coordinate values;
* the step: a library convolution on the masked box, the oracle's box step
  and its compact step agree.
"""
import numpy as np
import pytest
from scipy.ndimage import convolve
from scipy.signal import convolve2d

import oracle
from paper_2110_12952_gb300 import workloads as W


def all_coords(side, dim, margin=0):
    ax = np.arange(-margin, side + margin, dtype=np.int64)
    g = np.meshgrid(*([ax] * dim), indexing="ij")
    return np.stack([x.reshape(-1) for x in g[::-1]], axis=1)


def mix(s, dim, fams):
    return oracle.MixedFractal(s, len(fams), dim, [f.table() for f in fams])


#: a 3D table for mixing with the Menger sponge: the 8 corners of the 3^3
#: digit box and its centre
CORNERS3 = W.Family("corners3", 9, 3, 3, tuple((x, y, z) for z in range(3) for y in range(3) for x in range(3)
                                               if (x != 1 and y != 1 and z != 1) or (x, y, z) == (1, 1, 1)))

MIXES = {
    "tri_square": (2, 2, [W.TRIANGLE, W.FULL_SQUARE, W.TRIANGLE, W.TRIANGLE_MIRRORED, W.FULL_SQUARE, W.TRIANGLE]),
    "carpet_vicsek_h": (3, 2, [W.CARPET, W.VICSEK, W.H_FRACTAL, W.CARPET]),
    "vicsek_x_chandelier": (3, 2, [W.VICSEK, W.X_FRACTAL, W.CHANDELIER, W.EMPTY_BOTTLES]),
    "menger_corners_3d": (3, 3, [W.MENGER, CORNERS3]),
}


@pytest.mark.parametrize("fam,r", [(W.TRIANGLE, 6), (W.CARPET, 3), (W.VICSEK, 4), (W.MENGER, 2)],
                         ids=lambda v: getattr(v, "name", str(v)))
def test_same_table_every_level_is_the_fractal(fam, r):
    m = mix(fam.s, fam.dim, [fam] * r)
    f = oracle.Fractal(fam.k, fam.s, r, fam.dim, fam.table())
    assert m.cells == f.cells
    w = np.arange(f.cells)
    assert np.array_equal(m.lam(w), f.lam(w))
    c = all_coords(f.side, fam.dim, margin=1)
    assert np.array_equal(m.nu(c), f.nu(c))
    assert np.array_equal(m.nu2d(c), f.nu2d(c))
    rule = oracle.Rule(*W.default_rule(fam))
    init = f.init_bernoulli(3, 0.5)
    assert np.array_equal(m.step(init, rule=rule, steps=3), f.step(init, rule=rule, steps=3))


@pytest.mark.parametrize("r", range(1, 8))
def test_triangle_and_square_levels_closed_form(r):
    # levels 0, 2, 4, ... the triangle (not both digits 1), levels 1, 3, ...
    # the full square: a member has no 1 bit shared by x and y at an even level
    m = mix(2, 2, [W.TRIANGLE if mu % 2 == 0 else W.FULL_SQUARE for mu in range(r)])
    c = all_coords(2 ** r, 2)
    even = sum(1 << mu for mu in range(0, r, 2))
    want = ((c[:, 0] & c[:, 1] & even) == 0).astype(np.uint8)
    assert np.array_equal(m.member(c), want)
    assert int(want.sum()) == m.cells == 3 ** ((r + 1) // 2) * 4 ** (r // 2)


@pytest.mark.parametrize("name", sorted(MIXES))
def test_count_bijection_and_inverse(name):
    s, dim, fams = MIXES[name]
    m = mix(s, dim, fams)
    assert m.cells == int(np.prod([f.k for f in fams]))
    c = all_coords(m.side, dim)
    member = m.member(c).astype(bool)
    assert int(member.sum()) == m.cells
    w = np.arange(m.cells)
    lam = m.lam(w)
    # lambda: onto exactly the members, one to one
    idx = sum(lam[:, i] * m.side ** i for i in range(dim))
    assert len(np.unique(idx)) == m.cells and member[idx].all()
    assert np.array_equal(m.nu(lam), w)
    nu = m.nu(c)
    assert (nu[~member] == -1).all()
    assert np.array_equal(m.lam(nu[member]), c[member])
    out = all_coords(m.side, dim, margin=1)
    outside = (out < 0).any(axis=1) | (out >= m.side).any(axis=1)
    assert (m.nu(out[outside]) == -1).all()


@pytest.mark.parametrize("name", sorted(MIXES))
def test_compact_coordinate_is_a_rectangle(name):
    s, dim, fams = MIXES[name]
    m = mix(s, dim, fams)
    c2 = m.nu2d(m.lam(np.arange(m.cells)))
    extents = [int(np.prod([f.k for mu, f in enumerate(fams) if mu % dim == a])) for a in range(dim)]
    assert c2.min(axis=0).tolist() == [0] * dim
    assert (c2.max(axis=0) + 1).tolist() == extents
    assert len({tuple(v) for v in c2}) == m.cells == int(np.prod(extents))


def test_hand_worked_values():
    # levels: 0 carpet (k 8), 1 Vicsek (k 5), 2 H-fractal (k 7); s = 3.
    # Replica IDs are row-major (x fastest) within each table:
    #   carpet (2,1) -> 4 (after (0,0),(1,0),(2,0),(0,1)); Vicsek (1,2) -> 4
    #   (its last row); H-fractal (2,0) -> 1 (row 0 holds (0,0) and (2,0)).
    # p = (2 + 3*1 + 9*2, 1 + 3*2 + 9*0) = (23, 7)
    # omega = 4 + 4*8 + 1*(8*5) = 76; compact coordinate: x gets 4 (level 0)
    # + 1*8 (level 2, weight k_0) = 12, y gets 4 (level 1) = 4.
    tabs = [W.CARPET, W.VICSEK, W.H_FRACTAL]
    ids = [{tuple(int(v) for v in row): j for j, row in enumerate(f.table())} for f in tabs]
    assert (ids[0][(2, 1)], ids[1][(1, 2)], ids[2][(2, 0)]) == (4, 4, 1)
    m = mix(3, 2, tabs)
    assert m.nu([[23, 7]]).tolist() == [76]
    assert m.lam([76]).tolist() == [[23, 7]]
    assert m.nu2d([[23, 7]]).tolist() == [[12, 4]]
    # the centre digit (1,1) is not in the carpet: off the fractal at level 0
    assert m.nu([[1 + 3, 1]]).tolist() == [-1]


def life_box(grid, member, birth, survive):
    g = grid.astype(np.int64) * member
    k = np.ones((3,) * g.ndim, dtype=np.int64)
    cnt = (convolve2d(g, k, mode="same") if g.ndim == 2 else convolve(g, k, mode="constant", cval=0)) - g
    new = np.where(g == 1, np.isin(cnt, survive), np.isin(cnt, birth)).astype(np.uint8)
    return new * member


@pytest.mark.parametrize("name", sorted(MIXES))
def test_three_routes_agree(name):
    s, dim, fams = MIXES[name]
    m = mix(s, dim, fams)
    birth, survive = ((5,), (4, 5)) if dim == 3 else ((3,), (2, 3))
    rule = oracle.Rule(list(birth), list(survive))
    shape = (m.side,) * dim
    member = m.member(all_coords(m.side, dim)).reshape(shape[::-1])
    rng = np.random.default_rng(len(name))
    box = (rng.random(shape[::-1]) < 0.45).astype(np.uint8) * member
    compact = m.gather(box.reshape(-1))
    for _ in range(4):
        ref = life_box(box, member, birth, survive)
        bb = m.bb_step(box.reshape(-1), rule=rule).reshape(shape[::-1])
        compact = m.step(compact, rule=rule)
        assert np.array_equal(bb, ref)
        assert np.array_equal(m.scatter(compact).reshape(shape[::-1]), ref)
        box = ref
