"""Pins of the CPU oracle to facts that do not come from the oracle itself.

Each test ties one oracle function to the paper (printed values, equations,
the unfolding of the compact layout), to closed forms (membership predicates,
k^r cells, bijections), to textbook results (Game of Life patterns, a library
convolution) or to published generator outputs.  A plausible mistake in the
oracle (dropped term, wrong sign or index, transposed operand) fails at least
one of them; ``test_oracle_mutants.py`` checks that for a set of planted ones.
"""
import itertools
import math
import os

import numpy as np
import pytest
from scipy.ndimage import convolve
from scipy.signal import convolve2d

import oracle
from paper_2110_12952_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def F(fam, r, lib=None):
    return oracle.Fractal(fam.k, fam.s, r, fam.dim, fam.table(), lib=lib)


def all_coords(side, dim):
    """Every box coordinate (x, y[, z]) in box order, x fastest."""
    idx = np.arange(side ** dim, dtype=np.int64)
    cols = []
    for _ in range(dim):
        cols.append(idx % side)
        idx = idx // side
    return np.stack(cols, axis=1)


def digits(v, s, r):
    return [(v // s**m) % s for m in range(r)]


# ------------------------------------------------------------- membership

@pytest.mark.parametrize("r", range(0, 8))
def test_triangle_membership_closed_form(r):
    f = F(W.TRIANGLE, r)
    c = all_coords(f.side, 2)
    m = f.member(c)
    expect = ((c[:, 0] & c[:, 1]) == 0).astype(np.uint8)
    assert np.array_equal(m, expect)


@pytest.mark.parametrize("r", range(0, 5))
def test_carpet_membership_no_centre_digit(r):
    f = F(W.CARPET, r)
    c = all_coords(f.side, 2)
    m = f.member(c)
    expect = [all(not (dx == 1 and dy == 1) for dx, dy in zip(digits(x, 3, r), digits(y, 3, r)))
              for x, y in c]
    assert np.array_equal(m, np.array(expect, dtype=np.uint8))


@pytest.mark.parametrize("r", range(0, 7))
def test_cantor_set_textbook(r):
    # the Cantor set: x has no base-3 digit 1, on the row y = 0
    f = F(W.CANTOR, r)
    c = all_coords(f.side, 2)
    expect = [y == 0 and all(d != 1 for d in digits(x, 3, r)) for x, y in c]
    assert np.array_equal(f.member(c), np.array(expect, dtype=np.uint8))


@pytest.mark.parametrize("r", range(0, 4))
def test_menger_membership_textbook(r):
    f = F(W.MENGER, r)
    c = all_coords(f.side, 3)
    m = f.member(c)
    # Menger sponge: a cell survives iff no level has two or more middle digits.
    dx = [digits(v, 3, r) for v in range(f.side)]
    expect = [all(((a == 1) + (b == 1) + (cc == 1)) < 2 for a, b, cc in zip(dx[x], dx[y], dx[z]))
              for x, y, z in c]
    assert np.array_equal(m, np.array(expect, dtype=np.uint8))


@pytest.mark.parametrize("fam,rmax", [(W.TRIANGLE, 8), (W.CARPET, 4), (W.VICSEK, 5),
                                      (W.MENGER, 3), (W.FULL_SQUARE, 6)] +
                         [(f, 4) for f in W.TABLE1_EXTRA])
def test_member_count_is_k_pow_r(fam, rmax):
    # Eq. 1: V = k^r
    for r in range(rmax + 1):
        f = F(fam, r)
        assert int(f.member(all_coords(f.side, fam.dim)).sum()) == fam.k ** r


def test_vicsek_symmetries():
    f = F(W.VICSEK, 4)
    c = all_coords(f.side, 2)
    m = f.member(c).reshape(f.side, f.side)  # [y, x]
    assert np.array_equal(m, m.T)
    assert np.array_equal(m, m[:, ::-1])
    assert np.array_equal(m, m[::-1, :])


def test_hausdorff_dimension_table1():
    rows = [l.split() for l in open(os.path.join(GOLDEN, "table1_hausdorff.txt"))
            if l.strip() and not l.startswith("#")]
    table = {name: (int(k), int(s), float(v)) for name, k, s, v in rows}
    for name, (k, s, v) in table.items():
        assert round(math.log(k) / math.log(s), 2) == pytest.approx(v)
    # box-counting dimension of the oracle's fractals equals the table's value
    for fam, name in [(W.TRIANGLE, "sierpinski_gasket"), (W.CARPET, "sierpinski_carpet"),
                      (W.VICSEK, "vicsek"), (W.H_FRACTAL, "h_fractal"), (W.X_FRACTAL, "x_fractal"),
                      (W.CANTOR, "cantor_set"), (W.CHANDELIER, "chandelier"), (W.CANDY, "candy"),
                      (W.EMPTY_BOTTLES, "empty_bottles")]:
        k, s, v = table[name]
        assert (fam.k, fam.s) == (k, s)
        n3 = F(fam, 3).member(all_coords(fam.s ** 3, 2)).sum()
        n4 = F(fam, 4).member(all_coords(fam.s ** 4, 2)).sum()
        assert round(math.log(n4 / n3) / math.log(s), 2) == pytest.approx(v)


def test_compaction_fraction_printed():
    fam, r, frac, tol = open(os.path.join(GOLDEN, "compaction.txt")).read().split("\n")[-2].split()
    r, frac, tol = int(r), float(frac), float(tol)
    # growth factor of the oracle's member count, level by level, is k
    counts = [F(W.TRIANGLE, q).member(all_coords(2 ** q, 2)).sum() for q in range(1, 7)]
    assert all(b == 3 * a for a, b in zip(counts, counts[1:]))
    cells = counts[0] * 3 ** (r - 1)
    assert abs(cells / (2 ** r) ** 2 - frac) < tol


def test_degenerate_levels():
    # r = 0: one cell; k = 1: one cell at every level
    f0 = F(W.CARPET, 0)
    assert f0.cells == 1 and f0.is_member([0, 0]) and f0.nu([[0, 0]])[0] == 0
    one = oracle.Fractal(1, 2, 5, 2, [[0, 0]])
    c = all_coords(32, 2)
    assert one.member(c).sum() == 1 and one.is_member([0, 0])
    assert one.lam([0]).tolist() == [[0, 0]]


# ------------------------------------------------------------- lambda, nu

CASES = [(W.TRIANGLE, 7), (W.CARPET, 3), (W.VICSEK, 4), (W.MENGER, 2), (W.FULL_SQUARE, 4),
         (W.TRIANGLE_MIRRORED, 6), (W.TRIANGLE, 0), (W.MENGER, 0)]


@pytest.mark.parametrize("fam,r", CASES)
def test_lambda_is_bijection_onto_members(fam, r):
    f = F(fam, r)
    p = f.lam(np.arange(f.cells))
    assert len({tuple(x) for x in p}) == f.cells
    assert f.member(p).all()
    # every member is hit: members counted by brute force equal k^r
    assert f.member(all_coords(f.side, fam.dim)).sum() == f.cells


@pytest.mark.parametrize("fam,r", CASES)
def test_nu_inverts_lambda(fam, r):
    f = F(fam, r)
    w = np.arange(f.cells)
    assert np.array_equal(f.nu(f.lam(w)), w)
    c = all_coords(f.side, fam.dim)
    m = f.member(c).astype(bool)
    nu = f.nu(c)
    assert (nu[~m] == -1).all()
    assert np.array_equal(f.lam(nu[m]), c[m])


@pytest.mark.parametrize("fam,r", [(W.TRIANGLE, 5), (W.MENGER, 2), (W.CARPET, 2)])
def test_nu_outside_box(fam, r):
    f = F(fam, r)
    n = f.side
    pts = []
    for d in range(fam.dim):
        for v in (-1, n, -n, 2 * n):
            q = [0] * fam.dim
            q[d] = v
            pts.append(q)
    assert (f.nu(pts) == -1).all()
    assert not f.member(pts).any()


def test_lambda_place_value_levels():
    # omega = j * k^mu has digit j at level mu and digit 0 elsewhere, so it
    # lands at s^mu * off[j] + sum over the other levels nu of s^nu * off[0]
    for fam, r in [(W.TRIANGLE, 9), (W.CARPET, 5), (W.MENGER, 3), (W.VICSEK, 6)]:
        f = F(fam, r)
        for mu in range(r):
            for j in range(fam.k):
                p = f.lam([j * fam.k ** mu])[0]
                expect = [fam.s ** mu * v + sum(fam.s ** q for q in range(r) if q != mu) * v0
                          for v, v0 in zip(fam.offsets[j], fam.offsets[0])]
                assert p.tolist() == expect


def _paper_H(x, y, mu):
    # Eq. 2, procedural replica ID of the paper
    return (x % 2 ** (mu + 1)) // 2 ** mu + (y % 2 ** (mu + 1)) // 2 ** mu


def test_nu_matches_paper_eq2_for_mirrored_triangle():
    # For the table (0,0),(1,0),(1,1) the inverse transition ID is exactly
    # Eq. 2's bit_x + bit_y, and nu is the base-k sum of those IDs.
    r = 7
    f = F(W.TRIANGLE_MIRRORED, r)
    c = all_coords(f.side, 2)
    nu = f.nu(c)
    for (x, y), w in zip(c, nu):
        member = (y & ~x) == 0
        if member:
            assert w == sum(_paper_H(x, y, mu) * 3 ** mu for mu in range(r))
        else:
            assert w == -1


@pytest.mark.parametrize("r", range(1, 8))
def test_nu2d_is_paper_eqs_6_8(r):
    # Eqs. 6-8 with Eq. 2 as H (mirrored triangle), tau_x = k^(mu/2) on even
    # levels and tau_y = k^((mu-1)/2) on odd levels.
    f = F(W.TRIANGLE_MIRRORED, r)
    c = all_coords(f.side, 2)
    m = f.member(c).astype(bool)
    got = f.nu2d(c[m])
    for (x, y), (cx, cy) in zip(c[m], got):
        ex = sum(3 ** (mu // 2) * ((mu + 1) % 2) * _paper_H(x, y, mu) for mu in range(r))
        ey = sum(3 ** (mu // 2) * (mu % 2) * _paper_H(x, y, mu) for mu in range(r))
        assert (cx, cy) == (ex, ey)


@pytest.mark.parametrize("fam,rmax", [(W.TRIANGLE, 8), (W.CARPET, 4), (W.VICSEK, 5)])
def test_nu2d_unfolding(fam, rmax):
    # Sec. 3 / compact-form figure: the compact layout of level r is k copies
    # of level r-1, side by side to the right when r is odd and stacked down
    # when r is even; its size is k^ceil(r/2) x k^floor(r/2).
    prev = {(0, 0)}
    for r in range(1, rmax + 1):
        f = F(fam, r)
        w = np.arange(f.cells)
        c2 = f.nu2d(f.lam(w))
        width, height = fam.k ** ((r + 1) // 2), fam.k ** (r // 2)
        assert c2[:, 0].min() == 0 and c2[:, 0].max() == width - 1
        assert c2[:, 1].min() == 0 and c2[:, 1].max() == height - 1
        assert len({tuple(v) for v in c2}) == width * height == f.cells
        pw, ph = fam.k ** (r // 2), fam.k ** ((r - 1) // 2)
        top = w // fam.k ** (r - 1)
        for j in range(fam.k):
            sub = {tuple(v) for v in c2[top == j]}
            shift = (j * pw, 0) if r % 2 == 1 else (0, j * ph)
            assert sub == {(a + shift[0], b + shift[1]) for a, b in prev}
        # the copy of level r-1 keeps its own layout: digits below the top one
        prev = {tuple(v) for v in c2}


def test_nu2d_3d_cycles_axes():
    f = F(W.MENGER, 3)
    c2 = f.nu2d(f.lam(np.arange(f.cells)))
    assert c2.max(axis=0).tolist() == [19, 19, 19]
    assert len({tuple(v) for v in c2}) == f.cells


def test_nu2d_3d_hand_worked():
    # reading O6 (axes cycle x, y, z; level mu adds H_mu * k^floor(mu/3) to
    # axis mu mod 3), worked by hand for the Menger sponge.  Its replica IDs
    # (row-major, x fastest, tuples with at most one digit 1): (2,0,0) -> 2,
    # (0,2,1) -> 10, (1,0,2) -> 13, (2,2,2) -> 19, (0,1,0) -> 3, (2,1,2) -> 16.
    # Levels 0..5 take these tuples in that order, so p = sum_mu 3^mu t_mu:
    #   x = 2 + 0*3 + 1*9 + 2*27 + 0*81 + 2*243 = 551
    #   y = 0 + 2*3 + 0*9 + 2*27 + 1*81 + 1*243 = 384
    #   z = 0 + 1*3 + 2*9 + 2*27 + 0*81 + 2*243 = 561
    # compact coordinate: x gets 2 (mu 0) + 19*20 (mu 3) = 382, y gets 10
    # (mu 1) + 3*20 (mu 4) = 70, z gets 13 (mu 2) + 16*20 (mu 5) = 333;
    # omega = 2 + 10*20 + 13*20^2 + 19*20^3 + 3*20^4 + 16*20^5.
    tab = {tuple(int(v) for v in row): j for j, row in enumerate(W.MENGER.table())}
    assert [tab[t] for t in [(2, 0, 0), (0, 2, 1), (1, 0, 2), (2, 2, 2), (0, 1, 0), (2, 1, 2)]] == \
        [2, 10, 13, 19, 3, 16]
    f6 = F(W.MENGER, 6)
    assert f6.nu2d([[551, 384, 561]]).tolist() == [[382, 70, 333]]
    w = 2 + 10 * 20 + 13 * 400 + 19 * 8000 + 3 * 160000 + 16 * 3200000
    assert f6.nu([[551, 384, 561]]).tolist() == [w]
    assert f6.lam([w]).tolist() == [[551, 384, 561]]
    # the first four levels alone (r = 4): x 65, y 60, z 75 -> (382, 10, 13)
    f4 = F(W.MENGER, 4)
    assert f4.nu2d([[65, 60, 75]]).tolist() == [[382, 10, 13]]


# ---------------------------------------------------------------- stepping

def life_box(grid, member=None, birth=(3,), survive=(2, 3)):
    """Textbook synchronous life-like update via a library convolution, with
    an optional membership mask (cells off the mask are dead)."""
    g = grid.astype(np.int64)
    if member is not None:
        g = g * member
    if g.ndim == 2:
        cnt = convolve2d(g, np.ones((3, 3), dtype=np.int64), mode="same") - g
    else:
        cnt = convolve(g, np.ones((3, 3, 3), dtype=np.int64), mode="constant", cval=0) - g
    new = np.where(g == 1, np.isin(cnt, survive), np.isin(cnt, birth)).astype(np.uint8)
    if member is not None:
        new = new * member.astype(np.uint8)
    return new


def read_patterns():
    lines = open(os.path.join(GOLDEN, "life_patterns.txt")).read().split("\n")
    out, i = [], 0
    while i < len(lines):
        if lines[i].startswith("pattern"):
            _, name, steps = lines[i].split()
            i += 2
            before = []
            while lines[i] != "after":
                before.append(lines[i])
                i += 1
            i += 1
            after = []
            while lines[i] != "end":
                after.append(lines[i])
                i += 1
            g = lambda rows: np.array([[ch == "#" for ch in row] for row in rows], dtype=np.uint8)
            out.append((name, int(steps), g(before), g(after)))
        i += 1
    return out


@pytest.mark.parametrize("name,steps,before,after", read_patterns())
def test_full_square_is_textbook_life(name, steps, before, after):
    # k = s^d: the compact step is plain Life on an n x n grid, dead border.
    r = 3
    f = F(W.FULL_SQUARE, r)
    box = np.zeros((8, 8), dtype=np.uint8)
    h, w = before.shape
    box[:h, :w] = before
    compact = f.gather(box.reshape(-1))
    out = f.scatter(f.step(compact, steps=steps)).reshape(8, 8)
    expect = np.zeros((8, 8), dtype=np.uint8)
    expect[:h, :w] = after
    assert np.array_equal(out, expect)
    bb = f.bb_step(box.reshape(-1), steps=steps).reshape(8, 8)
    assert np.array_equal(bb, expect)


def test_full_square_random_vs_convolution():
    f = F(W.FULL_SQUARE, 5)
    rng = np.random.default_rng(11)
    box = (rng.random((32, 32)) < 0.4).astype(np.uint8)
    compact = f.gather(box.reshape(-1))
    for _ in range(6):
        box = life_box(box)
        compact = f.step(compact)
        assert np.array_equal(f.scatter(compact).reshape(32, 32), box)


@pytest.mark.parametrize("fam,r", [(W.TRIANGLE, 6), (W.CARPET, 3), (W.VICSEK, 4),
                                   (W.TRIANGLE_MIRRORED, 5), (W.TRIANGLE, 1)] +
                         [(f, 3) for f in W.TABLE1_EXTRA])
def test_three_routes_agree_2d(fam, r):
    # (i) library convolution on the masked box, (ii) oracle BB step,
    # (iii) oracle compact step through lambda/nu.
    f = F(fam, r)
    n = f.side
    member = f.member(all_coords(n, 2)).reshape(n, n)
    rng = np.random.default_rng(r * 31 + fam.k)
    box = (rng.random((n, n)) < 0.45).astype(np.uint8) * member
    compact = f.gather(box.reshape(-1))
    for _ in range(5):
        ref = life_box(box, member)
        bb = f.bb_step(box.reshape(-1)).reshape(n, n)
        compact = f.step(compact)
        assert np.array_equal(bb, ref)
        assert np.array_equal(f.scatter(compact).reshape(n, n), ref)
        box = ref


def test_three_routes_agree_menger():
    fam, r = W.MENGER, 2
    f = F(fam, r)
    n = f.side
    member = f.member(all_coords(n, 3)).reshape(n, n, n)
    rng = np.random.default_rng(5)
    box = (rng.random((n, n, n)) < 0.5).astype(np.uint8) * member
    compact = f.gather(box.reshape(-1))
    rule = oracle.MENGER_RULE
    for _ in range(4):
        ref = life_box(box, member, birth=(5,), survive=(4, 5))
        bb = f.bb_step(box.reshape(-1), rule=rule).reshape(n, n, n)
        compact = f.step(compact, rule=rule)
        assert np.array_equal(bb, ref)
        assert np.array_equal(f.scatter(compact).reshape(n, n, n), ref)
        box = ref


def test_bb_masks_garbage_off_fractal():
    f = F(W.TRIANGLE, 5)
    n = f.side
    member = f.member(all_coords(n, 2)).reshape(n, n)
    rng = np.random.default_rng(3)
    box = rng.integers(0, 256, size=(n, n)).astype(np.uint8)
    out = f.bb_step(box.reshape(-1)).reshape(n, n)
    assert (out[member == 0] == 0).all()
    ref = life_box((box != 0).astype(np.uint8), member)
    assert np.array_equal(out, ref)


def test_invariants():
    f = F(W.CARPET, 3)
    z = np.zeros(f.cells, dtype=np.uint8)
    assert not f.step(z, steps=3).any()
    one = z.copy()
    one[f.cells // 2] = 1
    assert not f.step(one).any()  # a lone cell dies under B3/S23
    # nonzero bytes count as alive, output is exactly 0/1
    rng = np.random.default_rng(9)
    raw = rng.integers(0, 256, size=f.cells).astype(np.uint8)
    a = f.step(raw)
    b = f.step((raw != 0).astype(np.uint8))
    assert np.array_equal(a, b) and set(np.unique(a)) <= {0, 1}
    assert np.array_equal(f.step(raw, steps=0), (raw != 0).astype(np.uint8))


def test_step_range_and_cells_match_full_step():
    f = F(W.VICSEK, 5)
    st = f.init_bernoulli(17, 0.5)
    full = f.step(st)
    part = f.step_range(st, 100, 2000)
    assert np.array_equal(part[100:2000], full[100:2000])
    w = W.sample_omegas(f.cells, 200, 4)
    assert np.array_equal(f.step_cells(st, w), full[w])


@pytest.mark.parametrize("t", [1, 2, 3])
def test_cells_after_recursive_definition(t):
    f = F(W.TRIANGLE, 6)
    st = f.init_bernoulli(23, 0.4)
    w = W.sample_omegas(f.cells, 60, t)
    assert np.array_equal(f.cells_after(st, w, t), f.step(st, steps=t)[w])


# ----------------------------------------------------------- seeded inputs

def test_splitmix64_published_outputs():
    rows = [l.split() for l in open(os.path.join(GOLDEN, "splitmix64.txt"))
            if l.strip() and not l.startswith("#")]
    for seed, i, v in rows:
        assert oracle.splitmix64_nth(int(seed), int(i)) == int(v)


def test_bernoulli_init_definition():
    f = F(W.TRIANGLE, 9)
    for p in (0.0, 0.3, 0.5, 1.0):
        st = f.init_bernoulli(1234567, p)
        thr = math.floor(p * 2 ** 53)
        for w in (0, 1, 2, 3, 4, 777):
            assert st[w] == int((oracle.splitmix64_nth(1234567, w) >> 11) < thr)
        frac = st.mean()
        sigma = math.sqrt(max(p * (1 - p), 1e-12) / f.cells)
        assert abs(frac - p) <= 6 * sigma + 1e-12
    st = f.init_bernoulli(5, 0.5, w0=100, w1=200)
    assert not st[:100].any() and not st[200:].any() and st[100:200].any()
