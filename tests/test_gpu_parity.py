"""GPU path (through the C ABI) against the CPU oracle, element by element.

All of this is integer work, so the bar is bit-exact equality everywhere.
Small levels are compared exhaustively (every omega, every box coordinate,
every output cell, several tile depths, so that tiles, halos and ragged
tails are all exercised); the full-size workloads are compared on seeded
samples the oracle computes one by one, after one and after several
generations, in the launch configuration the benchmark times.
"""
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


def gpu_fr(P, fam, r):
    return P.Fractal.from_family(fam, r)


def ora(fam, r):
    return oracle.Fractal(fam.k, fam.s, r, fam.dim, fam.table())


def all_coords(side, dim, margin=0):
    lo, hi = -margin, side + margin
    ax = np.arange(lo, hi, dtype=np.int64)
    g = np.meshgrid(*([ax] * dim), indexing="ij")
    return np.stack([x.reshape(-1) for x in g[::-1]], axis=1)


def rule_of(fam):
    return W.default_rule(fam)


def oracle_rule(fam):
    b, s = rule_of(fam)
    return oracle.Rule(b, s)


SMALL = [(W.TRIANGLE, 7), (W.CARPET, 4), (W.VICSEK, 4), (W.MENGER, 3), (W.FULL_SQUARE, 5),
         (W.TRIANGLE_MIRRORED, 6), (W.TRIANGLE, 0), (W.TRIANGLE, 1), (W.MENGER, 1)]


# --------------------------------------------------------------------- maps

@pytest.mark.parametrize("fam,r", SMALL)
def test_maps_exhaustive(P, fam, r):
    g, o = gpu_fr(P, fam, r), ora(fam, r)
    w = torch.arange(g.cells, dtype=torch.int64, device="cuda")
    lam = g.lam(w).cpu().numpy()
    assert np.array_equal(lam, o.lam(np.arange(g.cells)))
    c = all_coords(g.side, fam.dim, margin=2)
    ct = torch.from_numpy(c.astype(np.int32)).cuda()
    assert np.array_equal(g.nu(ct).cpu().numpy(), o.nu(c))
    assert np.array_equal(g.nu2d(ct).cpu().numpy(), o.nu2d(c))


def test_lambda_out_of_range(P):
    g = gpu_fr(P, W.TRIANGLE, 5)
    w = torch.tensor([-1, g.cells, g.cells - 1], dtype=torch.int64, device="cuda")
    out = g.lam(w).cpu().numpy()
    assert (out[:2] == -1).all() and (out[2] >= 0).all()


FULL = [(W.TRIANGLE, 16), (W.TRIANGLE, 20), (W.CARPET, 10), (W.VICSEK, 12), (W.MENGER, 6)]


def boundary_omegas(k, r):
    out = [0, k ** r - 1]
    for mu in range(r):
        for j in range(1, k):
            out.append(j * k ** mu)
            out.append(k ** r - 1 - j * k ** mu)
    return np.unique(np.array(out, dtype=np.int64))


@pytest.mark.parametrize("fam,r", FULL)
def test_maps_sampled_full_size(P, fam, r):
    g, o = gpu_fr(P, fam, r), ora(fam, r)
    w = np.concatenate([boundary_omegas(fam.k, r), W.sample_omegas(g.cells, 200_000, 101 + r)])
    lam = g.lam(torch.from_numpy(w).cuda()).cpu().numpy()
    ref = o.lam(w)
    assert np.array_equal(lam, ref)
    c = np.concatenate([ref, W.sample_coords(g.side, fam.dim, 200_000, 202 + r, margin=1)])
    ct = torch.from_numpy(c.astype(np.int32)).cuda()
    assert np.array_equal(g.nu(ct).cpu().numpy(), o.nu(c))
    assert np.array_equal(g.nu2d(ct).cpu().numpy(), o.nu2d(c))


# -------------------------------------------------------------------- init

@pytest.mark.parametrize("p", [0.0, 0.3, 0.5, 1.0])
def test_init_bernoulli(P, p):
    g, o = gpu_fr(P, W.CARPET, 5), ora(W.CARPET, 5)
    # offset views exercise the unaligned head/tail of the vectorised writer
    buf = torch.zeros(g.cells + 7, dtype=torch.uint8, device="cuda")
    for off in (0, 3):
        st = buf[off:off + g.cells]
        g.init_bernoulli(99, p, out=st)
        assert np.array_equal(st.cpu().numpy(), o.init_bernoulli(99, p))


def test_init_full_size_sampled(P):
    inst = W.TRI_R20
    g = gpu_fr(P, inst.family, inst.r)
    st = g.init_bernoulli(inst.seed, inst.p)
    o = ora(inst.family, inst.r)
    ref = np.zeros(g.cells, dtype=np.uint8)
    n = 4_000_000
    o.init_bernoulli(inst.seed, inst.p, 0, n, out=ref)
    o.init_bernoulli(inst.seed, inst.p, g.cells - n, g.cells, out=ref)
    assert np.array_equal(st[:n].cpu().numpy(), ref[:n])
    assert np.array_equal(st[-n:].cpu().numpy(), ref[-n:])
    del st
    torch.cuda.empty_cache()


# ------------------------------------------------------------------- steps

@pytest.mark.parametrize("fam,r,levels", [
    (W.TRIANGLE, 6, [0, 1, 2, 3, 5, 6]), (W.CARPET, 4, [0, 1, 2, 3, 4]),
    (W.VICSEK, 5, [0, 2, 4, 5]), (W.MENGER, 3, [0, 1, 2, 3]), (W.FULL_SQUARE, 5, [0, 2, 5]),
    (W.TRIANGLE_MIRRORED, 7, [3, 7]), (W.TRIANGLE, 0, [0]), (W.MENGER, 1, [0, 1])])
def test_step_exhaustive_all_tile_depths(P, fam, r, levels):
    g, o = gpu_fr(P, fam, r), ora(fam, r)
    init = o.init_bernoulli(1000 + r, 0.45)
    ref = o.step(init, rule=oracle_rule(fam), steps=3)
    x = torch.from_numpy(init).cuda()
    for L in levels:
        g.tile_levels = L
        assert g.tile_levels == L
        out = g.step(x, steps=3, rule=rule_of(fam))
        assert np.array_equal(out.cpu().numpy(), ref), f"L={L}"


@pytest.mark.parametrize("fam,r", [(W.H_FRACTAL, 4), (W.X_FRACTAL, 4), (W.CANTOR, 6), (W.CHANDELIER, 5),
                                   (W.CANDY, 3), (W.EMPTY_BOTTLES, 4)], ids=lambda v: getattr(v, "name", str(v)))
def test_table1_fractals_every_tile_depth(P, fam, r):
    # the further Table 1 fractals run through the generic group and cell
    # policies (s = 3 or 4, k = 2 .. 12): every tile depth, three generations
    from paper_2110_12952_gb300.capi import FractalError
    g, o = gpu_fr(P, fam, r), ora(fam, r)
    init = o.init_bernoulli(500 + fam.k, 0.5)
    ref = o.step(init, rule=oracle_rule(fam), steps=3)
    x = torch.from_numpy(init).cuda()
    for L in range(0, r + 1):
        g.tile_levels = L
        if (fam.s ** L + 2) ** 2 > 100_000:
            # a sparse fractal's tile box outgrows shared memory: refused
            with pytest.raises(FractalError, match="does not fit"):
                g.step(x, steps=3, rule=rule_of(fam))
            continue
        out = g.step(x, steps=3, rule=rule_of(fam))
        assert np.array_equal(out.cpu().numpy(), ref), f"L={L}"


@pytest.mark.parametrize("fam,r,L", [(W.H_FRACTAL, 7, 3), (W.CANDY, 6, 3)], ids=lambda v: getattr(v, "name", str(v)))
def test_table1_fractals_many_tiles(P, fam, r, L):
    g, o = gpu_fr(P, fam, r), ora(fam, r)
    init = o.init_bernoulli(600 + fam.k, 0.4)
    g.tile_levels = L
    out = g.step(torch.from_numpy(init).cuda(), steps=2, rule=rule_of(fam))
    assert np.array_equal(out.cpu().numpy(), o.step(init, rule=oracle_rule(fam), steps=2))


@pytest.mark.parametrize("L", [2, 3, 4, 5, 6, 7, 8, 9])
def test_triangle_many_tiles_per_cta(P, L):
    # r = 14 gives thousands of tiles at every depth, so each CTA reuses its
    # pipeline stages many times
    fam, r = W.TRIANGLE, 14
    g, o = gpu_fr(P, fam, r), ora(fam, r)
    init = o.init_bernoulli(8, 0.4)
    x = torch.from_numpy(init).cuda()
    g.tile_levels = L
    assert np.array_equal(g.step(x, steps=2).cpu().numpy(), o.step(init, steps=2)), f"L={L}"


@pytest.mark.parametrize("fam,r,L", [(W.TRIANGLE, 12, L) for L in range(2, 10)] +
                         [(W.CARPET, 6, L) for L in range(1, 6)] + [(W.VICSEK, 7, L) for L in range(1, 6)] +
                         [(W.MENGER, 4, L) for L in range(0, 4)])
def test_nonbinary_input_every_depth(P, fam, r, L):
    # any nonzero byte is alive: the first generation must read 0..255 as
    # 0/1 wherever a cell is read (own cells, taps, frames, halo)
    g, o = gpu_fr(P, fam, r), ora(fam, r)
    rng = np.random.default_rng(100 + L)
    raw = (rng.integers(0, 2, size=g.cells) * rng.integers(1, 256, size=g.cells)).astype(np.uint8)
    g.tile_levels = L
    out = g.step(torch.from_numpy(raw).cuda(), steps=1, rule=rule_of(fam))
    assert np.array_equal(out.cpu().numpy(), o.step(raw, rule=oracle_rule(fam), steps=1)), f"L={L}"


@pytest.mark.parametrize("fam,r,L", [(W.CARPET, 8, L) for L in (2, 3, 4, 5)] +
                         [(W.VICSEK, 9, L) for L in (2, 3, 4, 5, 6)] + [(W.VICSEK, 10, 6)] +
                         [(W.MENGER, 5, L) for L in (2, 3)])
def test_rows_and_lid_policies_many_tiles_per_cta(P, fam, r, L):
    # thousands of tiles per launch: every CTA reuses its stages many times
    g, o = gpu_fr(P, fam, r), ora(fam, r)
    init = o.init_bernoulli(9, 0.5)
    g.tile_levels = L
    steps = 2 if fam.dim == 3 else 3
    out = g.step(torch.from_numpy(init).cuda(), steps=steps, rule=rule_of(fam))
    assert np.array_equal(out.cpu().numpy(), o.step(init, rule=oracle_rule(fam), steps=steps)), f"L={L}"


def test_autotune_keeps_parity(P):
    fam, r = W.TRIANGLE, 11
    g, o = gpu_fr(P, fam, r), ora(fam, r)
    init = o.init_bernoulli(31, 0.4)
    x = torch.from_numpy(init).cuda()
    scratch = torch.empty_like(x)
    L = g.autotune(x, scratch)
    assert 0 <= L <= r and g.tile_levels == L
    assert np.array_equal(x.cpu().numpy(), init)
    assert np.array_equal(g.step(x, steps=3).cpu().numpy(), o.step(init, steps=3))
    # a new handle of the same fractal starts from the tuned depth
    assert gpu_fr(P, fam, r).tile_levels == L


def test_handles_with_different_tiles_interleaved(P):
    # the kernel's shared-memory limit is per function: a handle planned later
    # with a smaller tile must not break an earlier handle's larger plan
    big, small = gpu_fr(P, W.CARPET, 6), gpu_fr(P, W.CARPET, 2)
    ob, osm = ora(W.CARPET, 6), ora(W.CARPET, 2)
    ib, ism = ob.init_bernoulli(3, 0.5), osm.init_bernoulli(4, 0.5)
    xb, xs = torch.from_numpy(ib).cuda(), torch.from_numpy(ism).cuda()
    assert big.tile_levels > small.tile_levels
    for _ in range(2):
        assert np.array_equal(big.step(xb, steps=2).cpu().numpy(), ob.step(ib, steps=2))
        assert np.array_equal(small.step(xs, steps=2).cpu().numpy(), osm.step(ism, steps=2))


@pytest.mark.parametrize("steps", [0, 1, 2, 3, 4])
def test_step_ping_pong_counts(P, steps):
    fam, r = W.VICSEK, 5
    g, o = gpu_fr(P, fam, r), ora(fam, r)
    rng = np.random.default_rng(steps)
    raw = rng.integers(0, 256, size=g.cells).astype(np.uint8)  # nonzero bytes are alive
    x = torch.from_numpy(raw).cuda()
    out = g.step(x, steps=steps)
    assert np.array_equal(out.cpu().numpy(), o.step(raw, steps=steps))
    assert np.array_equal(x.cpu().numpy(), raw)  # input never written


def test_config1_triangle_r8_compact_and_bb(P):
    inst = W.TRI_R8
    fam, r = inst.family, inst.r
    g, o = gpu_fr(P, fam, r), ora(fam, r)
    st = g.init_bernoulli(inst.seed, inst.p)
    init = o.init_bernoulli(inst.seed, inst.p)
    assert np.array_equal(st.cpu().numpy(), init)
    ref = o.step(init, steps=inst.steps)
    out = g.step(st, steps=inst.steps)
    assert np.array_equal(out.cpu().numpy(), ref)
    box = g.scatter(st)
    assert np.array_equal(box.cpu().numpy(), o.scatter(init))
    bb = g.bb_step(box, steps=inst.steps)
    ref_box = o.bb_step(o.scatter(init), steps=inst.steps)
    assert np.array_equal(bb.cpu().numpy(), ref_box)
    assert np.array_equal(g.gather(bb).cpu().numpy(), ref)


@pytest.mark.parametrize("fam,r", [(W.TRIANGLE, 6), (W.CARPET, 3), (W.VICSEK, 4), (W.MENGER, 2),
                                   (W.TRIANGLE, 0), (W.FULL_SQUARE, 4)])
def test_bb_exhaustive_with_garbage(P, fam, r):
    g, o = gpu_fr(P, fam, r), ora(fam, r)
    rng = np.random.default_rng(r + 7)
    box = rng.integers(0, 4, size=g.box_cells).astype(np.uint8)  # garbage off the fractal too
    b = torch.from_numpy(box).cuda()
    for steps in (0, 1, 2, 5):
        out = g.bb_step(b, steps=steps, rule=rule_of(fam))
        assert np.array_equal(out.cpu().numpy(), o.bb_step(box, rule=oracle_rule(fam), steps=steps))


@pytest.mark.parametrize("fam,r", [(W.TRIANGLE, 10), (W.TRIANGLE_MIRRORED, 9), (W.FULL_SQUARE, 9)])
def test_bb_bits_path_s2_with_garbage(P, fam, r):
    # s = 2 boxes (16-byte aligned rows) take the bit-sliced row path
    g, o = gpu_fr(P, fam, r), ora(fam, r)
    rng = np.random.default_rng(r)
    box = rng.integers(0, 3, size=g.box_cells).astype(np.uint8) * rng.integers(1, 200, size=g.box_cells).astype(np.uint8)
    b = torch.from_numpy(box).cuda()
    for steps in (1, 2):
        out = g.bb_step(b, steps=steps)
        assert np.array_equal(out.cpu().numpy(), o.bb_step(box, steps=steps)), steps


@pytest.mark.parametrize("fam,r", [(W.CARPET, 5), (W.CARPET, 6), (W.VICSEK, 6), (W.H_FRACTAL, 5), (W.X_FRACTAL, 6),
                                   (W.TRIANGLE, 7), (W.TRIANGLE_MIRRORED, 8)],
                         ids=lambda v: getattr(v, "name", str(v)))
def test_bb_bits_path_with_garbage(P, fam, r):
    # 2D boxes of side >= 32, rows not 16-byte aligned, take the bit-sliced
    # row path; garbage and non-binary bytes off the fractal
    g, o = gpu_fr(P, fam, r), ora(fam, r)
    rng = np.random.default_rng(100 + r)
    box = rng.integers(0, 3, size=g.box_cells).astype(np.uint8) * rng.integers(1, 200, size=g.box_cells).astype(np.uint8)
    b = torch.from_numpy(box).cuda()
    for steps in (1, 2, 3):
        out = g.bb_step(b, steps=steps, rule=rule_of(fam))
        assert np.array_equal(out.cpu().numpy(), o.bb_step(box, rule=oracle_rule(fam), steps=steps)), steps
    # buffers at unaligned addresses take the generic kernel, with the same result
    base = torch.zeros(g.box_cells + 16, dtype=torch.uint8, device="cuda")
    x = base[3:3 + g.box_cells]
    x.copy_(b)
    assert np.array_equal(g.bb_step(x, steps=1, rule=rule_of(fam)).cpu().numpy(),
                          o.bb_step(box, rule=oracle_rule(fam), steps=1))


@pytest.mark.parametrize("rule", [W.MENGER_B5S45, (0x6, 0x1E)], ids=lambda r: f"B{r[0]:x}S{r[1]:x}")
def test_bb_bits3_path_menger_r5_with_garbage(P, rule):
    # 3D boxes of side >= 32 take the plane-walking bit-sliced row path
    g, o = gpu_fr(P, W.MENGER, 5), ora(W.MENGER, 5)
    rng = np.random.default_rng(55)
    box = rng.integers(0, 3, size=g.box_cells).astype(np.uint8) * rng.integers(1, 200, size=g.box_cells).astype(np.uint8)
    b = torch.from_numpy(box).cuda()
    orl = oracle.Rule([i for i in range(27) if (rule[0] >> i) & 1], [i for i in range(27) if (rule[1] >> i) & 1])
    for steps in (1, 2):
        out = g.bb_step(b, steps=steps, rule=rule)
        assert np.array_equal(out.cpu().numpy(), o.bb_step(box, rule=orl, steps=steps)), steps


def test_bb_bits3_path_menger_r6_against_compact(P):
    g, o = gpu_fr(P, W.MENGER, 6), ora(W.MENGER, 6)
    x = g.init_bernoulli(6, 0.5)
    init = x.cpu().numpy()
    out = g.bb_step(g.scatter(x), steps=2, rule=W.MENGER_B5S45)
    got = g.gather(out).cpu().numpy()
    assert np.array_equal(got, g.step(x, steps=2, rule=W.MENGER_B5S45).cpu().numpy())
    # and the compact step itself against the oracle on sampled cells
    want = o.step(init, rule=oracle.Rule([5], [4, 5]), steps=2)
    idx = W.sample_omegas(g.cells, 20_000, 7)
    assert np.array_equal(got[idx], want[idx])


def test_bb_bits_path_carpet_r8_whole_box(P):
    g, o = gpu_fr(P, W.CARPET, 8), ora(W.CARPET, 8)
    init = o.init_bernoulli(9, 0.5)
    box = o.scatter(init)
    out = g.bb_step(torch.from_numpy(box).cuda(), steps=2)
    assert np.array_equal(out.cpu().numpy(), o.bb_step(box, steps=2))
    assert np.array_equal(g.gather(out).cpu().numpy(), o.step(init, steps=2))


def test_bb_bits_path_three_strips_carpet_r7(P):
    # side 2187: three strips of 992 cells per row, garbage off the fractal
    g, o = gpu_fr(P, W.CARPET, 7), ora(W.CARPET, 7)
    rng = np.random.default_rng(77)
    box = rng.integers(0, 3, size=g.box_cells).astype(np.uint8) * rng.integers(1, 200, size=g.box_cells).astype(np.uint8)
    for rule in (W.LIFE_B3S23, (0x6, 0x1E)):
        orl = oracle.Rule([i for i in range(9) if (rule[0] >> i) & 1], [i for i in range(9) if (rule[1] >> i) & 1])
        out = g.bb_step(torch.from_numpy(box).cuda(), steps=2, rule=rule)
        assert np.array_equal(out.cpu().numpy(), o.bb_step(box, rule=orl, steps=2)), rule


TETRA4 = W.Family("tetra4", 4, 2, 3, ((0, 0, 0), (1, 0, 0), (0, 1, 0), (0, 0, 1)))


def test_bb_bits3_path_two_strips_side_1024(P):
    # a 3D box of side 1024 (two strips per row, 1.07e9 cells) with garbage
    # off the fractal: its members against the oracle's compact step, and
    # nothing alive off the fractal
    g, o = gpu_fr(P, TETRA4, 10), ora(TETRA4, 10)
    init = o.init_bernoulli(13, 0.5)
    x = torch.from_numpy(init).cuda()
    member = g.scatter(torch.ones_like(x)).bool()
    box = torch.randint(0, 256, (g.box_cells,), dtype=torch.uint8, device="cuda")
    box = torch.where(member, g.scatter(x), box)
    del member
    rule = (0x6, 0x1E)
    orl = oracle.Rule([1, 2], [1, 2, 3, 4])
    out = g.bb_step(box, steps=1, rule=rule)
    del box
    got = g.gather(out)
    assert int(torch.count_nonzero(out)) == int(torch.count_nonzero(got))
    assert np.array_equal(got.cpu().numpy(), o.step(init, rule=orl, steps=1))


def test_scatter_gather_roundtrip(P):
    for fam, r in [(W.CARPET, 4), (W.MENGER, 3), (W.TRIANGLE, 9)]:
        g, o = gpu_fr(P, fam, r), ora(fam, r)
        init = o.init_bernoulli(5, 0.5)
        x = torch.from_numpy(init).cuda()
        box = g.scatter(x)
        assert np.array_equal(box.cpu().numpy(), o.scatter(init))
        assert np.array_equal(g.gather(box).cpu().numpy(), o.gather(o.scatter(init)))


def test_run_host_matches_device(P):
    fam, r = W.TRIANGLE, 9
    g, o = gpu_fr(P, fam, r), ora(fam, r)
    init = o.init_bernoulli(77, 0.4)
    hin = torch.from_numpy(init).pin_memory()
    hout = torch.zeros_like(hin).pin_memory()
    g.run_host(hin, hout, steps=7)
    assert np.array_equal(hout.numpy(), o.step(init, steps=7))


def test_run_host_large_state(P):
    # 3^17 = 129,140,163 bytes each way (an odd size, larger than L2): the
    # result must equal the device-resident step, which the oracle checks
    # elsewhere
    fam, r = W.TRIANGLE, 17
    g = gpu_fr(P, fam, r)
    x = g.init_bernoulli(78, 0.4)
    want = g.step(x, steps=2).cpu()
    hin = x.cpu().pin_memory()
    hout = torch.zeros_like(hin).pin_memory()
    g.run_host(hin, hout, steps=2)
    assert torch.equal(hout, want)
    del x, want
    torch.cuda.empty_cache()


# ---------------------------------------------------- full-size, sampled

def _full_size_check(P, inst, samples, gens=(1, 2)):
    fam, r = inst.family, inst.r
    g, o = gpu_fr(P, fam, r), ora(fam, r)
    init = o.init_bernoulli(inst.seed, inst.p)           # oracle's own input
    st = g.init_bernoulli(inst.seed, inst.p)             # the library's input
    w = np.concatenate([boundary_omegas(fam.k, r), W.sample_omegas(g.cells, samples, 7 + r)])
    wt = torch.from_numpy(w).cuda()
    assert np.array_equal(st[wt].cpu().numpy(), init[w])
    a = st
    b = torch.empty_like(st)
    done = 0
    for t in sorted(gens):
        while done < t:
            g.step(a, out=b, steps=1, rule=rule_of(fam))
            a, b = b, a
            done += 1
        ref = o.cells_after(init, w, t, rule=oracle_rule(fam))
        assert np.array_equal(a[wt].cpu().numpy(), ref), f"generation {t}"
    del a, b, st
    torch.cuda.empty_cache()


def test_full_size_triangle_r20(P):
    _full_size_check(P, W.TRI_R20, 20_000, gens=(1, 2))


def test_full_size_triangle_r16_full_generation(P):
    inst = W.TRI_R16
    g, o = gpu_fr(P, inst.family, inst.r), ora(inst.family, inst.r)
    init = o.init_bernoulli(inst.seed, inst.p)
    st = g.init_bernoulli(inst.seed, inst.p)
    out = g.step(st, steps=1)
    assert np.array_equal(out.cpu().numpy(), o.step(init, steps=1))
    _full_size_check(P, inst, 20_000, gens=(3,))


@pytest.mark.parametrize("inst", [W.CARPET_R10, W.VICSEK_R12, W.MENGER_R6], ids=lambda i: i.family.name)
def test_full_size_other_fractals(P, inst):
    _full_size_check(P, inst, 10_000, gens=(1, 2))


def test_full_size_bb_triangle_r16(P):
    inst = W.TRI_R16
    fam, r = inst.family, inst.r
    g, o = gpu_fr(P, fam, r), ora(fam, r)
    init = o.init_bernoulli(inst.seed, inst.p)
    st = g.init_bernoulli(inst.seed, inst.p)
    box = g.scatter(st)
    out = g.bb_step(box, steps=1)
    del box
    ref = o.step(init, steps=1)
    # sampled box cells: members must equal the compact oracle, the rest 0
    c = np.concatenate([o.lam(W.sample_omegas(g.cells, 50_000, 3)),
                        W.sample_coords(g.side, 2, 50_000, 4)])
    idx = c[:, 0] + g.side * c[:, 1]
    nu = o.nu(c)
    expect = np.where(nu >= 0, ref[np.maximum(nu, 0)], 0).astype(np.uint8)
    got = out[torch.from_numpy(idx).cuda()].cpu().numpy()
    assert np.array_equal(got, expect)
    # and the whole box gathers back to the oracle's compact generation
    assert np.array_equal(g.gather(out).cpu().numpy(), ref)
    del out
    torch.cuda.empty_cache()


# ------------------------------------------------------------ error paths

def test_plan_info(P):
    import ctypes
    g = gpu_fr(P, W.TRIANGLE, 12)
    g.tile_levels = 8
    info = g.plan_info()
    # 81 units of 81 cells per tile of 3^8 cells: 96 threads, two input stages
    assert info["policy_name"] == "tap" and info["tile_levels"] == 8
    assert info["block"] == 96 and info["stages"] == 2
    assert 1 <= info["grid"] <= 3 ** 4 and info["smem_bytes"] > 3 ** 8 and info["blocks_per_sm"] >= 1
    g.tile_levels = 3   # too shallow for 81-cell units
    assert g.plan_info()["policy_name"] != "tap"
    c = gpu_fr(P, W.CARPET, 5)
    c.tile_levels = 4
    ci = c.plan_info()
    assert ci["policy_name"] == "rows_carpet" and ci["block"] == 64   # 8^2 units of 64 cells
    c.tile_levels = 1
    assert c.plan_info()["policy_name"] in ("group3", "cell")
    v = gpu_fr(P, W.VICSEK, 8)
    v.tile_levels = 6
    vi = v.plan_info()
    assert vi["policy_name"] == "lid_vicsek" and vi["block"] == 128   # 5^3 units of 125 cells
    v.tile_levels = 2
    assert v.plan_info()["policy_name"] == "rows_vicsek"
    m = gpu_fr(P, W.MENGER, 4)
    m.tile_levels = 2
    mi = m.plan_info()
    # a 9^3 box in 16-byte rows and its totals box: two stages
    assert mi["policy_name"] == "box3" and mi["stages"] == 2 and mi["smem_bytes"] <= 100 * 1024
    m.tile_levels = 3
    mi = m.plan_info()
    # a warp per 27^3 tile, its box as 29 x 29 row words: no stages, 8 tiles per block
    assert mi["policy_name"] == "bit3" and mi["stages"] == 0 and mi["block"] == 256
    arr = (ctypes.c_int32 * 8)()
    assert g._lib.fractal_plan_info(g._h, arr, 0) != 0
    assert g._lib.fractal_plan_info(g._h, arr, 8) != 0
    assert g._lib.fractal_plan_info(g._h, arr, 2) == 0 and arr[1] == 3


def test_errors(P):
    from paper_2110_12952_gb300.capi import FractalError
    with pytest.raises(FractalError, match="EINVAL"):
        P.Fractal(3, 2, 4, 2, [[0, 0], [1, 0], [1, 0]])  # duplicate rows
    with pytest.raises(FractalError, match="EINVAL"):
        P.Fractal(3, 2, 4, 2, [[0, 0], [1, 0], [2, 0]])  # outside [0,s)
    with pytest.raises(FractalError, match="EINVAL"):
        P.Fractal(5, 2, 4, 2, [[0, 0], [1, 0], [0, 1], [1, 1], [0, 0]])  # k > s^dim
    with pytest.raises(FractalError, match="EOVERFLOW"):
        P.Fractal(3, 2, 31, 2, W.TRIANGLE.table())  # s^r >= 2^31
    g = gpu_fr(P, W.TRIANGLE, 6)
    x = torch.zeros(g.cells * 2, dtype=torch.uint8, device="cuda")
    with pytest.raises(FractalError, match="EINVAL"):
        g.step(x[: g.cells], out=x[5: 5 + g.cells])  # overlapping buffers
    with pytest.raises(FractalError, match="EINVAL"):
        g.step(x[: g.cells], out=x[g.cells:], steps=-1)
    with pytest.raises(FractalError, match="EINVAL"):
        g.tile_levels = 7


@pytest.mark.parametrize("fam,r", [(W.TRIANGLE, 17), (W.CARPET, 9), (W.VICSEK, 12)],
                         ids=lambda v: getattr(v, "name", str(v)))
def test_run_host_pipelined_chunks(P, fam, r):
    # one generation from host memory runs in chunks of tiles whose copies
    # overlap: the result must equal the device-resident step (checked against
    # the oracle elsewhere), also from and to host buffers that are not
    # 16-byte aligned
    g = gpu_fr(P, fam, r)
    x = g.init_bernoulli(79 + r, 0.4)
    want = g.step(x, steps=1, rule=rule_of(fam)).cpu()
    hbuf = torch.zeros(g.cells + 8, dtype=torch.uint8).pin_memory()
    obuf = torch.zeros(g.cells + 8, dtype=torch.uint8).pin_memory()
    for off in (0, 3):
        hin, hout = hbuf[off:off + g.cells], obuf[5:5 + g.cells] if off else obuf[:g.cells]
        hin.copy_(x.cpu())
        hout.zero_()
        g.run_host(hin, hout, steps=1, rule=rule_of(fam))
        assert torch.equal(hout, want), off
    del x, want
    torch.cuda.empty_cache()
