"""The bit3 policy of the compact step (3D, s = 3, tiles of three levels; a
warp per tile, box rows as bit-sliced words) against the oracle: the rule
evaluated with constants (B5/S45) and in general, non-binary input, other 3D
tables whose replica counts are multiples of 4 (and a permuted replica
order), buffers at unaligned addresses, tile ranges (the chunked host call),
a batch of instances with different rules, the bit-packed state between the
generations of a multi-generation call, the plan it is chosen for, and the
3D bounding-box row kernel on the same tables."""
import numpy as np
import pytest
import torch

import oracle
from paper_2110_12952_gb300 import workloads as W

pytestmark = pytest.mark.gpu

CORNERS8 = W.Family("corners8", 8, 3, 3, tuple((x, y, z) for z in (0, 2) for y in (0, 2) for x in (0, 2)))
EDGES12 = W.Family("edges12", 12, 3, 3, tuple((x, y, z) for z in range(3) for y in range(3) for x in range(3)
                                              if [x, y, z].count(1) == 1))
MENGER_REV = W.Family("menger_rev", 20, 3, 3, tuple(reversed(W.MENGER.table())))
# the extremes of k: one word per block (4 cells) and six (24 cells; its
# tables and boxes need more than 48 KB of shared memory per block)
FOUR4 = W.Family("four4", 4, 3, 3, ((0, 0, 0), (2, 0, 0), (1, 2, 0), (1, 1, 2)))
DENSE24 = W.Family("dense24", 24, 3, 3, tuple((x, y, z) for z in range(3) for y in range(3) for x in range(3)
                                              if (x, y, z) not in ((1, 1, 1), (0, 1, 1), (1, 0, 2))))

RULES = [W.MENGER_B5S45, (1 << 4, 1 << 4), (0x6, 0x1E), (0x7FFE000, 0x7FFE000), (0x2, 0x3), (0, 0)]


@pytest.fixture(scope="module")
def P():
    from paper_2110_12952_gb300 import build
    build.build()
    import paper_2110_12952_gb300 as pkg
    return pkg


def pair(P, fam, r):
    g = P.Fractal.from_family(fam, r)
    o = oracle.Fractal(fam.k, fam.s, r, fam.dim, [tuple(int(v) for v in t) for t in fam.table()])
    return g, o


def orule(rule):
    b, s = rule
    return oracle.Rule([i for i in range(27) if (b >> i) & 1], [i for i in range(27) if (s >> i) & 1])


def nonbinary(n, seed):
    rng = np.random.default_rng(seed)
    return (rng.integers(0, 2, size=n) * rng.integers(1, 256, size=n)).astype(np.uint8)


def test_plan_is_bit3_at_three_levels(P):
    g, _ = pair(P, W.MENGER, 5)
    info = g.plan_info()
    assert info["policy_name"] == "bit3" and info["tile_levels"] == 3 and info["block"] == 256
    assert info["stages"] == 0 and info["smem_bytes"] <= 56 * 1024 and info["blocks_per_sm"] >= 3
    g.tile_levels = 2
    assert g.plan_info()["policy_name"] == "box3"
    for fam in (CORNERS8, EDGES12, MENGER_REV):
        h, _ = pair(P, fam, 4)
        assert h.plan_info()["policy_name"] == "bit3", fam.name
    c, _ = pair(P, W.Family("corners9", 9, 3, 3, tuple((x, y, z) for z in range(3) for y in range(3)
                                                      for x in range(3) if (x != 1 and y != 1 and z != 1)
                                                      or (x, y, z) == (1, 1, 1))), 4)
    assert c.plan_info()["policy_name"] != "bit3"   # k = 9 is not a multiple of 4


@pytest.mark.parametrize("rule", RULES, ids=lambda r: f"B{r[0]:x}S{r[1]:x}")
def test_rules_on_nonbinary_input(P, rule):
    g, o = pair(P, W.MENGER, 4)
    raw = nonbinary(o.cells, 11)
    got = g.step(torch.from_numpy(raw).cuda(), steps=1, rule=rule).cpu().numpy()
    assert np.array_equal(got, o.step(raw, rule=orule(rule), steps=1))
    init = o.init_bernoulli(12, 0.45)
    got = g.step(torch.from_numpy(init).cuda(), steps=6, rule=rule).cpu().numpy()
    assert np.array_equal(got, o.step(init, rule=orule(rule), steps=6))


@pytest.mark.parametrize("fam,r", [(CORNERS8, 5), (EDGES12, 4), (MENGER_REV, 4), (W.MENGER, 3), (W.MENGER, 5),
                                   (FOUR4, 6), (DENSE24, 4)],
                         ids=lambda v: getattr(v, "name", str(v)))
def test_tables_and_sizes(P, fam, r):
    g, o = pair(P, fam, r)
    assert g.plan_info()["policy_name"] == "bit3"
    init = o.init_bernoulli(r, 0.5)
    for rule in (W.MENGER_B5S45, (0x6, 0x1E), (0x2, 0x3)):
        got = g.step(torch.from_numpy(init).cuda(), steps=3, rule=rule).cpu().numpy()
        assert np.array_equal(got, o.step(init, rule=orule(rule), steps=3)), rule


@pytest.mark.parametrize("shift_in,shift_out", [(1, 3), (4, 8), (2, 0), (0, 5)])
def test_unaligned_buffers(P, shift_in, shift_out):
    g, o = pair(P, W.MENGER, 4)
    init = o.init_bernoulli(5, 0.5)
    base_in = torch.zeros(o.cells + 32, dtype=torch.uint8, device="cuda")
    base_out = torch.full((o.cells + 32,), 9, dtype=torch.uint8, device="cuda")
    x = base_in[shift_in:shift_in + o.cells]
    x.copy_(torch.from_numpy(init))
    y = base_out[shift_out:shift_out + o.cells]
    g.step(x, out=y, steps=1, rule=W.MENGER_B5S45)
    assert np.array_equal(y.cpu().numpy(), o.step(init, rule=orule(W.MENGER_B5S45), steps=1))
    # nothing outside the output view was written
    assert (base_out[:shift_out] == 9).all() and (base_out[shift_out + o.cells:] == 9).all()


def test_tile_ranges_of_the_host_call(P):
    # fractal_run_host's single generation runs the tiles in chunks (range launches)
    g, o = pair(P, W.MENGER, 5)
    init = o.init_bernoulli(8, 0.5)
    hin = torch.from_numpy(init).pin_memory()
    hout = torch.empty_like(hin).pin_memory()
    g.run_host(hin, hout, steps=1, rule=W.MENGER_B5S45)
    assert np.array_equal(hout.numpy(), o.step(init, rule=orule(W.MENGER_B5S45), steps=1))


def test_batch_with_different_rules(P):
    cases = [(W.MENGER, 4, W.MENGER_B5S45), (W.MENGER, 3, (0x6, 0x1E)), (EDGES12, 4, (0x2, 0x3)),
             (W.MENGER, 4, (1 << 4, 1 << 4))]
    batch = P.Batch()
    keep = []
    for i, (fam, r, rule) in enumerate(cases):
        g, o = pair(P, fam, r)
        init = o.init_bernoulli(30 + i, 0.5)
        x = torch.from_numpy(init).cuda()
        y = torch.empty_like(x)
        batch.add(g, x, y, 5, rule=rule)
        keep.append((g, o, init, y, rule))
    batch.run()
    torch.cuda.synchronize()
    for g, o, init, y, rule in keep:
        assert np.array_equal(y.cpu().numpy(), o.step(init, rule=orule(rule), steps=5))
    batch.close()


@pytest.mark.parametrize("fam,r", [(W.MENGER, 4), (EDGES12, 4), (MENGER_REV, 5)], ids=lambda v: getattr(v, "name", str(v)))
@pytest.mark.parametrize("rule", [W.MENGER_B5S45, (0x6, 0x1E)], ids=lambda r: f"B{r[0]:x}S{r[1]:x}")
def test_bit_packed_generations(P, fam, r, rule):
    # steps >= 2: the first generation writes bit-packed tile states, the
    # ones between read and write them, the last writes bytes
    g, o = pair(P, fam, r)
    raw = nonbinary(o.cells, 21)
    x = torch.from_numpy(raw).cuda()
    for steps in (2, 3, 5):
        got = g.step(x, steps=steps, rule=rule).cpu().numpy()
        assert np.array_equal(got, o.step(raw, rule=orule(rule), steps=steps)), steps


@pytest.mark.parametrize("fam,r", [(EDGES12, 5), (CORNERS8, 5), (DENSE24, 5)], ids=lambda v: getattr(v, "name", str(v)))
def test_bb_bits3_other_tables(P, fam, r):
    # the 3D bit-sliced row kernel of the bounding-box step on tables other than the Menger sponge's
    g, o = pair(P, fam, r)
    rng = np.random.default_rng(r)
    box = rng.integers(0, 3, size=g.box_cells).astype(np.uint8) * rng.integers(1, 200, size=g.box_cells).astype(np.uint8)
    got = g.bb_step(torch.from_numpy(box).cuda(), steps=2, rule=(0x6, 0x1E)).cpu().numpy()
    assert np.array_equal(got, o.bb_step(box, rule=orule((0x6, 0x1E)), steps=2))
