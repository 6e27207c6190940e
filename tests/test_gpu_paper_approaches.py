"""The paper's own approaches (Sec. 4): "lambda(omega)" on the masked box and
"nu(omega)" on the blocked rho x rho storage, against the oracle at every
block size, through the library's layout conversions (whose round trips are
checked too)."""
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


CASES = [(W.TRIANGLE, 8, [1, 2, 3, 4, 5]), (W.CARPET, 4, [1, 2, 3]), (W.VICSEK, 5, [1, 2, 3]),
         (W.MENGER, 3, [1, 2]), (W.H_FRACTAL, 4, [1, 2])]


@pytest.mark.parametrize("fam,r,levels", CASES, ids=lambda v: getattr(v, "name", str(v)))
def test_lambda_box_and_blocked_match_oracle(P, fam, r, levels):
    g, o = P.Fractal.from_family(fam, r), ora(fam, r)
    rule = W.default_rule(fam)
    init = o.init_bernoulli(900 + r, 0.45)
    x = torch.from_numpy(init).cuda()
    steps = 5
    want = o.step(init, rule=oracle.Rule(*rule), steps=steps)
    box = g.scatter(x)
    for l in levels:
        # lambda(omega): box in, box out (cells off the fractal stay 0)
        out_box = g.lambda_box_step(box, l, out=torch.zeros_like(box), steps=steps, rule=rule)
        assert np.array_equal(g.gather(out_box).cpu().numpy(), want), f"lambda rho_levels={l}"
        assert np.array_equal(out_box.cpu().numpy(), o.scatter(want)), f"lambda box rho_levels={l}"
        # nu(omega) on blocked storage
        blk = g.blocked_pack(x, l)
        assert blk.numel() == fam.k ** (r - l) * (fam.s ** l) ** fam.dim
        assert np.array_equal(g.blocked_unpack(blk, l).cpu().numpy(), init != 0)
        out_blk = g.blocked_step(blk, l, steps=steps, rule=rule)
        assert np.array_equal(g.blocked_unpack(out_blk, l).cpu().numpy(), want), f"blocked rho_levels={l}"
        # off-fractal bytes of the blocked layout are 0
        assert int(out_blk.sum().item()) == int(want.sum())


def test_blocked_many_blocks_triangle_r14(P):
    fam, r = W.TRIANGLE, 14
    g, o = P.Fractal.from_family(fam, r), ora(fam, r)
    init = o.init_bernoulli(17, 0.3)
    x = torch.from_numpy(init).cuda()
    want = o.step(init, steps=3)
    for l in (3, 5):
        out = g.blocked_unpack(g.blocked_step(g.blocked_pack(x, l), l, steps=3), l)
        assert np.array_equal(out.cpu().numpy(), want), l
    box = g.scatter(x)
    assert np.array_equal(g.gather(g.lambda_box_step(box, 4, steps=3)).cpu().numpy(), want)


def test_paper_approaches_reject_bad_block_sizes(P):
    from paper_2110_12952_gb300.capi import FractalError
    g = P.Fractal.from_family(W.TRIANGLE, 8)
    with pytest.raises(FractalError, match="EINVAL"):
        g.blocked_bytes(6)            # 64 x 64 threads per block
    with pytest.raises(FractalError, match="EINVAL"):
        g.blocked_bytes(0)
