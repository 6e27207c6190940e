"""Failure detection without a GPU fault: a step launch whose pipeline
barriers are armed for more bytes than are ever copied (a stage that never
completes, as a lost copy would leave it) must give up its bounded waits,
report FR_ETIMEOUT through fractal_check, leave the context usable, and the
next call must be bit-exact against the oracle.  The waits are shortened to a
few hundred tries for the armed launch only (fractal_test_arm_timeout)."""
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


# one fractal per tile loop: the tap policy (triangle), the padded-unit rows
# policy (carpet), the lid policy (Vicsek) and the box3 policy (Menger at two
# levels; at three levels its bit3 policy reads with plain loads, no waits)
CASES = [(W.TRIANGLE, 12, 9), (W.CARPET, 6, 4), (W.VICSEK, 7, 6), (W.MENGER, 4, 2)]


@pytest.mark.parametrize("fam,r,L", CASES, ids=lambda v: getattr(v, "name", str(v)))
def test_bounded_wait_times_out_and_recovers(P, fam, r, L):
    g = P.Fractal.from_family(fam, r)
    g.tile_levels = L
    o = oracle.Fractal(fam.k, fam.s, r, fam.dim, fam.table())
    rule = W.default_rule(fam)
    init = o.init_bernoulli(40 + r, 0.45)
    x = torch.from_numpy(init).cuda()
    lib = g._lib
    assert lib.fractal_check(g._h) == 0
    assert lib.fractal_test_arm_timeout(g._h, 16, 256) == 0
    y = torch.full_like(x, 7)
    g.step(x, out=y, steps=1, rule=rule)          # enqueued: the error is asynchronous
    rc = lib.fractal_check(g._h)
    assert rc == -5, lib.fractal_last_error()     # FR_ETIMEOUT
    assert b"gave up" in lib.fractal_last_error()
    assert lib.fractal_check(g._h) == 0           # the flag was cleared
    # the context and the handle are still usable, and exact
    out = g.step(x, steps=3, rule=rule)
    assert lib.fractal_check(g._h) == 0
    ref = o.step(init, rule=oracle.Rule(*rule), steps=3)
    assert np.array_equal(out.cpu().numpy(), ref)


def test_arm_timeout_rejects_bad_arguments(P):
    g = P.Fractal.from_family(W.TRIANGLE, 5)
    assert g._lib.fractal_test_arm_timeout(g._h, 0, 10) == -1
    assert g._lib.fractal_test_arm_timeout(g._h, 16, 0) == -1
    assert g._lib.fractal_test_arm_timeout(g._h, 8192, 10) == -1
