"""Planted mistakes in the oracle must be caught by its pins.

Each mutant is a one-line textual edit of ``oracle/oracle.c`` (a dropped term,
a wrong index or sign, a transposed operand), compiled on the CPU into a
throw-away shared object.  The pin checks below, which depend only on closed
forms, the paper's equations and textbook results, must fail for every
mutant and pass for the unmodified source.
"""
import os
import subprocess

import numpy as np
import pytest
from scipy.signal import convolve2d

import oracle
from paper_2110_12952_gb300 import workloads as W

SRC = os.path.join(os.path.dirname(oracle.__file__), "oracle.c")

MUTANTS = {
    # lambda: x and y offsets swapped
    "lambda_transposed": ("p[i] += smu * off[d * dim + i];",
                          "p[i] += smu * off[d * dim + (dim - 1 - i)];"),
    # lambda: digit taken with the wrong base
    "lambda_wrong_base": ("int64_t d = (omega / oracle_ipow(k, mu)) % k;",
                          "int64_t d = (omega / oracle_ipow(s, mu)) % k;"),
    # nu: level weight off by one
    "nu_level_off_by_one": ("omega += (int64_t)h * oracle_ipow(k, mu);",
                            "omega += (int64_t)h * oracle_ipow(k, mu + 1) / k + (mu == 1);"),
    # nu2d: tau exponent rounded up instead of down
    "tau_ceil": ("c[axis] += (int64_t)h * oracle_ipow(k, mu / dim);",
                 "c[axis] += (int64_t)h * oracle_ipow(k, (mu + dim - 1) / dim);"),
    # nu2d: axis order reversed
    "tau_axis_swapped": ("int axis = mu % dim;", "int axis = (dim - 1) - mu % dim;"),
    # step: the centre cell counted as its own neighbour
    "count_self": ("if (is_zero_offset(dim, delta)) continue;\n        for (int i = 0; i < dim; ++i) q[i] = p[i] + delta[i];\n        if (!in_box(s, r, dim, q)) continue;\n        int64_t w",
                   "for (int i = 0; i < dim; ++i) q[i] = p[i] + delta[i];\n        if (!in_box(s, r, dim, q)) continue;\n        int64_t w"),
    # step: one diagonal dropped (Moore offsets enumerated as 0..3^d-2)
    "drop_last_neighbour": ("    for (int e = 0; e < nq; ++e) {\n        moore_offset(dim, e, delta);\n        if (is_zero_offset(dim, delta)) continue;\n        for (int i = 0; i < dim; ++i) q[i] = p[i] + delta[i];\n        if (!in_box(s, r, dim, q)) continue;",
                            "    for (int e = 0; e < nq - 1; ++e) {\n        moore_offset(dim, e, delta);\n        if (is_zero_offset(dim, delta)) continue;\n        for (int i = 0; i < dim; ++i) q[i] = p[i] + delta[i];\n        if (!in_box(s, r, dim, q)) continue;"),
    # rule: birth and survive masks exchanged
    "rule_swapped": ("uint32_t mask = alive ? survive : birth;", "uint32_t mask = alive ? birth : survive;"),
    # membership: only the top level checked
    "member_top_only": ("for (int mu = 0; mu < r; ++mu) {\n        int64_t smu = oracle_ipow(s, mu);\n        int64_t t[OR_MAXDIM];\n        for (int i = 0; i < dim; ++i) t[i] = (p[i] / smu) % s;\n        if (replica_id(k, dim, off, t) < 0) return 0;",
                        "for (int mu = r - 1; mu < r; ++mu) {\n        int64_t smu = oracle_ipow(s, mu);\n        int64_t t[OR_MAXDIM];\n        for (int i = 0; i < dim; ++i) t[i] = (p[i] / smu) % s;\n        if (replica_id(k, dim, off, t) < 0) return 0;"),
    # box: wrap-around neighbours (torus) instead of a dead border
    "box_wraps": ("        if (!oracle_is_member(k, s, r, dim, off, q)) continue;\n        if (box[box_index(n, dim, q)] != 0) ++count;",
                  "        for (int i = 0; i < dim; ++i) q[i] = (q[i] + n) % n;\n        if (!oracle_is_member(k, s, r, dim, off, q)) continue;\n        if (box[box_index(n, dim, q)] != 0) ++count;"),
    # init: counter not offset by one
    "init_counter": ("return oracle_splitmix64_mix(seed + (i + 1) * 0x9e3779b97f4a7c15ULL);",
                     "return oracle_splitmix64_mix(seed + i * 0x9e3779b97f4a7c15ULL);"),
}


def build_variant(tmp_path, name, edit):
    src = open(SRC).read()
    if edit is not None:
        old, new = edit
        assert src.count(old) >= 1, name
        src = src.replace(old, new, 1)
    c = tmp_path / f"{name}.c"
    so = tmp_path / f"{name}.so"
    c.write_text(src)
    subprocess.run(["gcc", "-O1", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-o", str(so), str(c)],
                   check=True)
    return oracle.load(str(so))


def all_coords(side, dim):
    idx = np.arange(side ** dim, dtype=np.int64)
    cols = []
    for _ in range(dim):
        cols.append(idx % side)
        idx = idx // side
    return np.stack(cols, axis=1)


def life(g, member):
    g = g.astype(np.int64) * member
    cnt = convolve2d(g, np.ones((3, 3), dtype=np.int64), mode="same") - g
    return (np.where(g == 1, np.isin(cnt, (2, 3)), cnt == 3) * member).astype(np.uint8)


GOLDEN_SM = [(0, 0, 16294208416658607535), (1234567, 1, 3203168211198807973)]


def pins_hold(lib) -> bool:
    """A compact subset of the oracle pins; True iff all of them hold."""
    try:
        # membership closed form and k^r
        f = oracle.Fractal(3, 2, 5, 2, W.TRIANGLE.table(), lib=lib)
        c = all_coords(32, 2)
        if not np.array_equal(f.member(c), ((c[:, 0] & c[:, 1]) == 0).astype(np.uint8)):
            return False
        for fam, r in [(W.TRIANGLE, 5), (W.VICSEK, 3), (W.CARPET, 2)]:
            g = oracle.Fractal(fam.k, fam.s, r, 2, fam.table(), lib=lib)
            cc = all_coords(g.side, 2)
            m = g.member(cc).astype(bool)
            if m.sum() != g.cells:
                return False
            w = np.arange(g.cells)
            p = g.lam(w)
            if not g.member(p).all() or len({tuple(x) for x in p}) != g.cells:
                return False
            if not np.array_equal(g.nu(p), w) or (g.nu(cc[~m]) != -1).any():
                return False
            # unfolding of the 2D compact view
            c2 = g.nu2d(p)
            if c2[:, 0].max() != fam.k ** ((r + 1) // 2) - 1 or c2[:, 1].max() != fam.k ** (r // 2) - 1:
                return False
            top = w // fam.k ** (r - 1)
            sub0 = {tuple(v) for v in c2[top == 0]}
            sub1 = {tuple(v) for v in c2[top == 1]}
            d = (fam.k ** (r // 2), 0) if r % 2 == 1 else (0, fam.k ** ((r - 1) // 2))
            if sub1 != {(a + d[0], b + d[1]) for a, b in sub0}:
                return False
            # compact and BB steps against a library convolution
            rng = np.random.default_rng(r)
            mm = m.reshape(g.side, g.side).astype(np.uint8)
            box = (rng.random((g.side, g.side)) < 0.5).astype(np.uint8) * mm
            ref = life(box, mm)
            if not np.array_equal(g.bb_step(box.reshape(-1)).reshape(g.side, g.side), ref):
                return False
            comp = g.step(g.gather(box.reshape(-1)))
            if not np.array_equal(g.scatter(comp).reshape(g.side, g.side), ref):
                return False
        for seed, i, v in GOLDEN_SM:
            if int(lib.oracle_splitmix64_nth(seed, i)) != v:
                return False
        return True
    except AssertionError:
        return False


def test_unmodified_oracle_passes(tmp_path):
    assert pins_hold(build_variant(tmp_path, "clean", None))


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(tmp_path, name):
    assert not pins_hold(build_variant(tmp_path, name, MUTANTS[name]))
