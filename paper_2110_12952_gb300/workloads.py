"""Seeded synthetic inputs: fractal transition tables, rules and workload mixes.

This module only describes inputs.  It holds none of the method's arithmetic
(no lambda, nu, membership or rule evaluation), so that the GPU library and the
CPU oracle can both be fed from it without sharing any computation.

Transition tables (the paper's "transition function", Sec. 1): row j is the
offset, in units of s^mu, of replica j inside the next level.  Replica IDs are
numbered row-major over the s^dim digit box (x fastest, then y, then z); for
the Sierpinski triangle that gives (0,0), (1,0), (0,1), the table of the
triangle workload in Sec. 4.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np


def _rowmajor(s, dim, keep):
    cells = []
    rng = range(s)
    if dim == 2:
        for y in rng:
            for x in rng:
                if keep((x, y)):
                    cells.append((x, y))
    elif dim == 3:
        for z in rng:
            for y in rng:
                for x in rng:
                    if keep((x, y, z)):
                        cells.append((x, y, z))
    else:
        raise ValueError("dim must be 2 or 3")
    return cells


@dataclasses.dataclass(frozen=True)
class Family:
    name: str
    k: int
    s: int
    dim: int
    offsets: tuple

    def table(self) -> np.ndarray:
        return np.asarray(self.offsets, dtype=np.int32).reshape(self.k, self.dim)


def _family(name, s, dim, keep):
    cells = _rowmajor(s, dim, keep)
    return Family(name, len(cells), s, dim, tuple(cells))


#: Sierpinski triangle F^{3,2} (Table 1 "Sierpinski Gasket"; Sec. 4 benchmark).
TRIANGLE = Family("triangle", 3, 2, 2, ((0, 0), (1, 0), (0, 1)))
#: Sierpinski carpet F^{8,3}: the 3x3 digit box without its centre (Table 1).
CARPET = _family("carpet", 3, 2, lambda c: c != (1, 1))
#: Vicsek fractal F^{5,3}: centre plus the 4 orthogonal neighbours (Table 1).
VICSEK = _family("vicsek", 3, 2, lambda c: (c[0] == 1) or (c[1] == 1))
#: Menger sponge F^{20,3} in 3D: the 3^3 digit box without the centre and the
#: 6 face centres (tuples with two or more digits equal to 1).
MENGER = _family("menger", 3, 3, lambda c: sum(1 for v in c if v == 1) < 2)
#: The full square F^{4,2}: every digit tuple kept, so the fractal is the
#: whole n x n box (used to reduce the step to the textbook Game of Life).
FULL_SQUARE = _family("full_square", 2, 2, lambda c: True)
#: The triangle mirrored so that its cells satisfy (y AND NOT x) == 0 at every
#: level; for this table the replica ID equals the paper's procedural Eq. 2.
TRIANGLE_MIRRORED = Family("triangle_mirrored", 3, 2, 2, ((0, 0), (1, 0), (1, 1)))

# Further fractals of Table 1 (Sec. 1).  Their NBB steps are drawn in the
# paper, and the drawings are not in its source: the H- and X-fractals and the
# Cantor set have textbook patterns; for the paper's own "custom" fractals the
# patterns below are readings with the table's k and s.
#: H-fractal F^{7,3}: the two outer columns and the centre.
H_FRACTAL = _family("h_fractal", 3, 2, lambda c: c[0] != 1 or c[1] == 1)
#: X-fractal F^{5,3}: the four corners and the centre.
X_FRACTAL = _family("x_fractal", 3, 2, lambda c: (c[0] == 1) == (c[1] == 1))
#: Cantor set F^{2,3}, on a line of the plane: replicas at x = 0 and 2 of row 0.
CANTOR = _family("cantor_set", 3, 2, lambda c: c[1] == 0 and c[0] != 1)
#: Chandelier F^{4,3} (reading): the top row and the centre below it.
CHANDELIER = _family("chandelier", 3, 2, lambda c: c[1] == 0 or c == (1, 1))
#: Candy F^{12,4} (reading): the 12 border cells of the 4 x 4 box.
CANDY = _family("candy", 4, 2, lambda c: c[0] in (0, 3) or c[1] in (0, 3))
#: Empty-Bottles F^{7,3} (reading): the 3 x 3 box without the top two cells of
#: the middle column, a cup open at the top.
EMPTY_BOTTLES = _family("empty_bottles", 3, 2, lambda c: not (c[0] == 1 and c[1] < 2))

TABLE1_EXTRA = (H_FRACTAL, X_FRACTAL, CANTOR, CHANDELIER, CANDY, EMPTY_BOTTLES)

FAMILIES = {f.name: f for f in (TRIANGLE, CARPET, VICSEK, MENGER, FULL_SQUARE, TRIANGLE_MIRRORED) + TABLE1_EXTRA}


def rule_masks(birth, survive):
    """(birth_mask, survive_mask): bit c set = outcome 1 for c live neighbours."""
    return sum(1 << c for c in birth), sum(1 << c for c in survive)


LIFE_B3S23 = rule_masks([3], [2, 3])
MENGER_B5S45 = rule_masks([5], [4, 5])


def default_rule(family: Family):
    return MENGER_B5S45 if family.dim == 3 else LIFE_B3S23


# ----------------------------------------------------------------- configs

@dataclasses.dataclass(frozen=True)
class Instance:
    family: Family
    r: int
    p: float
    seed: int
    steps: int

    @property
    def cells(self) -> int:
        return self.family.k ** self.r


#: Single-instance workloads (fractal, level, Bernoulli p, seed, generations).
TRI_R8 = Instance(TRIANGLE, 8, 0.5, 1, 100)
TRI_R16 = Instance(TRIANGLE, 16, 0.3, 2, 1000)
TRI_R20 = Instance(TRIANGLE, 20, 0.3, 3, 1000)
CARPET_R10 = Instance(CARPET, 10, 0.5, 4, 500)
VICSEK_R12 = Instance(VICSEK, 12, 0.5, 5, 500)
MENGER_R6 = Instance(MENGER, 6, 0.5, 6, 500)
#: One level above the Menger config: 1.28e9 cells, far larger than L2.
MENGER_R7 = Instance(MENGER, 7, 0.5, 7, 500)

#: Level ranges of the batched / served mixes.
MIX_LEVELS = {"triangle": (6, 14), "carpet": (3, 8), "vicsek": (3, 9)}
MIX_FAMILIES = (TRIANGLE, CARPET, VICSEK)


def batched_mix(n_instances: int = 4096, master_seed: int = 7, steps: int = 200,
                level_ranges=None):
    """Uneven independent instances: family uniform, r uniform in its range,
    p ~ U[0.2, 0.6], per-instance seed drawn from the master seed."""
    rng = np.random.default_rng(master_seed)
    lv = level_ranges or MIX_LEVELS
    out = []
    for _ in range(n_instances):
        fam = MIX_FAMILIES[int(rng.integers(0, len(MIX_FAMILIES)))]
        lo, hi = lv[fam.name]
        r = int(rng.integers(lo, hi + 1))
        p = float(rng.uniform(0.2, 0.6))
        seed = int(rng.integers(0, 2**63 - 1))
        out.append(Instance(fam, r, p, seed, steps))
    return out


@dataclasses.dataclass(frozen=True)
class Request:
    arrival_s: float
    instance: Instance


def poisson_trace(rate_per_s: float = 2000.0, duration_s: float = 60.0, master_seed: int = 8,
                  steps_range=(10, 1000), level_ranges=None):
    """Open-loop Poisson request stream: exponential inter-arrival times, family
    uniform, r uniform in its range, steps log-uniform in ``steps_range``."""
    rng = np.random.default_rng(master_seed)
    lv = level_ranges or MIX_LEVELS
    t = 0.0
    reqs = []
    lo_s, hi_s = steps_range
    while True:
        t += float(rng.exponential(1.0 / rate_per_s))
        if t >= duration_s:
            break
        fam = MIX_FAMILIES[int(rng.integers(0, len(MIX_FAMILIES)))]
        lo, hi = lv[fam.name]
        r = int(rng.integers(lo, hi + 1))
        steps = int(round(math.exp(rng.uniform(math.log(lo_s), math.log(hi_s)))))
        p = float(rng.uniform(0.2, 0.6))
        seed = int(rng.integers(0, 2**63 - 1))
        reqs.append(Request(t, Instance(fam, r, p, seed, steps)))
    return reqs


def sample_omegas(cells: int, count: int, seed: int) -> np.ndarray:
    """Seeded sample of compact indices: the boundary digits first (0, cells-1),
    then uniform draws."""
    rng = np.random.default_rng(seed)
    fixed = np.array([0, cells - 1], dtype=np.int64)
    draws = rng.integers(0, cells, size=max(0, count - len(fixed)), dtype=np.int64)
    return np.unique(np.concatenate([fixed, draws]))


def sample_coords(side: int, dim: int, count: int, seed: int, margin: int = 0) -> np.ndarray:
    """Seeded sample of embedded coordinates in [-margin, side + margin)^dim."""
    rng = np.random.default_rng(seed)
    return rng.integers(-margin, side + margin, size=(count, dim), dtype=np.int64)
