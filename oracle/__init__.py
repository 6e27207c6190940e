"""CPU oracle for cellular automata on compact NBB fractals.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the CPU-baseline / reference legs of ``bench.py`` may import this package.  The
library under ``paper_2110_12952_gb300/`` never imports it and shares no code
with it: the C source ``oracle.c`` is compiled on its own into ``_oracle.so``
and is loaded here through ctypes.

Each function follows the paper's definitions (Quezada & Navarro 2021):
NBB fractals and the volume k^r (Sec. 1, Eq. 1), the replica-ID helper H and
the compact map nu (Sec. 3.1, Eqs. 2-8), its inverse lambda (Sec. 3), the
stencil procedure that combines them (Sec. 3) and the bounding-box approach it
is compared with (Sec. 4).  See ``oracle.c`` for the definitions themselves.

Parity status: every function here is pinned by the tests in
``tests/test_oracle_pins.py`` except the numeric values of nu for the specific
cells drawn in the paper's worked-example figure, which the source does not
contain ("parity unpinned" for that figure only).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import sys
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_SO = os.path.join(_HERE, "_oracle.so")
_lock = threading.Lock()
_lib = None

_i32p = ctypes.POINTER(ctypes.c_int32)
_i64p = ctypes.POINTER(ctypes.c_int64)
_u8p = ctypes.POINTER(ctypes.c_uint8)


def build(force: bool = False, so_path: str | None = None, defines=()) -> str:
    """Compile ``oracle.c`` with gcc (OpenMP on) into a shared object."""
    out = so_path or _SO
    if not force and os.path.exists(out) and os.path.getmtime(out) >= os.path.getmtime(_SRC):
        return out
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp"]
    cmd += [f"-D{d}" for d in defines]
    cmd += ["-o", out + ".tmp", _SRC]
    subprocess.run(cmd, check=True)
    os.replace(out + ".tmp", out)
    return out


def _declare(lib):
    I, L, D, U32, U64 = ctypes.c_int, ctypes.c_int64, ctypes.c_double, ctypes.c_uint32, ctypes.c_uint64
    fr = [I, I, I, I, _i32p]
    sig = {
        "oracle_ipow": (L, [L, I]),
        "oracle_threads": (I, []),
        "oracle_is_member": (I, fr + [_i64p]),
        "oracle_lambda": (None, fr + [L, _i64p]),
        "oracle_nu": (L, fr + [_i64p]),
        "oracle_nu2d": (I, fr + [_i64p, _i64p]),
        "oracle_lambda_batch": (None, fr + [_i64p, L, _i64p]),
        "oracle_nu_batch": (None, fr + [_i64p, L, _i64p]),
        "oracle_nu2d_batch": (None, fr + [_i64p, L, _i64p]),
        "oracle_member_batch": (None, fr + [_i64p, L, _u8p]),
        "oracle_step_compact_range": (None, fr + [_u8p, _u8p, U32, U32, L, L]),
        "oracle_step_compact_cells": (None, fr + [_u8p, _i64p, L, U32, U32, _u8p]),
        "oracle_run_compact": (I, fr + [_u8p, _u8p, L, U32, U32]),
        "oracle_cells_after": (None, fr + [_u8p, _i64p, L, I, U32, U32, _u8p]),
        "oracle_step_bb": (None, fr + [_u8p, _u8p, U32, U32]),
        "oracle_step_bb_cells": (None, fr + [_u8p, _i64p, L, U32, U32, _u8p]),
        "oracle_run_bb": (I, fr + [_u8p, _u8p, L, U32, U32]),
        "oracle_scatter": (None, fr + [_u8p, _u8p]),
        "oracle_gather": (None, fr + [_u8p, _u8p]),
        "oracle_splitmix64_nth": (U64, [U64, U64]),
        "oracle_bernoulli_threshold": (U64, [D]),
        "oracle_init_bernoulli": (None, [U64, D, _u8p, L, L]),
    }
    mx = [I, I, I, _i32p, _i32p]   # s, r, dim, ks, offs
    sig.update({
        "oracle_mix_cells": (L, [I, _i32p]),
        "oracle_mix_lambda_batch": (None, mx + [_i64p, L, _i64p]),
        "oracle_mix_nu_batch": (None, mx + [_i64p, L, _i64p]),
        "oracle_mix_nu2d_batch": (None, mx + [_i64p, L, _i64p]),
        "oracle_mix_member_batch": (None, mx + [_i64p, L, _u8p]),
        "oracle_mix_run": (I, mx + [_u8p, _u8p, L, U32, U32]),
        "oracle_mix_run_bb": (I, mx + [_u8p, _u8p, L, U32, U32]),
        "oracle_mix_scatter": (None, mx + [_u8p, _u8p]),
        "oracle_mix_gather": (None, mx + [_u8p, _u8p]),
    })
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


def load(so_path: str | None = None):
    """Load (building first if needed) the oracle shared object."""
    global _lib
    if so_path is not None:
        return _declare(ctypes.CDLL(so_path))
    with _lock:
        if _lib is None:
            _lib = _declare(ctypes.CDLL(build()))
    return _lib


def _p(a, t):
    return a.ctypes.data_as(t)


def threads() -> int:
    return int(load().oracle_threads())


def splitmix64_nth(seed: int, i: int) -> int:
    return int(load().oracle_splitmix64_nth(seed & (2**64 - 1), i))


class Rule:
    """Life-like rule: bit c of ``birth``/``survive`` decides a cell with c live neighbours."""

    def __init__(self, birth, survive):
        self.birth = sum(1 << c for c in birth) if not isinstance(birth, int) else birth
        self.survive = sum(1 << c for c in survive) if not isinstance(survive, int) else survive


LIFE = Rule([3], [2, 3])          # B3/S23
MENGER_RULE = Rule([5], [4, 5])   # B5/S45


class Fractal:
    """An NBB fractal F_n^{k,s} at level r with transition table ``offsets`` (k x dim)."""

    def __init__(self, k, s, r, dim, offsets, lib=None):
        off = np.ascontiguousarray(np.asarray(offsets, dtype=np.int32).reshape(k, dim))
        self.k, self.s, self.r, self.dim = int(k), int(s), int(r), int(dim)
        self.off = off
        self.lib = lib or load()
        self.cells = self.k ** self.r
        self.side = self.s ** self.r
        self.box_cells = self.side ** self.dim

    # common leading arguments
    def _fa(self):
        return (self.k, self.s, self.r, self.dim, _p(self.off, _i32p))

    def is_member(self, p) -> bool:
        q = np.ascontiguousarray(np.asarray(p, dtype=np.int64))
        return bool(self.lib.oracle_is_member(*self._fa(), _p(q, _i64p)))

    def member(self, coords) -> np.ndarray:
        c = np.ascontiguousarray(np.asarray(coords, dtype=np.int64).reshape(-1, self.dim))
        m = np.zeros(len(c), dtype=np.uint8)
        self.lib.oracle_member_batch(*self._fa(), _p(c, _i64p), len(c), _p(m, _u8p))
        return m

    def lam(self, omega) -> np.ndarray:
        w = np.ascontiguousarray(np.asarray(omega, dtype=np.int64).reshape(-1))
        out = np.zeros((len(w), self.dim), dtype=np.int64)
        self.lib.oracle_lambda_batch(*self._fa(), _p(w, _i64p), len(w), _p(out, _i64p))
        return out

    def nu(self, coords) -> np.ndarray:
        c = np.ascontiguousarray(np.asarray(coords, dtype=np.int64).reshape(-1, self.dim))
        out = np.zeros(len(c), dtype=np.int64)
        self.lib.oracle_nu_batch(*self._fa(), _p(c, _i64p), len(c), _p(out, _i64p))
        return out

    def nu2d(self, coords) -> np.ndarray:
        c = np.ascontiguousarray(np.asarray(coords, dtype=np.int64).reshape(-1, self.dim))
        out = np.zeros((len(c), self.dim), dtype=np.int64)
        self.lib.oracle_nu2d_batch(*self._fa(), _p(c, _i64p), len(c), _p(out, _i64p))
        return out

    def init_bernoulli(self, seed: int, p: float, w0: int = 0, w1: int | None = None,
                       out: np.ndarray | None = None) -> np.ndarray:
        w1 = self.cells if w1 is None else w1
        st = out if out is not None else np.zeros(self.cells, dtype=np.uint8)
        self.lib.oracle_init_bernoulli(seed & (2**64 - 1), float(p), _p(st, _u8p), w0, w1)
        return st

    def step(self, state, rule=LIFE, steps: int = 1) -> np.ndarray:
        a = np.ascontiguousarray(np.asarray(state, dtype=np.uint8))
        assert a.size == self.cells
        out = np.zeros_like(a)
        rc = self.lib.oracle_run_compact(*self._fa(), _p(a, _u8p), _p(out, _u8p), steps,
                                         rule.birth, rule.survive)
        assert rc == 0
        return out

    def step_range(self, state, w0, w1, rule=LIFE, out=None) -> np.ndarray:
        a = np.ascontiguousarray(state)
        o = out if out is not None else np.zeros_like(a)
        self.lib.oracle_step_compact_range(*self._fa(), _p(a, _u8p), _p(o, _u8p),
                                           rule.birth, rule.survive, w0, w1)
        return o

    def step_cells(self, state, omegas, rule=LIFE) -> np.ndarray:
        a = np.ascontiguousarray(state)
        w = np.ascontiguousarray(np.asarray(omegas, dtype=np.int64))
        v = np.zeros(len(w), dtype=np.uint8)
        self.lib.oracle_step_compact_cells(*self._fa(), _p(a, _u8p), _p(w, _i64p), len(w),
                                           rule.birth, rule.survive, _p(v, _u8p))
        return v

    def cells_after(self, init, omegas, t: int, rule=LIFE) -> np.ndarray:
        a = np.ascontiguousarray(init)
        w = np.ascontiguousarray(np.asarray(omegas, dtype=np.int64))
        v = np.zeros(len(w), dtype=np.uint8)
        self.lib.oracle_cells_after(*self._fa(), _p(a, _u8p), _p(w, _i64p), len(w), t,
                                    rule.birth, rule.survive, _p(v, _u8p))
        return v

    def bb_step(self, box, rule=LIFE, steps: int = 1) -> np.ndarray:
        a = np.ascontiguousarray(np.asarray(box, dtype=np.uint8)).reshape(-1)
        assert a.size == self.box_cells
        out = np.zeros_like(a)
        rc = self.lib.oracle_run_bb(*self._fa(), _p(a, _u8p), _p(out, _u8p), steps,
                                    rule.birth, rule.survive)
        assert rc == 0
        return out

    def bb_cells(self, box, idxs, rule=LIFE) -> np.ndarray:
        a = np.ascontiguousarray(box).reshape(-1)
        w = np.ascontiguousarray(np.asarray(idxs, dtype=np.int64))
        v = np.zeros(len(w), dtype=np.uint8)
        self.lib.oracle_step_bb_cells(*self._fa(), _p(a, _u8p), _p(w, _i64p), len(w),
                                      rule.birth, rule.survive, _p(v, _u8p))
        return v

    def scatter(self, compact) -> np.ndarray:
        a = np.ascontiguousarray(np.asarray(compact, dtype=np.uint8))
        box = np.zeros(self.box_cells, dtype=np.uint8)
        self.lib.oracle_scatter(*self._fa(), _p(a, _u8p), _p(box, _u8p))
        return box

    def gather(self, box) -> np.ndarray:
        a = np.ascontiguousarray(np.asarray(box, dtype=np.uint8)).reshape(-1)
        out = np.zeros(self.cells, dtype=np.uint8)
        self.lib.oracle_gather(*self._fa(), _p(a, _u8p), _p(out, _u8p))
        return out


class MixedFractal:
    """A fractal with a different NBB transition table at each level
    (``tables[mu]``: k_mu x dim offsets for level mu, mu = 0 the finest),
    common growth ratio ``s``: the combination the paper's conclusions name as
    future work.  Compact indices are mixed-radix (level mu's digit has
    weight k_0 ... k_(mu-1)); see ``oracle.c``."""

    def __init__(self, s, r, dim, tables, lib=None):
        assert len(tables) == r
        self.s, self.r, self.dim = int(s), int(r), int(dim)
        tabs = [np.asarray(t, dtype=np.int32).reshape(-1, dim) for t in tables]
        self.ks = np.ascontiguousarray(np.array([len(t) for t in tabs] or [1], dtype=np.int32))
        self.offs = np.ascontiguousarray(np.concatenate([t.reshape(-1) for t in tabs]) if tabs
                                         else np.zeros(1, dtype=np.int32))
        self.lib = lib or load()
        self.cells = int(np.prod([len(t) for t in tabs])) if tabs else 1
        self.side = self.s ** self.r
        self.box_cells = self.side ** self.dim

    def _fa(self):
        return (self.s, self.r, self.dim, _p(self.ks, _i32p), _p(self.offs, _i32p))

    def member(self, coords) -> np.ndarray:
        c = np.ascontiguousarray(np.asarray(coords, dtype=np.int64).reshape(-1, self.dim))
        m = np.zeros(len(c), dtype=np.uint8)
        self.lib.oracle_mix_member_batch(*self._fa(), _p(c, _i64p), len(c), _p(m, _u8p))
        return m

    def lam(self, omega) -> np.ndarray:
        w = np.ascontiguousarray(np.asarray(omega, dtype=np.int64).reshape(-1))
        out = np.zeros((len(w), self.dim), dtype=np.int64)
        self.lib.oracle_mix_lambda_batch(*self._fa(), _p(w, _i64p), len(w), _p(out, _i64p))
        return out

    def nu(self, coords) -> np.ndarray:
        c = np.ascontiguousarray(np.asarray(coords, dtype=np.int64).reshape(-1, self.dim))
        out = np.zeros(len(c), dtype=np.int64)
        self.lib.oracle_mix_nu_batch(*self._fa(), _p(c, _i64p), len(c), _p(out, _i64p))
        return out

    def nu2d(self, coords) -> np.ndarray:
        c = np.ascontiguousarray(np.asarray(coords, dtype=np.int64).reshape(-1, self.dim))
        out = np.zeros((len(c), self.dim), dtype=np.int64)
        self.lib.oracle_mix_nu2d_batch(*self._fa(), _p(c, _i64p), len(c), _p(out, _i64p))
        return out

    def init_bernoulli(self, seed: int, p: float) -> np.ndarray:
        st = np.zeros(self.cells, dtype=np.uint8)
        self.lib.oracle_init_bernoulli(seed & (2**64 - 1), float(p), _p(st, _u8p), 0, self.cells)
        return st

    def step(self, state, rule=LIFE, steps: int = 1) -> np.ndarray:
        a = np.ascontiguousarray(np.asarray(state, dtype=np.uint8))
        assert a.size == self.cells
        out = np.zeros_like(a)
        assert self.lib.oracle_mix_run(*self._fa(), _p(a, _u8p), _p(out, _u8p), steps,
                                       rule.birth, rule.survive) == 0
        return out

    def bb_step(self, box, rule=LIFE, steps: int = 1) -> np.ndarray:
        a = np.ascontiguousarray(np.asarray(box, dtype=np.uint8)).reshape(-1)
        assert a.size == self.box_cells
        out = np.zeros_like(a)
        assert self.lib.oracle_mix_run_bb(*self._fa(), _p(a, _u8p), _p(out, _u8p), steps,
                                          rule.birth, rule.survive) == 0
        return out

    def scatter(self, compact) -> np.ndarray:
        a = np.ascontiguousarray(np.asarray(compact, dtype=np.uint8))
        box = np.zeros(self.box_cells, dtype=np.uint8)
        self.lib.oracle_mix_scatter(*self._fa(), _p(a, _u8p), _p(box, _u8p))
        return box

    def gather(self, box) -> np.ndarray:
        a = np.ascontiguousarray(np.asarray(box, dtype=np.uint8)).reshape(-1)
        out = np.zeros(self.cells, dtype=np.uint8)
        self.lib.oracle_mix_gather(*self._fa(), _p(a, _u8p), _p(out, _u8p))
        return out


if __name__ == "__main__":  # pragma: no cover
    print(build(force="--force" in sys.argv))
