"""Python binding of the compact-fractal library: the same calls as the C ABI
(``include/fractal.h``), taking PyTorch CUDA tensors and the current stream.

This module only marshals arguments; every map, step and copy runs in
``libfractal.so``.  PyTorch provides device memory and streams.
"""
from __future__ import annotations

import ctypes

import numpy as np
import torch

from . import capi
from .workloads import Family, LIFE_B3S23, default_rule


def _stream(stream=None) -> int:
    s = stream if stream is not None else torch.cuda.current_stream()
    return s.cuda_stream


def _dev_ptr(t: torch.Tensor, dtype, name: str) -> int:
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must have dtype {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    return t.data_ptr()


class Fractal:
    """Handle on an NBB fractal F^{k,s} at level r (``fractal_create``)."""

    def __init__(self, k: int, s: int, r: int, dim: int, offsets):
        self._lib = capi.load()
        off = np.ascontiguousarray(np.asarray(offsets, dtype=np.int32).reshape(k * dim))
        h = capi.c_fp()
        capi.check(self._lib.fractal_create(k, s, r, dim, off.ctypes.data_as(capi.c_i32p),
                                            ctypes.byref(h)), self._lib)
        self._h = h
        self.k, self.s, self.r, self.dim = k, s, r, dim
        self.offsets = off.reshape(k, dim).copy()
        cells, side = ctypes.c_int64(), ctypes.c_int64()
        capi.check(self._lib.fractal_info(h, ctypes.byref(cells), ctypes.byref(side)), self._lib)
        self.cells, self.side = cells.value, side.value
        self.box_cells = self.side ** dim

    @classmethod
    def from_family(cls, fam: Family, r: int) -> "Fractal":
        return cls(fam.k, fam.s, r, fam.dim, fam.table())

    @classmethod
    def mixed(cls, s: int, dim: int, tables) -> "Fractal":
        """``fractal_create_mixed``: level mu (mu = 0 the finest) uses
        ``tables[mu]`` (k_mu x dim offsets); r = len(tables)."""
        tabs = [np.asarray(t, dtype=np.int32).reshape(-1, dim) for t in tables]
        ks = np.ascontiguousarray(np.array([len(t) for t in tabs], dtype=np.int32))
        off = np.ascontiguousarray(np.concatenate([t.reshape(-1) for t in tabs]).astype(np.int32))
        self = cls.__new__(cls)
        self._lib = capi.load()
        h = capi.c_fp()
        capi.check(self._lib.fractal_create_mixed(s, len(tabs), dim, ks.ctypes.data_as(capi.c_i32p),
                                                  off.ctypes.data_as(capi.c_i32p), ctypes.byref(h)), self._lib)
        self._h = h
        self.k, self.s, self.r, self.dim = int(ks[0]), s, len(tabs), dim
        self.offsets = tabs[0].copy()
        self.level_tables = [t.copy() for t in tabs]
        cells, side = ctypes.c_int64(), ctypes.c_int64()
        capi.check(self._lib.fractal_info(h, ctypes.byref(cells), ctypes.byref(side)), self._lib)
        self.cells, self.side = cells.value, side.value
        self.box_cells = self.side ** dim
        return self

    # ------------------------------------------------------------ lifetime
    def close(self):
        if getattr(self, "_h", None):
            self._lib.fractal_destroy(self._h)
            self._h = None

    def __del__(self):  # pragma: no cover
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def _check(self, rc):
        return capi.check(rc, self._lib)

    # -------------------------------------------------------------- maps
    def lam(self, omega: torch.Tensor, out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
        n = omega.numel()
        out = out if out is not None else torch.empty((n, self.dim), dtype=torch.int32, device=omega.device)
        self._check(self._lib.fractal_lambda(self._h, _dev_ptr(omega, torch.int64, "omega"), n,
                                             _dev_ptr(out, torch.int32, "coords"), _stream(stream)))
        return out

    def nu(self, coords: torch.Tensor, out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
        n = coords.numel() // self.dim
        out = out if out is not None else torch.empty(n, dtype=torch.int64, device=coords.device)
        self._check(self._lib.fractal_nu(self._h, _dev_ptr(coords, torch.int32, "coords"), n,
                                         _dev_ptr(out, torch.int64, "omega"), _stream(stream)))
        return out

    def lam_tc(self, omega: torch.Tensor, out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
        """``fractal_lambda_tc``: lambda with its level sums on the tensor cores."""
        n = omega.numel()
        out = out if out is not None else torch.empty((n, self.dim), dtype=torch.int32, device=omega.device)
        self._check(self._lib.fractal_lambda_tc(self._h, _dev_ptr(omega, torch.int64, "omega"), n,
                                                _dev_ptr(out, torch.int32, "coords"), _stream(stream)))
        return out

    def nu_tc(self, coords: torch.Tensor, compact: bool = False, stream=None):
        """``fractal_nu_tc``: nu (and, with ``compact``, the compact coordinate of
        ``nu2d``) with the level sums on the tensor cores."""
        n = coords.shape[0]
        om = torch.empty(n, dtype=torch.int64, device=coords.device)
        c2 = torch.empty((n, self.dim), dtype=torch.int64, device=coords.device) if compact else None
        self._check(self._lib.fractal_nu_tc(self._h, _dev_ptr(coords, torch.int32, "coords"), n,
                                            om.data_ptr(), c2.data_ptr() if c2 is not None else None,
                                            _stream(stream)))
        return (om, c2) if compact else om

    def nu2d(self, coords: torch.Tensor, out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
        n = coords.numel() // self.dim
        out = out if out is not None else torch.empty((n, self.dim), dtype=torch.int64, device=coords.device)
        self._check(self._lib.fractal_nu2d(self._h, _dev_ptr(coords, torch.int32, "coords"), n,
                                           _dev_ptr(out, torch.int64, "compact"), _stream(stream)))
        return out

    # ------------------------------------------------------------- states
    def empty_state(self, device="cuda") -> torch.Tensor:
        return torch.empty(self.cells, dtype=torch.uint8, device=device)

    def init_bernoulli(self, seed: int, p: float, out: torch.Tensor | None = None, stream=None):
        out = out if out is not None else self.empty_state()
        self._check(self._lib.fractal_init_bernoulli(self._h, _dev_ptr(out, torch.uint8, "state"),
                                                     seed & (2**64 - 1), float(p), _stream(stream)))
        return out

    def step(self, state: torch.Tensor, out: torch.Tensor | None = None, steps: int = 1,
             rule=None, stream=None) -> torch.Tensor:
        birth, survive = rule if rule is not None else self.default_rule()
        out = out if out is not None else torch.empty_like(state)
        self._check(self._lib.fractal_step(self._h, _dev_ptr(state, torch.uint8, "state_in"),
                                           _dev_ptr(out, torch.uint8, "state_out"), steps,
                                           birth, survive, _stream(stream)))
        return out

    def bb_step(self, box: torch.Tensor, out: torch.Tensor | None = None, steps: int = 1,
                rule=None, stream=None) -> torch.Tensor:
        birth, survive = rule if rule is not None else self.default_rule()
        out = out if out is not None else torch.empty_like(box)
        self._check(self._lib.fractal_bb_step(self._h, _dev_ptr(box, torch.uint8, "box_in"),
                                              _dev_ptr(out, torch.uint8, "box_out"), steps,
                                              birth, survive, _stream(stream)))
        return out

    def scatter(self, compact: torch.Tensor, out: torch.Tensor | None = None, stream=None):
        out = out if out is not None else torch.empty(self.box_cells, dtype=torch.uint8, device=compact.device)
        self._check(self._lib.fractal_scatter_to_box(self._h, _dev_ptr(compact, torch.uint8, "compact"),
                                                     _dev_ptr(out, torch.uint8, "box"), _stream(stream)))
        return out

    def gather(self, box: torch.Tensor, out: torch.Tensor | None = None, stream=None):
        out = out if out is not None else torch.empty(self.cells, dtype=torch.uint8, device=box.device)
        self._check(self._lib.fractal_gather_from_box(self._h, _dev_ptr(box, torch.uint8, "box"),
                                                      _dev_ptr(out, torch.uint8, "compact"), _stream(stream)))
        return out

    def run_host(self, host_in: torch.Tensor, host_out: torch.Tensor, steps: int = 1, rule=None,
                 stream=None):
        """End-to-end call from host buffers (``fractal_run_host``)."""
        birth, survive = rule if rule is not None else self.default_rule()
        for t, name in ((host_in, "host_in"), (host_out, "host_out")):
            if t.is_cuda or t.dtype != torch.uint8 or not t.is_contiguous() or t.numel() != self.cells:
                raise TypeError(f"{name} must be a contiguous host uint8 tensor of {self.cells} cells")
        self._check(self._lib.fractal_run_host(self._h, host_in.data_ptr(), host_out.data_ptr(), steps,
                                               birth, survive, _stream(stream)))
        return host_out

    # ------------------------------------------------------------- tuning
    @property
    def tile_levels(self) -> int:
        v = ctypes.c_int()
        self._check(self._lib.fractal_get_tile_levels(self._h, ctypes.byref(v)))
        return v.value

    @tile_levels.setter
    def tile_levels(self, levels: int):
        self._check(self._lib.fractal_set_tile_levels(self._h, int(levels)))

    # ------------------------------------------- the paper's approaches
    def lambda_box_step(self, box: torch.Tensor, rho_levels: int, out: torch.Tensor | None = None,
                        steps: int = 1, rule=None, stream=None) -> torch.Tensor:
        """``fractal_lambda_box_step``: the paper's lambda(omega) approach on a
        box whose cells off the fractal are 0."""
        rule = rule or self.default_rule()
        out = out if out is not None else torch.zeros_like(box)
        self._check(self._lib.fractal_lambda_box_step(self._h, int(rho_levels), _dev_ptr(box, torch.uint8, "box"),
                                                      _dev_ptr(out, torch.uint8, "out"), steps, rule[0], rule[1],
                                                      _stream(stream)))
        return out

    def blocked_bytes(self, rho_levels: int) -> int:
        v = ctypes.c_int64()
        self._check(self._lib.fractal_blocked_info(self._h, int(rho_levels), ctypes.byref(v)))
        return v.value

    def blocked_pack(self, compact: torch.Tensor, rho_levels: int, stream=None) -> torch.Tensor:
        out = torch.empty(self.blocked_bytes(rho_levels), dtype=torch.uint8, device=compact.device)
        self._check(self._lib.fractal_blocked_pack(self._h, int(rho_levels), _dev_ptr(compact, torch.uint8, "compact"),
                                                   out.data_ptr(), _stream(stream)))
        return out

    def blocked_unpack(self, blocked: torch.Tensor, rho_levels: int, stream=None) -> torch.Tensor:
        out = torch.empty(self.cells, dtype=torch.uint8, device=blocked.device)
        self._check(self._lib.fractal_blocked_unpack(self._h, int(rho_levels), _dev_ptr(blocked, torch.uint8, "blocked"),
                                                     out.data_ptr(), _stream(stream)))
        return out

    def blocked_step(self, blocked: torch.Tensor, rho_levels: int, out: torch.Tensor | None = None, steps: int = 1,
                     rule=None, stream=None) -> torch.Tensor:
        """``fractal_blocked_step``: the paper's nu(omega) approach on blocked storage."""
        rule = rule or self.default_rule()
        out = out if out is not None else torch.empty_like(blocked)
        self._check(self._lib.fractal_blocked_step(self._h, int(rho_levels), _dev_ptr(blocked, torch.uint8, "blocked"),
                                                   _dev_ptr(out, torch.uint8, "out"), steps, rule[0], rule[1],
                                                   _stream(stream)))
        return out

    def set_temporal_blocking(self, generations: int, tile_levels: int = -1):
        """``fractal_set_temporal_blocking``: up to ``generations`` (1..9)
        generations per pass of ``step``; 0 turns it off."""
        self._check(self._lib.fractal_set_temporal_blocking(self._h, int(generations), int(tile_levels)))

    @property
    def pipeline_stages(self) -> int:
        """Input pipeline stages of the step's plan (``fractal_plan_info``)."""
        return self.plan_info()["stages"]

    @pipeline_stages.setter
    def pipeline_stages(self, stages: int):
        self._check(self._lib.fractal_set_pipeline_stages(self._h, int(stages)))

    POLICIES = {0: "cell", 3: "group3", 4: "group4", 9: "quad", 10: "tap", 11: "rows_carpet", 12: "rows_vicsek", 13: "lid_vicsek", 14: "box3", 15: "bit3"}

    def plan_info(self) -> dict:
        """The step's launch plan (``fractal_plan_info``)."""
        v = (ctypes.c_int32 * 7)()
        self._check(self._lib.fractal_plan_info(self._h, v, 7))
        keys = ("policy", "tile_levels", "block", "grid", "smem_bytes", "stages", "blocks_per_sm")
        d = dict(zip(keys, (int(x) for x in v)))
        d["policy_name"] = self.POLICIES.get(d["policy"], str(d["policy"]))
        return d

    def autotune(self, state: torch.Tensor, out: torch.Tensor | None = None, rule=None,
                 stream=None) -> int:
        """Pick the fastest tile depth on these buffers (``fractal_autotune``);
        ``out`` is overwritten.  Returns the chosen depth."""
        birth, survive = rule if rule is not None else self.default_rule()
        out = out if out is not None else torch.empty_like(state)
        v = ctypes.c_int()
        self._check(self._lib.fractal_autotune(self._h, _dev_ptr(state, torch.uint8, "state_in"),
                                               _dev_ptr(out, torch.uint8, "state_out"), birth, survive,
                                               _stream(stream), ctypes.byref(v)))
        return v.value

    def default_rule(self):
        return (0x20, 0x30) if self.dim == 3 else LIFE_B3S23

    def sync(self, stream=None):
        self._check(self._lib.fractal_sync(_stream(stream)))

    def check(self):
        """Raise if a bounded device-side wait of this handle gave up."""
        self._check(self._lib.fractal_check(self._h))


class Batch:
    """Many independent instances advanced together (``fractal_batch_*``).

    ``add(fractal, state_in, state_out, steps, rule)`` queues an instance;
    ``run()`` advances all of them, each exactly as ``Fractal.step`` would,
    with one launch per generation for each group of instances that share a
    fractal and tile depth, replayed from a captured CUDA graph."""

    def __init__(self):
        self._lib = capi.load()
        h = ctypes.c_void_p()
        capi.check(self._lib.fractal_batch_create(ctypes.byref(h)), self._lib)
        self._h = h
        self._keep = []   # tensors and handles that must outlive the runs

    def add(self, fr: Fractal, state: torch.Tensor, out: torch.Tensor, steps: int, rule=None) -> int:
        birth, survive = rule if rule is not None else fr.default_rule()
        idx = ctypes.c_int64()
        capi.check(self._lib.fractal_batch_add(self._h, fr._h, _dev_ptr(state, torch.uint8, "state"),
                                               _dev_ptr(out, torch.uint8, "out"), steps, birth, survive,
                                               ctypes.byref(idx)), self._lib)
        self._keep.append((fr, state, out))
        return idx.value

    def run(self, stream=None):
        capi.check(self._lib.fractal_batch_run(self._h, _stream(stream)), self._lib)

    def clear(self):
        capi.check(self._lib.fractal_batch_clear(self._h), self._lib)
        self._keep = []

    def stats(self):
        u, l = ctypes.c_int64(), ctypes.c_int64()
        capi.check(self._lib.fractal_batch_stats(self._h, ctypes.byref(u), ctypes.byref(l)), self._lib)
        return u.value, l.value

    def close(self):
        if getattr(self, "_h", None):
            self._lib.fractal_batch_destroy(self._h)
            self._h = None

    def __del__(self):  # pragma: no cover
        try:
            self.close()
        except Exception:
            pass


class Server:
    """Continuous-batching request server (``fractal_server_*``)."""

    def __init__(self, hbm_budget_bytes: int = 0, chunk: int = 8):
        self._lib = capi.load()
        h = ctypes.c_void_p()
        capi.check(self._lib.fractal_server_create(int(hbm_budget_bytes), int(chunk), ctypes.byref(h)),
                   self._lib)
        self._h = h
        self._keep = {}

    def submit(self, fr: Fractal, seed: int, p: float, steps: int, rule=None,
               host_out: torch.Tensor | None = None) -> int:
        birth, survive = rule if rule is not None else fr.default_rule()
        ptr = None
        if host_out is not None:
            if host_out.is_cuda or host_out.dtype != torch.uint8 or host_out.numel() != fr.cells:
                raise TypeError("host_out must be a host uint8 tensor of k^r cells")
            ptr = host_out.data_ptr()
        rid = ctypes.c_int64()
        capi.check(self._lib.fractal_server_submit(self._h, fr._h, seed & (2**64 - 1), float(p), int(steps),
                                                   birth, survive, ptr, ctypes.byref(rid)), self._lib)
        self._keep[rid.value] = (fr, host_out)
        return rid.value

    def poll(self, rid: int):
        """(done, latency_s, population)."""
        d, lat, pop = ctypes.c_int(), ctypes.c_double(), ctypes.c_int64()
        capi.check(self._lib.fractal_server_poll(self._h, rid, ctypes.byref(d), ctypes.byref(lat),
                                                 ctypes.byref(pop)), self._lib)
        return bool(d.value), lat.value, pop.value

    def wait_all(self):
        capi.check(self._lib.fractal_server_wait_all(self._h), self._lib)

    def stats(self) -> dict:
        v = [ctypes.c_int64() for _ in range(6)]
        capi.check(self._lib.fractal_server_stats(self._h, *[ctypes.byref(x) for x in v]), self._lib)
        keys = ["completed", "queued", "resident", "cell_updates", "launches", "hbm_used"]
        return dict(zip(keys, (x.value for x in v)))

    def close(self):
        if getattr(self, "_h", None):
            self._lib.fractal_server_destroy(self._h)
            self._h = None
            self._keep = {}

    def __del__(self):  # pragma: no cover
        try:
            self.close()
        except Exception:
            pass
