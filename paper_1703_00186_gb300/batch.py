"""Many independent D2Q37 lattices stepped by one CUDA graph (include/lbm_batch.h).

Each lattice has its own size, tau, g, wall temperatures and FP32 shift; one
batch step is one kernel over a tile work list spanning all lattices, and n
steps are one graph launch.  PyTorch only owns the buffers and the stream.
"""
from __future__ import annotations

import ctypes

import numpy as np
import torch

from . import _lib as L
from .lbm import HALO, NPOP, _field, _ptr


class Batch:
    def __init__(self, specs, precision: str = "fp32", device=None, stream=None):
        """specs: sequence of dicts with lx, ly, tau, g, t_top, t_bottom, rho0."""
        self.lib = L.load()
        if not torch.cuda.is_available():
            raise RuntimeError("a CUDA device is required")
        self.device = torch.device(device if device is not None else "cuda")
        prec = {"fp64": L.LBM_FP64, "fp32": L.LBM_FP32_SHIFTED, "fp64df": L.LBM_FP64_DF}[precision]
        self.precision = precision
        self.dtype = torch.float32 if prec == L.LBM_FP32_SHIFTED else torch.float64
        self.specs = [dict(s) for s in specs]
        self.buffers = []
        descs = (L.LbmLatticeDesc * len(self.specs))()
        for i, s in enumerate(self.specs):
            shape = (NPOP, int(s["ly"]) + 2 * HALO, int(s["lx"]))
            fa = torch.full(shape, float("nan"), dtype=self.dtype, device=self.device)
            fb = torch.full(shape, float("nan"), dtype=self.dtype, device=self.device)
            self.buffers.append((fa, fb))
            descs[i] = L.LbmLatticeDesc(int(s["lx"]), int(s["ly"]), float(s["tau"]), float(s.get("g", 0.0)),
                                        float(s.get("t_top", 1.0)), float(s.get("t_bottom", 1.0)),
                                        float(s.get("rho0", 1.0)), fa.data_ptr(), fb.data_ptr())
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        h = ctypes.c_void_p()
        rc = self.lib.lbm_batch_create(ctypes.byref(h), len(self.specs), descs, prec,
                                       ctypes.c_void_p(self.stream.cuda_stream))
        if rc != 0:
            raise L.LBMError(rc, "lbm_batch_create failed")
        self.h = h

    def _check(self, rc):
        if rc != 0:
            msg = self.lib.lbm_batch_last_error(self.h)
            raise L.LBMError(rc, msg.decode() if msg else "")

    def close(self):
        if getattr(self, "h", None):
            self.lib.lbm_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __len__(self):
        return len(self.specs)

    @property
    def sites(self) -> int:
        return int(self.lib.lbm_batch_sites(self.h))

    def init(self, i, rho, ux, uy, T):
        s = self.specs[i]
        f = [_field(v, int(s["ly"]), int(s["lx"]), self.device) for v in (rho, ux, uy, T)]
        self._check(self.lib.lbm_batch_init(self.h, int(i), *[_ptr(t) for t in f]))
        torch.cuda.current_stream(self.device).synchronize()
        return self

    @staticmethod
    def tile_shapes():
        """(threads along x, threads along y, sites per thread along y) of every
        launch candidate the autotuner chooses from: the tile shapes of the
        one-launch batch kernel, then the per-lattice launches."""
        lib = L.load()
        out = []
        for i in range(lib.lbm_batch_tile_count()):
            bx, by = ctypes.c_int(), ctypes.c_int()
            lib.lbm_batch_tile_shape(i, ctypes.byref(bx), ctypes.byref(by))
            out.append((bx.value, by.value, lib.lbm_batch_tile_rows(i)))
        return out

    @staticmethod
    def tile_labels():
        """A name for every launch candidate ("32x4x8" for a shared-memory tile
        shape, "per-lattice 32x4" for the per-lattice launches, "params
        32x4x8" for a tile shape of the parameter-table kernel)."""
        lib = L.load()
        out = []
        for i, (bx, by, rows) in enumerate(Batch.tile_shapes()):
            kind = lib.lbm_batch_tile_kind(i)
            if kind == L.LBM_BATCH_PER_LATTICE:
                out.append(f"per-lattice {bx}x{by}")
            elif kind == L.LBM_BATCH_PARAM_TILES:
                out.append(f"params {bx}x{by}x{rows}")
            else:
                out.append(f"{bx}x{by}x{rows}")
        return out

    def set_tile(self, t: int):
        self._check(self.lib.lbm_batch_set_tile(self.h, int(t)))
        return self

    def autotune(self, steps: int = 5):
        n = self.lib.lbm_batch_tile_count()
        times = (ctypes.c_double * n)()
        best = ctypes.c_int()
        self._check(self.lib.lbm_batch_autotune(self.h, int(steps), ctypes.byref(best), times))
        return best.value, list(times)

    def step(self, n: int = 1):
        self._check(self.lib.lbm_batch_step(self.h, int(n)))
        return self

    def step_persistent(self, n: int = 1):
        """n steps in one persistent cooperative launch (bounded grid barrier)."""
        self._check(self.lib.lbm_batch_step_persistent(self.h, int(n)))
        return self

    def barrier_selftest(self, budget_ms: int = 20) -> int:
        """Return code of the bounded-wait self-test (LBM_ERR_TIMEOUT expected)."""
        return self.lib.lbm_batch_barrier_selftest(self.h, int(budget_ms))

    def state(self, i) -> torch.Tensor:
        ptr = self.lib.lbm_batch_current(self.h, int(i))
        fa, fb = self.buffers[i]
        return fa if ptr == fa.data_ptr() else fb

    def moments(self, i):
        s = self.specs[i]
        out = [torch.empty((int(s["ly"]), int(s["lx"])), dtype=torch.float64, device=self.device)
               for _ in range(4)]
        self._check(self.lib.lbm_batch_moments(self.h, int(i), *[_ptr(t) for t in out]))
        return tuple(out)

    def status(self) -> int:
        return self.lib.lbm_batch_status(self.h)
