"""Python front end of the D2Q37 library: a lattice whose state lives in HBM.

PyTorch supplies device memory and the stream; every step of the method runs
in liblbm.so's CUDA kernels (include/lbm.h documents each call).
"""
from __future__ import annotations

import ctypes

import numpy as np
import torch

from . import _lib as L

NPOP = 37
HALO = 3


def _ptr(t):
    if t is None:
        return None
    if not isinstance(t, torch.Tensor):
        raise TypeError("expected a torch tensor")
    if not t.is_contiguous():
        raise ValueError("tensor must be contiguous")
    return ctypes.c_void_p(t.data_ptr())


def _check_tensor(t, name, dtype, shape, device):
    """Reject a tensor the kernels cannot take: every state, cotangent and
    field pointer handed to liblbm.so (except the host-or-device checkpoint
    copies) must be contiguous memory of the lattice's own GPU with the
    expected dtype and shape.  A host pointer given to a kernel would be
    dereferenced on the device, so this check runs before any call."""
    if not isinstance(t, torch.Tensor):
        raise TypeError(f"{name}: expected a torch tensor, got {type(t).__name__}")
    if t.device != device:
        raise ValueError(f"{name}: tensor on {t.device}, the lattice lives on {device}")
    if t.dtype != dtype:
        raise ValueError(f"{name}: dtype {t.dtype}, expected {dtype}")
    if tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name}: shape {tuple(t.shape)}, expected {tuple(shape)}")
    if not t.is_contiguous():
        raise ValueError(f"{name}: tensor must be contiguous")
    return t


def _field(v, ly, lx, device):
    """A float64 (ly, lx) contiguous device tensor from a tensor or array."""
    if isinstance(v, torch.Tensor):
        t = v.to(device=device, dtype=torch.float64)
    else:
        t = torch.as_tensor(np.asarray(v, dtype=np.float64), device=device)
    t = t.contiguous()
    if tuple(t.shape) != (ly, lx):
        raise ValueError(f"field shape {tuple(t.shape)} != {(ly, lx)}")
    return t


class Lattice:
    """One D2Q37 lattice with walls at the top and bottom rows and periodic x.

    State buffers are (37, ly + 6, lx) tensors (three halo rows on each side,
    x fastest); dtype float64, or float32 holding f_l - w_l rho0 when
    ``precision="fp32"``.  ``fp32_arith`` selects the arithmetic of the
    float32-store collide: "split" (default), "fp64_terms" (float64 moment
    sums and temperature-dependent equilibrium terms) or "fp64_collide" (the
    float64 collide on the decoded populations).
    """

    FP32_ARITH = {"split": 0, "fp64_terms": L.LBM_FLAG_FP32_F64_TERMS,
                  "fp64_collide": L.LBM_FLAG_FP32_F64_COLLIDE}

    def __init__(self, lx: int, ly: int, tau: float, g: float = 0.0, t_top: float = 1.0,
                 t_bottom: float = 1.0, precision: str = "fp64", rho0: float = 1.0,
                 periodic_y: bool = False, regularized: bool = False, tma_loads: bool = False,
                 fp32_arith: str = "split", device=None, stream=None):
        self.lib = L.load()
        if not torch.cuda.is_available():
            raise RuntimeError("a CUDA device is required")
        dev = torch.device(device if device is not None else "cuda")
        if dev.type != "cuda":
            raise ValueError(f"device {dev} is not a CUDA device")
        self.device = dev if dev.index is not None else torch.device("cuda", torch.cuda.current_device())
        self.lx, self.ly = int(lx), int(ly)
        self.precision = precision
        prec = {"fp64": L.LBM_FP64, "fp32": L.LBM_FP32_SHIFTED, "fp64df": L.LBM_FP64_DF}[precision]
        self.dtype = torch.float32 if prec == L.LBM_FP32_SHIFTED else torch.float64
        flags = ((L.LBM_FLAG_PERIODIC_Y if periodic_y else 0) | (L.LBM_FLAG_REGULARIZED if regularized else 0)
                 | (L.LBM_FLAG_TMA_LOADS if tma_loads else 0) | self.FP32_ARITH[fp32_arith])
        self.params = L.LbmParams(self.lx, self.ly, prec, flags,
                                  float(tau), float(g), float(t_top), float(t_bottom), float(rho0))
        self.tau, self.g, self.t_top, self.t_bottom, self.rho0 = tau, g, t_top, t_bottom, rho0
        self.periodic_y = periodic_y
        nbytes = self.lib.lbm_state_bytes(ctypes.byref(self.params))
        if nbytes == 0:
            raise L.LBMError(L.LBM_ERR_INVALID, "invalid lattice parameters")
        self.nbytes = nbytes
        self.shape = (NPOP, self.ly + 2 * HALO, self.lx)
        self.buffers = [torch.full(self.shape, float("nan"), dtype=self.dtype, device=self.device)
                        for _ in range(2)]
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        ctx = ctypes.c_void_p()
        rc = self.lib.lbm_create(ctypes.byref(ctx), ctypes.byref(self.params), _ptr(self.buffers[0]),
                                 _ptr(self.buffers[1]), nbytes, ctypes.c_void_p(self.stream.cuda_stream))
        if rc != 0:
            raise L.LBMError(rc, "lbm_create failed (invalid parameters, size or alignment)")
        self.ctx = ctx

    # ------------------------------------------------------------------
    def _check(self, rc):
        if rc != 0:
            msg = self.lib.lbm_last_error(self.ctx)
            raise L.LBMError(rc, msg.decode() if msg else "")

    def close(self):
        if getattr(self, "ctx", None):
            self.lib.lbm_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _state(self, t, name):
        return _check_tensor(t, name, self.dtype, self.shape, self.device)

    def _opt_state(self, t, name):
        return None if t is None else self._state(t, name)

    def _cotangent(self, t, name, dtype=torch.float64):
        return _check_tensor(t, name, dtype, self.shape, self.device)

    def new_state(self, fill=float("nan")):
        return torch.full(self.shape, fill, dtype=self.dtype, device=self.device)

    def new_cotangent(self, fill=float("nan"), dtype=torch.float64):
        """A cotangent buffer in the state layout: float64, or float32 for the
        float32 adjoint of FP32-store lattices (adjoint_step dispatches on it)."""
        if dtype not in (torch.float64, torch.float32):
            raise ValueError(f"cotangent dtype {dtype}: float64 or float32")
        return torch.full((NPOP, self.ly + 2 * HALO, self.lx), fill, dtype=dtype, device=self.device)

    # ------------------------------------------------------------------
    def init(self, rho, ux, uy, T):
        """Current state := f^eq(rho, u, T) (fields (ly, lx))."""
        f = [_field(v, self.ly, self.lx, self.device) for v in (rho, ux, uy, T)]
        self._check(self.lib.lbm_init(self.ctx, *[_ptr(t) for t in f]))
        self._keep = f  # alive until the next call on this stream
        return self

    def step(self, n: int = 1, graph: bool = False):
        """n time steps; graph=True replays them as one cached CUDA graph
        launch (same results; for small lattices, whose steps are shorter
        than a kernel launch)."""
        fn = self.lib.lbm_step_graph if graph else self.lib.lbm_step
        self._check(fn(self.ctx, int(n)))
        return self

    def step_from(self, src: torch.Tensor, dst: torch.Tensor):
        """One step from state src into state dst (context buffers untouched)."""
        self._state(src, "src")
        self._state(dst, "dst")
        self._check(self.lib.lbm_step_from(self.ctx, _ptr(src), _ptr(dst)))
        return dst

    def step_columns(self, src: torch.Tensor, dst: torch.Tensor, x0: int, x1: int):
        """One step from src into dst for the sites of columns x0 <= x < x1."""
        self._state(src, "src")
        self._state(dst, "dst")
        self._check(self.lib.lbm_step_columns(self.ctx, _ptr(src), _ptr(dst), int(x0), int(x1)))
        return dst

    def pack_columns(self, f: torch.Tensor, x0: int, n: int, buf: torch.Tensor):
        """Columns x0 .. x0+n-1 of f's physical rows into buf (37, ly, n)."""
        self._state(f, "f")
        _check_tensor(buf, "buf", self.dtype, (NPOP, self.ly, n), self.device)
        self._check(self.lib.lbm_pack_columns(self.ctx, _ptr(f), int(x0), int(n), _ptr(buf)))
        return buf

    def unpack_columns(self, buf: torch.Tensor, x0: int, n: int, f: torch.Tensor):
        """buf (37, ly, n) into columns x0 .. x0+n-1 of f's physical rows."""
        self._state(f, "f")
        _check_tensor(buf, "buf", self.dtype, (NPOP, self.ly, n), self.device)
        self._check(self.lib.lbm_unpack_columns(self.ctx, _ptr(buf), int(x0), int(n), _ptr(f)))
        return f

    def other(self) -> torch.Tensor:
        """The buffer not holding the current state."""
        cur = self.state()
        return self.buffers[1] if cur is self.buffers[0] else self.buffers[0]

    def swap(self):
        """Make the other buffer current (after a step written into it with
        step_columns): the role change lbm_step makes after each step."""
        self._check(self.lib.lbm_swap(self.ctx))
        return self

    def state(self) -> torch.Tensor:
        """The buffer holding the current state (a view; it changes role at each step)."""
        ptr = self.lib.lbm_current(self.ctx)
        return self.buffers[0] if ptr == self.buffers[0].data_ptr() else self.buffers[1]

    def set_state(self, src: torch.Tensor):
        """Copy a state (device memory, or host memory such as a pinned
        tensor) into the current buffer, asynchronously on the lattice's
        stream."""
        if src.dtype != self.dtype or tuple(src.shape) != self.shape:
            raise ValueError("state dtype/shape mismatch")
        if src.device.type == "cuda" and src.device != self.device:
            raise ValueError(f"src: tensor on {src.device}, the lattice lives on {self.device}")
        src = src.contiguous()
        self._check(self.lib.lbm_set_state(self.ctx, _ptr(src)))
        self._keep = src  # alive until the copy is ordered before later work
        return self

    def get_state(self, dst: torch.Tensor):
        if dst.dtype != self.dtype or tuple(dst.shape) != self.shape or not dst.is_contiguous():
            raise ValueError("state dtype/shape mismatch")
        if dst.device.type == "cuda" and dst.device != self.device:
            raise ValueError(f"dst: tensor on {dst.device}, the lattice lives on {self.device}")
        self._check(self.lib.lbm_get_state(self.ctx, _ptr(dst)))
        return dst

    def moments(self, f: torch.Tensor | None = None):
        self._opt_state(f, "f")
        out = [torch.empty((self.ly, self.lx), dtype=torch.float64, device=self.device) for _ in range(4)]
        self._check(self.lib.lbm_moments(self.ctx, _ptr(f), *[_ptr(t) for t in out]))
        return tuple(out)

    def profiles(self, f: torch.Tensor | None = None) -> torch.Tensor:
        """Row averages (8, ly) of rho, u_x, u_y, T, T^2, u_y T, rho|u|^2/2, rho u_y."""
        self._opt_state(f, "f")
        out = torch.empty((L.LBM_NOBS, self.ly), dtype=torch.float64, device=self.device)
        self._check(self.lib.lbm_profiles(self.ctx, _ptr(f), _ptr(out)))
        return out

    def step_observe(self, n: int, every: int) -> torch.Tensor:
        """n steps; the row averages after every `every`-th step, (n // every, 8, ly)."""
        out = torch.empty((max(1, n // every), L.LBM_NOBS, self.ly), dtype=torch.float64, device=self.device)
        rec = ctypes.c_int(0)
        self._check(self.lib.lbm_step_observe(self.ctx, int(n), int(every), _ptr(out), ctypes.byref(rec)))
        return out[:rec.value]

    def propagate_bc(self, src: torch.Tensor, dst: torch.Tensor | None = None):
        self._state(src, "src")
        if dst is None:
            dst = self.new_state()
        self._state(dst, "dst")
        self._check(self.lib.lbm_propagate_bc(self.ctx, _ptr(src), _ptr(dst)))
        return dst

    def adjoint_step(self, f_t: torch.Tensor, lam_in: torch.Tensor, lam_out: torch.Tensor | None = None):
        """lam_out = P^T B^T C^T lam_in at state f_t; float32 cotangents take
        the float32 adjoint (FP32-store lattices only)."""
        self._state(f_t, "f_t")
        if not isinstance(lam_in, torch.Tensor):
            raise TypeError("lam_in: expected a torch tensor")
        dt = lam_in.dtype
        self._cotangent(lam_in, "lam_in", dt)
        if lam_out is None:
            lam_out = self.new_cotangent(dtype=dt)
        self._cotangent(lam_out, "lam_out", dt)
        fn = self.lib.lbm_adjoint_step_f32 if dt == torch.float32 else self.lib.lbm_adjoint_step
        self._check(fn(self.ctx, _ptr(f_t), _ptr(lam_in), _ptr(lam_out)))
        return lam_out

    def moments_vjp(self, f, g_rho=None, g_ux=None, g_uy=None, g_T=None, lam_out=None, dtype=torch.float64):
        self._state(f, "f")
        if lam_out is None:
            lam_out = self.new_cotangent(dtype=dtype)
        dt = lam_out.dtype if isinstance(lam_out, torch.Tensor) else dtype
        self._cotangent(lam_out, "lam_out", dt)
        gs = [None if g is None else _field(g, self.ly, self.lx, self.device) for g in (g_rho, g_ux, g_uy, g_T)]
        fn = self.lib.lbm_moments_vjp_f32 if dt == torch.float32 else self.lib.lbm_moments_vjp
        self._check(fn(self.ctx, _ptr(f), *[_ptr(g) for g in gs], _ptr(lam_out)))
        self._keep = gs
        return lam_out

    def init_vjp(self, rho, ux, uy, T, lam):
        f = [_field(v, self.ly, self.lx, self.device) for v in (rho, ux, uy, T)]
        if not isinstance(lam, torch.Tensor):
            raise TypeError("lam: expected a torch tensor")
        self._cotangent(lam, "lam", lam.dtype if lam.dtype == torch.float32 else torch.float64)
        out = [torch.empty((self.ly, self.lx), dtype=torch.float64, device=self.device) for _ in range(4)]
        fn = self.lib.lbm_init_vjp_f32 if lam.dtype == torch.float32 else self.lib.lbm_init_vjp
        self._check(fn(self.ctx, *[_ptr(t) for t in f], _ptr(lam), *[_ptr(t) for t in out]))
        self._keep = f
        return tuple(out)

    def check_finite(self, f: torch.Tensor | None = None) -> bool:
        self._opt_state(f, "f")
        ok = ctypes.c_int(0)
        self._check(self.lib.lbm_check_finite(self.ctx, _ptr(f), ctypes.byref(ok)))
        return bool(ok.value)

    def status(self) -> int:
        return self.lib.lbm_status(self.ctx)

    def step_path(self) -> str:
        """'tma' when step() stages the pull sources with TMA loads, else 'plain'."""
        rc = self.lib.lbm_step_path(self.ctx)
        if rc < 0:
            raise L.LBMError(rc, "lbm_step_path")
        return "tma" if rc == L.LBM_PATH_TMA else "plain"

    def constants(self):
        r = ctypes.c_double()
        arrs = [(ctypes.c_double * NPOP)() for _ in range(3)]
        self._check(self.lib.lbm_constants(self.ctx, ctypes.byref(r), *arrs))
        return r.value, *[np.array(a[:]) for a in arrs]
