"""Thin Python binding of libenomr.so (argument marshalling only).

Every computation runs in the CUDA kernels of the library; this module only
checks tensors, passes device pointers and the current torch stream, and
turns status codes into exceptions.  There is no CPU fallback: importing this
module fails if the compiled library is missing.

C ABI: include/enomr.h.
"""
from __future__ import annotations

import ctypes
import os

import torch

ADVECTION, EULER, BURGERS = 0, 1, 2
SIDE_TRANSMISSIVE, SIDE_REFLECTIVE, SIDE_INFLOW = 1, 2, 3
_SIDE_KINDS = {"transmissive": SIDE_TRANSMISSIVE, "reflective": SIDE_REFLECTIVE,
               "inflow": SIDE_INFLOW}


class _Side(ctypes.Structure):
    _fields_ = [("kind_lo", ctypes.c_int), ("kind_hi", ctypes.c_int),
                ("split0", ctypes.c_double), ("split_rate", ctypes.c_double),
                ("state_lo", ctypes.c_double * 4), ("state_hi", ctypes.c_double * 4)]
PERIODIC, TRANSMISSIVE = 0, 1
ORDERS = (5, 7, 9, 11, 13, 15, 17)
# staging of the 2D sweeps' tiles (enomr_set_staging)
STAGING_AUTO, STAGING_LOADS, STAGING_TMA = 0, 1, 2
# instance of the 2D sweeps (enomr_set_occupancy)
OCCUPANCY_AUTO, OCCUPANCY_HIGH, OCCUPANCY_LOW = 0, 1, 2

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libenomr.so")

if not os.path.exists(LIB_PATH):
    raise ImportError(f"{LIB_PATH} is missing: run __graft_entry__.build() first "
                      "(the ENO-MR path has no CPU fallback)")

_lib = ctypes.CDLL(LIB_PATH)
_P, _I, _D, _L = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_int64
_SIGS = {
    "enomr_init": (_I, [ctypes.POINTER(_P), _I, _I, _L, _L, _D, _D, _I, _D, _I, _D, _P]),
    "enomr_free": (None, [_P]),
    "enomr_strerror": (ctypes.c_char_p, [_I]),
    "enomr_set_stream": (_I, [_P, _P]),
    "enomr_rhs": (_I, [_P, _P, _P]),
    "enomr_stage": (_I, [_P, _I, _P, _P, _P, _D]),
    "enomr_step": (_I, [_P, _P, _D, _D, _P]),
    "enomr_cfl_dt": (_I, [_P, _P, _D, _P]),
    "enomr_step_lssp": (_I, [_P, _P, _D, _I]),
    "enomr_debug_selection": (_I, [_P, _P, _P]),
    "enomr_get_status": (_I, [_P]),
    "enomr_num_tested": (_I, [_I]),
    "enomr_profile_begin": (_I, [_P, _I, _I]),
    "enomr_profile_end": (_I, [_P, ctypes.POINTER(_I), ctypes.POINTER(_D)]),
    "enomr_probe_fp64_fma": (_I, [_P, ctypes.c_int64, _P, ctypes.POINTER(_D),
                                 ctypes.POINTER(_D)]),
    "enomr_rhs_euler2d_noalloc": (_I, [_P, _P, _L, _L, _D, _D, _I, _D, _I, _P]),
    "enomr_rhs_vjp": (_I, [_P, _P, _P, _P, _D, _I]),
    "enomr_step_vjp": (_I, [_P, _P, _D, _P, _P]),
    "enomr_step_vjp_cfl": (_I, [_P, _P, _D, _P, _P]),
    "enomr_debug_alpha": (_I, [_P, _P, _P, _P, _P, _P, _P]),
    "enomr_batch_init": (_I, [ctypes.POINTER(_P), _L, _P, _P, _I, _D, _I, _P]),
    "enomr_batch_free": (None, [_P]),
    "enomr_batch_set_stream": (_I, [_P, _P]),
    "enomr_batch_total_cells": (_L, [_P]),
    "enomr_batch_step": (_I, [_P, _P, _D]),
    "enomr_batch_autotune": (_I, [_P, _P, _I, ctypes.POINTER(_I), ctypes.POINTER(_I)]),
    "enomr_batch_get_status": (_I, [_P]),
    "enomr_batch_config": (_I, [_P, ctypes.POINTER(_I), ctypes.POINTER(_I), ctypes.POINTER(_I)]),
    "enomr_set_side": (_I, [_P, _I, _P]),
    "enomr_set_body_force": (_I, [_P, _D, _D]),
    "enomr_set_time": (_I, [_P, _D]),
    "enomr_get_time": (_I, [_P, ctypes.POINTER(_D)]),
    "enomr_set_staging": (_I, [_P, _I]),
    "enomr_stage_frozen": (_I, [_P, _I, _P, _P, _P, _D, _P]),
    "enomr_set_occupancy": (_I, [_P, _I]),
}
for _name, (_res, _args) in _SIGS.items():
    _fn = getattr(_lib, _name)
    _fn.restype = _res
    _fn.argtypes = _args

EXPORTED = tuple(_SIGS)


class EnomrError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        super().__init__(f"{where}: {_lib.enomr_strerror(code).decode()} (status {code})")


def _check(code: int, where: str):
    if code != 0:
        raise EnomrError(code, where)


def num_tested(order: int) -> int:
    return _lib.enomr_num_tested(order)


def probe_fp64_fma(iters: int = 20000, device=None):
    """Measured FP64 FMA throughput of the device in flop/s."""
    dev = torch.device(device if device is not None else "cuda")
    sink = torch.zeros(8 * 1024, dtype=torch.float64, device=dev)
    sec, fl = ctypes.c_double(), ctypes.c_double()
    s = torch.cuda.current_stream(dev).cuda_stream
    _check(_lib.enomr_probe_fp64_fma(_P(s), int(iters), _P(sink.data_ptr()), ctypes.byref(sec),
                                     ctypes.byref(fl)), "enomr_probe_fp64_fma")
    return fl.value / sec.value, sec.value


class Solver:
    """One ENO-MR problem on one GPU.

    eq: ADVECTION (1D, f = adv_speed * u), BURGERS (1D, f = u^2/2) or EULER
    (1D: shape = nx, state [3, nx]; 2D: shape = (ny, nx), state
    [4, ny, nx]).  States are float64 CUDA tensors, contiguous.
    """

    def __init__(self, eq, shape, order=9, dx=1.0, dy=None, bc=TRANSMISSIVE, gamma=1.4,
                 adv_speed=1.0, device=None):
        if isinstance(shape, int):
            ndim, ny, nx = 1, 1, shape
        else:
            ndim, (ny, nx) = 2, shape
        self.eq, self.ndim, self.nx, self.ny, self.order = eq, ndim, nx, ny, order
        self.bc = bc
        self.device = torch.device(device if device is not None else "cuda")
        if self.device.type != "cuda":
            raise ValueError("the ENO-MR solver runs on CUDA devices only")
        scalar = eq in (ADVECTION, BURGERS)
        self.ncomp = 1 if scalar else (4 if ndim == 2 else 3)
        self.state_shape = ((nx,) if scalar else ((3, nx) if ndim == 1 else (4, ny, nx)))
        ctx = _P()
        with torch.cuda.device(self.device):
            stream = torch.cuda.current_stream(self.device).cuda_stream
            _check(_lib.enomr_init(ctypes.byref(ctx), eq, ndim, nx, ny, dx,
                                   dy if dy is not None else dx, order, gamma, bc, adv_speed,
                                   _P(stream)), "enomr_init")
        self._ctx = ctx

    # -- helpers ----------------------------------------------------------
    def _stream(self):
        s = torch.cuda.current_stream(self.device).cuda_stream
        _check(_lib.enomr_set_stream(self._ctx, _P(s)), "enomr_set_stream")

    def _state(self, U, name="U"):
        if not isinstance(U, torch.Tensor) or U.dtype != torch.float64:
            raise TypeError(f"{name} must be a float64 tensor")
        if U.device != self.device and not (U.device.type == "cuda" and self.device.index is None):
            raise ValueError(f"{name} must live on {self.device}")
        if tuple(U.shape) != self.state_shape or not U.is_contiguous():
            raise ValueError(f"{name} must be contiguous with shape {self.state_shape}")
        return _P(U.data_ptr())

    def n_sel(self):
        if self.eq in (ADVECTION, BURGERS):
            return 2 * (self.nx + 1)
        if self.ndim == 1:
            return 6 * (self.nx + 1)
        return 8 * self.ny * (self.nx + 1) + 8 * self.nx * (self.ny + 1)

    # -- API --------------------------------------------------------------
    def rhs(self, U, out=None):
        pu = self._state(U)
        if out is None:
            out = torch.empty_like(U)
        po = self._state(out, "out")
        self._stream()
        _check(_lib.enomr_rhs(self._ctx, pu, po), "enomr_rhs")
        return out

    def stage(self, s, Un, Us, out, dt):
        self._stream()
        _check(_lib.enomr_stage(self._ctx, s, self._state(Un), self._state(Us),
                                self._state(out, "out"), float(dt)), "enomr_stage")
        return out

    def stage_frozen(self, s, Un, Us, out, dt, Uref):
        """Stage s with the discrete choices (stencils, minmod branches, alpha
        argmax cells) of the reference state Uref (enomr_stage_frozen)."""
        self._stream()
        _check(_lib.enomr_stage_frozen(self._ctx, s, self._state(Un), self._state(Us),
                                       self._state(out, "out"), float(dt),
                                       self._state(Uref, "Uref")), "enomr_stage_frozen")
        return out

    def step(self, U, dt=0.0, cfl=0.5, return_dt=False):
        pu = self._state(U)
        self._stream()
        if return_dt:
            d = ctypes.c_double()
            _check(_lib.enomr_step(self._ctx, pu, float(dt), float(cfl), ctypes.byref(d)),
                   "enomr_step")
            return d.value
        _check(_lib.enomr_step(self._ctx, pu, float(dt), float(cfl), None), "enomr_step")
        return None

    def step_lssp(self, U, dt, m):
        """One linear SSP-RK(m, m-1) step of size dt, in place."""
        self._stream()
        _check(_lib.enomr_step_lssp(self._ctx, self._state(U), float(dt), int(m)),
               "enomr_step_lssp")

    def cfl_dt(self, U, cfl=0.5):
        d = ctypes.c_double()
        self._stream()
        _check(_lib.enomr_cfl_dt(self._ctx, self._state(U), float(cfl), ctypes.byref(d)),
               "enomr_cfl_dt")
        return d.value

    def selection(self, U):
        sel = torch.empty(self.n_sel(), dtype=torch.uint8, device=self.device)
        self._stream()
        _check(_lib.enomr_debug_selection(self._ctx, self._state(U), _P(sel.data_ptr())),
               "enomr_debug_selection")
        return sel

    def rhs_vjp(self, U, Lbar, out=None, scale=1.0, accumulate=False):
        """scale * J(U)^T Lbar with the forward choices at U frozen."""
        if out is None:
            out = torch.zeros_like(U)
            accumulate = True
        self._stream()
        _check(_lib.enomr_rhs_vjp(self._ctx, self._state(U), self._state(Lbar, "Lbar"),
                                  self._state(out, "out"), float(scale), int(accumulate)),
               "enomr_rhs_vjp")
        return out

    def debug_alpha(self):
        """(alpha_x, alpha_y, alpha_bar_x, alpha_bar_y, argmax_x, argmax_y) of the
        last calls (see enomr_debug_alpha)."""
        ax = torch.empty(self.ny, 3, dtype=torch.float64, device=self.device)
        ay = torch.empty(self.nx, 3, dtype=torch.float64, device=self.device)
        bx, by = torch.empty_like(ax), torch.empty_like(ay)
        ix = torch.empty(self.ny, 3, dtype=torch.int64, device=self.device)
        iy = torch.empty(self.nx, 3, dtype=torch.int64, device=self.device)
        self._stream()
        _check(_lib.enomr_debug_alpha(self._ctx, _P(ax.data_ptr()), _P(ay.data_ptr()),
                                      _P(bx.data_ptr()), _P(by.data_ptr()), _P(ix.data_ptr()),
                                      _P(iy.data_ptr())), "enomr_debug_alpha")
        return ax, ay, bx, by, ix, iy

    def step_vjp(self, Un, dt, Ubar_np1, out=None):
        """(dU_{n+1}/dU_n)^T Ubar_np1 for one SSP-RK3 step of size dt from Un."""
        if out is None:
            out = torch.empty_like(Un)
        self._stream()
        _check(_lib.enomr_step_vjp(self._ctx, self._state(Un), float(dt),
                                   self._state(Ubar_np1, "Ubar_np1"), self._state(out, "out")),
               "enomr_step_vjp")
        return out

    def step_vjp_cfl(self, Un, cfl, Ubar_np1, out=None):
        """As step_vjp for a CFL step (enomr_step with dt <= 0): the step's dt
        is recomputed on the device from Un (no host round trip)."""
        if out is None:
            out = torch.empty_like(Un)
        self._stream()
        _check(_lib.enomr_step_vjp_cfl(self._ctx, self._state(Un), float(cfl),
                                       self._state(Ubar_np1, "Ubar_np1"), self._state(out, "out")),
               "enomr_step_vjp_cfl")
        return out

    def profile_begin(self, kernel: int, max_launches: int):
        """Time the next launches of one kernel (1 x sweep, 2 y sweep, 3 alpha)."""
        _check(_lib.enomr_profile_begin(self._ctx, kernel, max_launches), "enomr_profile_begin")

    def profile_end(self):
        n, ms = _I(), _D()
        _check(_lib.enomr_profile_end(self._ctx, ctypes.byref(n), ctypes.byref(ms)),
               "enomr_profile_end")
        return n.value, ms.value

    def set_side(self, side, kind_lo, state_lo=None, kind_hi=None, state_hi=None,
                 split0=float("inf"), rate=0.0):
        """Boundary side (0 x low, 1 x high, 2 y low, 3 y high): kind_lo below
        the along-side position split0 + rate t, kind_hi above; kinds
        'transmissive', 'reflective', 'inflow' (with a conserved state)."""
        k_lo = _SIDE_KINDS.get(kind_lo, kind_lo)
        k_hi = k_lo if kind_hi is None else _SIDE_KINDS.get(kind_hi, kind_hi)
        d = _Side(k_lo, k_hi, float(split0), float(rate))
        for q in range(4):
            d.state_lo[q] = 0.0 if state_lo is None else float(state_lo[q])
            d.state_hi[q] = 0.0 if state_hi is None else float(state_hi[q])
        _check(_lib.enomr_set_side(self._ctx, int(side), ctypes.byref(d)), "enomr_set_side")

    def set_sides(self, sides):
        """Four sides as (kind_lo, state_lo, kind_hi, state_hi, split0, rate)."""
        for i, sd in enumerate(sides):
            self.set_side(i, sd[0], sd[1], sd[2], sd[3], sd[4], sd[5])

    def set_staging(self, mode):
        """STAGING_AUTO (TMA where the state allows it), STAGING_LOADS or
        STAGING_TMA (TMA only; other states raise)."""
        _check(_lib.enomr_set_staging(self._ctx, int(mode)), "enomr_set_staging")

    def set_occupancy(self, mode):
        """OCCUPANCY_AUTO, OCCUPANCY_HIGH or OCCUPANCY_LOW (2D sweeps)."""
        _check(_lib.enomr_set_occupancy(self._ctx, int(mode)), "enomr_set_occupancy")

    def set_body_force(self, gx, gy):
        _check(_lib.enomr_set_body_force(self._ctx, float(gx), float(gy)),
               "enomr_set_body_force")

    @property
    def time(self):
        self._stream()
        t = _D()
        _check(_lib.enomr_get_time(self._ctx, ctypes.byref(t)), "enomr_get_time")
        return t.value

    @time.setter
    def time(self, t):
        self._stream()
        _check(_lib.enomr_set_time(self._ctx, float(t)), "enomr_set_time")

    def check_status(self):
        self._stream()
        _check(_lib.enomr_get_status(self._ctx), "enomr_get_status")

    def close(self):
        if getattr(self, "_ctx", None):
            _lib.enomr_free(self._ctx)
            self._ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """Many independent 1D Euler problems advanced together (one persistent
    launch per RK stage).  State: one float64 CUDA tensor of 3 * sum(n)
    values, problem p's [3, n[p]] block after problem p-1's."""

    def __init__(self, sizes, dx, order=9, bc=TRANSMISSIVE, gamma=1.4, device=None):
        import numpy as np
        self.sizes = np.ascontiguousarray(sizes, dtype=np.int64)
        self.dx = np.ascontiguousarray(dx, dtype=np.float64)
        if self.sizes.shape != self.dx.shape or self.sizes.ndim != 1:
            raise ValueError("sizes and dx must be 1D arrays of the same length")
        self.device = torch.device(device if device is not None else "cuda")
        self.offsets = np.concatenate([[0], np.cumsum(3 * self.sizes)])
        ctx = _P()
        with torch.cuda.device(self.device):
            s = torch.cuda.current_stream(self.device).cuda_stream
            _check(_lib.enomr_batch_init(ctypes.byref(ctx), len(self.sizes),
                                         self.sizes.ctypes.data_as(_P),
                                         self.dx.ctypes.data_as(_P), order, gamma, bc, _P(s)),
                   "enomr_batch_init")
        self._ctx = ctx
        self.total = int(_lib.enomr_batch_total_cells(ctx))

    def _state(self, U):
        if (not isinstance(U, torch.Tensor) or U.dtype != torch.float64 or U.device.type != "cuda"
                or U.numel() != 3 * self.total or not U.is_contiguous()):
            raise ValueError(f"packed state must be a contiguous float64 CUDA tensor of {3 * self.total}")
        _check(_lib.enomr_batch_set_stream(self._ctx,
                                           _P(torch.cuda.current_stream(self.device).cuda_stream)),
               "enomr_batch_set_stream")
        return _P(U.data_ptr())

    def pack(self, states):
        return torch.cat([torch.as_tensor(u, dtype=torch.float64).reshape(-1) for u in states]).to(
            self.device)

    def view(self, U, p):
        return U[int(self.offsets[p]):int(self.offsets[p + 1])].view(3, int(self.sizes[p]))

    def step(self, U, cfl=0.5):
        _check(_lib.enomr_batch_step(self._ctx, self._state(U), float(cfl)), "enomr_batch_step")

    def autotune(self, U, reps=3):
        t, g = _I(), _I()
        _check(_lib.enomr_batch_autotune(self._ctx, self._state(U), int(reps), ctypes.byref(t),
                                         ctypes.byref(g)), "enomr_batch_autotune")
        return t.value, g.value

    def config(self):
        """(tile, grid, tiles_per_item) in use."""
        t, g, k = _I(), _I(), _I()
        _check(_lib.enomr_batch_config(self._ctx, ctypes.byref(t), ctypes.byref(g),
                                       ctypes.byref(k)), "enomr_batch_config")
        return t.value, g.value, k.value

    def check_status(self):
        _check(_lib.enomr_batch_get_status(self._ctx), "enomr_batch_get_status")

    def close(self):
        if getattr(self, "_ctx", None):
            _lib.enomr_batch_free(self._ctx)
            self._ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class _Rollout(torch.autograd.Function):
    """n SSP-RK3 steps with per-step checkpoints (one preallocated
    [n, *state] tensor); backward runs the step transposes in reverse,
    recomputing the stages from each checkpoint.  With CFL steps (dt <= 0)
    every step's dt stays on the device: the forward pass does not read it
    back and the backward pass recomputes it from the checkpoint
    (enomr_step_vjp_cfl), so neither direction synchronises per step."""

    @staticmethod
    def forward(ctx, U0, solver, nsteps, cfl, dt):
        U = U0.detach().clone()
        ckpt = torch.empty((nsteps,) + tuple(U.shape), dtype=U.dtype, device=U.device)
        for i in range(nsteps):
            ckpt[i].copy_(U)
            solver.step(U, dt, cfl)
        ctx.solver, ctx.ckpt, ctx.cfl, ctx.dt = solver, ckpt, cfl, dt
        return U

    @staticmethod
    def backward(ctx, gout):
        g = gout.contiguous().clone()
        tmp = torch.empty_like(g)
        for i in reversed(range(ctx.ckpt.shape[0])):
            if ctx.dt > 0.0:
                ctx.solver.step_vjp(ctx.ckpt[i], ctx.dt, g, out=tmp)
            else:
                ctx.solver.step_vjp_cfl(ctx.ckpt[i], ctx.cfl, g, out=tmp)
            g, tmp = tmp, g
        return g, None, None, None, None


def rollout(U0, solver, nsteps, cfl=0.5, dt=0.0):
    """Differentiable: U(t_n) after nsteps SSP-RK3 steps from U0 (CFL steps
    when dt <= 0; the step sizes are held fixed in the gradient)."""
    return _Rollout.apply(U0, solver, nsteps, cfl, dt)
