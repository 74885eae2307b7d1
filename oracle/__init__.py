"""Plain FP64 CPU oracle for the ENO-MR right-hand side (test infrastructure).

Only the test suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` import this package.  The product library never does.  The C
source (``enomr_oracle.c``) restates the paper's algorithm step by step: the
conservative finite-difference form (Sec. 2.1, Eq. 1DWENOFD), global
Lax-Friedrichs splitting (Eq. LF_Flux_Split), the ENO-MR selection (Sec. 3.2,
Steps 1-3) over the candidates of Eq. (Candidates) with the coefficients of
Tables 1-4, Roe-averaged characteristic decomposition (Sec. 4), SSP-RK3
(Eq. TVD3rdRK) and the linear SSP-RK family (Eq. lSSPRK).

Every function here is pinned by the ``-m "not gpu"`` tests against exact
rational derivations, brute force, closed forms and values printed in the
paper.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "enomr_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

EQ_ADVECTION, EQ_EULER1D, EQ_EULER2D, EQ_BURGERS = 0, 1, 2, 3
SIDE_TRANSMISSIVE, SIDE_REFLECTIVE, SIDE_INFLOW = 1, 2, 3
BC_PERIODIC, BC_TRANSMISSIVE = 0, 1
ORC_OK, ORC_EINVAL, ORC_ENONPHYS = 0, 1, 4


class OracleError(RuntimeError):
    pass


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (FP contraction off, OpenMP if present)."""
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    base = ["gcc", "-O2", "-std=c99", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
            "-shared", "-o", _LIB + ".tmp", _SRC, "-lm"]
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True,
                       capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True)
    os.replace(_LIB + ".tmp", _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB)
            P = ctypes.c_void_p
            L = ctypes.c_long
            I = ctypes.c_int
            D = ctypes.c_double
            sig = {
                "orc_num_tested": (I, [I]),
                "orc_candidate": (I, [I, I, P, P, P, P]),
                "orc_paper_stencil": (I, [I, P, P, P, P]),
                "orc_mr": (D, [I, P, I, P]),
                "orc_mr_indicators": (I, [I, P, P, P, P, P]),
                "orc_rhs_advection": (I, [L, P, D, I, I, D, P, P, P, P, P]),
                "orc_rhs_burgers": (I, [L, P, D, I, I, P, P, P, P, P]),
                "orc_rhs_euler2d_ext": (I, [L, L, P, D, D, I, D, P, D, D, D, P, P, P, P]),
                "orc_step_ssprk3_euler2d_ext": (I, [L, L, D, D, I, D, P, D, D, D, P, D]),
                "orc_rhs_euler1d": (I, [L, P, D, I, I, D, P, P, P, P, P, P]),
                "orc_rhs_euler2d": (I, [L, L, P, D, D, I, I, D, P, P, P, P, P, P, P]),
                "orc_euler_eigen": (I, [I, D, P, P, P, P, P]),
                "orc_rhs_euler1d_frozen": (I, [L, P, D, I, I, D, P, P, P, P]),
                "orc_rhs_euler2d_frozen": (I, [L, L, P, D, D, I, I, D, P, P, P, P, P, P]),
                "orc_rhs_euler2d_alpha": (I, [L, L, P, D, D, I, I, D, P, P, P, P]),
                "orc_rhs": (I, [I, L, L, D, D, I, I, D, D, P, P]),
                "orc_cfl_dt": (I, [I, L, L, D, D, D, D, P, D, P]),
                "orc_step_ssprk3": (I, [I, L, L, D, D, I, I, D, D, P, D]),
                "orc_lssp_coeffs": (I, [I, P]),
                "orc_step_lssp": (I, [I, I, L, L, D, D, I, I, D, D, P, D]),
                "orc_num_threads": (I, []),
                "orc_set_threads": (None, [I]),
            }
            for name, (res, args) in sig.items():
                fn = getattr(lib, name)
                fn.restype = res
                fn.argtypes = args
            _lib = lib
    return _lib


def _p(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _check(st):
    if st == ORC_ENONPHYS:
        raise OracleError("non-physical state (rho<=0, p<=0, c^2<=0 or non-finite)")
    if st != ORC_OK:
        raise OracleError(f"oracle error {st}")


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def num_threads() -> int:
    return _load().orc_num_threads()


def set_threads(n: int) -> None:
    _load().orc_set_threads(int(n))


# --------------------------------------------------------------------------
# Tables and single-window reconstruction
# --------------------------------------------------------------------------
def num_tested(R: int) -> int:
    n = _load().orc_num_tested(R)
    if n < 0:
        raise OracleError(f"unsupported order {R}")
    return n


def candidate(R: int, t: int):
    """(m, n, a_l, b_l) of the t-th tested candidate for order R."""
    m, n = ctypes.c_int(), ctypes.c_int()
    a = np.zeros(17)
    b = np.zeros(17)
    _check(_load().orc_candidate(R, t, ctypes.byref(m), ctypes.byref(n), _p(a), _p(b)))
    k = m.value + n.value + 1
    return m.value, n.value, a[:k].copy(), b[:k].copy()


def paper_stencil(s: int):
    """Entry s of Eq. (Candidates) as typed in the oracle: (m, n, den, nums)."""
    m, n, den = ctypes.c_int(), ctypes.c_int(), ctypes.c_long()
    num = np.zeros(17, dtype=np.int64)
    _check(_load().orc_paper_stencil(s, ctypes.byref(m), ctypes.byref(n),
                                     ctypes.byref(den), _p(num)))
    k = m.value + n.value + 1
    return m.value, n.value, den.value, [int(x) for x in num[:k]]


def mr(R: int, window, forced: int = -1):
    """ENO-MR value and selection id for one window of 2g-1 values."""
    w = _f64(window)
    g = (R + 1) // 2
    assert w.shape == (2 * g - 1,)
    sel = ctypes.c_int()
    v = _load().orc_mr(R, _p(w), forced, ctypes.byref(sel))
    return v, sel.value


def mr_indicators(R: int, window):
    w = _f64(window)
    T = num_tested(R)
    is0, mag0 = ctypes.c_double(), ctypes.c_double()
    is_ = np.zeros(T)
    mag = np.zeros(T)
    _check(_load().orc_mr_indicators(R, _p(w), ctypes.byref(is0), ctypes.byref(mag0),
                                     _p(is_), _p(mag)))
    return is0.value, mag0.value, is_, mag


# --------------------------------------------------------------------------
# Right-hand sides
# --------------------------------------------------------------------------
def rhs_advection(u, h, R, bc=BC_PERIODIC, a=1.0, forced=None, want_sel=False,
                  want_win=False, want_count=False):
    u = _f64(u)
    N = u.shape[0]
    g = (R + 1) // 2
    rhs = np.zeros(N)
    sel = np.zeros(2 * (N + 1), dtype=np.uint8) if want_sel else None
    win = np.zeros(2 * (N + 1) * (2 * g - 1)) if want_win else None
    fz = None if forced is None else np.ascontiguousarray(forced, dtype=np.uint8)
    cnt = ctypes.c_long(0)
    _check(_load().orc_rhs_advection(N, _p(u), h, R, bc, a, _p(fz), _p(sel), _p(win),
                                     _p(rhs), ctypes.byref(cnt)))
    out = {"rhs": rhs}
    if want_sel:
        out["sel"] = sel.reshape(2, N + 1)
    if want_win:
        out["win"] = win.reshape(2, N + 1, 2 * g - 1)
    if want_count:
        out["ntested"] = cnt.value
    return out


def rhs_burgers(u, h, R, bc=BC_PERIODIC, forced=None, want_sel=False, want_win=False,
                want_count=False):
    """Inviscid Burgers (Sec. 4.2): f = u^2/2, unsplit where u keeps one sign
    over the line, else the global Lax-Friedrichs split with alpha = max|u|.
    Layouts as rhs_advection."""
    u = _f64(u)
    N = u.shape[0]
    g = (R + 1) // 2
    rhs = np.zeros(N)
    sel = np.zeros(2 * (N + 1), dtype=np.uint8) if want_sel else None
    win = np.zeros(2 * (N + 1) * (2 * g - 1)) if want_win else None
    fz = None if forced is None else np.ascontiguousarray(forced, dtype=np.uint8)
    cnt = ctypes.c_long(0)
    _check(_load().orc_rhs_burgers(N, _p(u), h, R, bc, _p(fz), _p(sel), _p(win), _p(rhs),
                                   ctypes.byref(cnt)))
    out = {"rhs": rhs}
    if want_sel:
        out["sel"] = sel.reshape(2, N + 1)
    if want_win:
        out["win"] = win.reshape(2, N + 1, 2 * g - 1)
    if want_count:
        out["ntested"] = cnt.value
    return out


def side(kind_lo, state_lo=None, kind_hi=None, state_hi=None, split0=np.inf, rate=0.0):
    """A boundary side: kind_lo below the along-side position split0 + rate t,
    kind_hi above it (SIDE_TRANSMISSIVE, SIDE_REFLECTIVE, SIDE_INFLOW with a
    conserved state (rho, rho u, rho v, E))."""
    kind_hi = kind_lo if kind_hi is None else kind_hi
    z = np.zeros(4)
    return np.concatenate([[kind_lo, kind_hi, split0, rate],
                           z if state_lo is None else np.asarray(state_lo, dtype=np.float64),
                           z if state_hi is None else np.asarray(state_hi, dtype=np.float64)])


def _sides(sides):
    """[x low, x high, y low, y high] -> 48 doubles (None: transmissive)."""
    t = side(SIDE_TRANSMISSIVE)
    return np.ascontiguousarray(np.concatenate([t if s_ is None else s_ for s_ in sides]))


def rhs_euler2d_ext(U, dx, dy, R, sides=(None, None, None, None), t=0.0, gravity=(0.0, 0.0),
                    gamma=1.4, forced=None, want_sel=False, want_win=False):
    """2D Euler on [0, nx dx] x [0, ny dy] with boundary sides at time t and a
    body force (gx, gy): S = (0, rho gx, rho gy, rho u gx + rho v gy).
    sel / win layouts as rhs_euler2d (win: one row of 2g-1 values per
    selection entry)."""
    U = _f64(U)
    _, ny, nx = U.shape
    g = (R + 1) // 2
    rhs = np.zeros_like(U)
    nsel = 8 * ny * (nx + 1) + 8 * nx * (ny + 1)
    sel = np.zeros(nsel, dtype=np.uint8) if want_sel else None
    win = np.zeros(nsel * (2 * g - 1)) if want_win else None
    fz = None if forced is None else np.ascontiguousarray(forced, dtype=np.uint8)
    sd = _sides(sides)
    _check(_load().orc_rhs_euler2d_ext(nx, ny, _p(U), dx, dy, R, gamma, _p(sd), t, gravity[0],
                                       gravity[1], _p(fz), _p(sel), _p(win), _p(rhs)))
    out = {"rhs": rhs}
    if want_sel:
        out["sel"] = sel
    if want_win:
        out["win"] = win.reshape(nsel, 2 * g - 1)
    return out


def step_euler2d_ext(U, dx, dy, R, dt, sides=(None, None, None, None), t=0.0,
                     gravity=(0.0, 0.0), gamma=1.4):
    """One SSP-RK3 step from time t (stage right-hand sides at t, t + dt,
    t + dt/2)."""
    U = _f64(U).copy()
    _, ny, nx = U.shape
    sd = _sides(sides)
    _check(_load().orc_step_ssprk3_euler2d_ext(nx, ny, dx, dy, R, gamma, _p(sd), t, gravity[0],
                                               gravity[1], _p(U), dt))
    return U


def rhs_euler1d(U, h, R, bc=BC_TRANSMISSIVE, gamma=1.4, forced=None, want_sel=False,
                want_win=False, want_count=False):
    U = _f64(U)
    assert U.shape[0] == 3
    N = U.shape[1]
    g = (R + 1) // 2
    rhs = np.zeros_like(U)
    alpha = np.zeros(3)
    sel = np.zeros(2 * 3 * (N + 1), dtype=np.uint8) if want_sel else None
    win = np.zeros(2 * 3 * (N + 1) * (2 * g - 1)) if want_win else None
    fz = None if forced is None else np.ascontiguousarray(forced, dtype=np.uint8)
    cnt = ctypes.c_long(0)
    _check(_load().orc_rhs_euler1d(N, _p(U), h, R, bc, gamma, _p(fz), _p(sel), _p(win),
                                   _p(rhs), _p(alpha), ctypes.byref(cnt)))
    out = {"rhs": rhs, "alpha": alpha}
    if want_sel:
        out["sel"] = sel.reshape(2, 3, N + 1)
    if want_win:
        out["win"] = win.reshape(2, 3, N + 1, 2 * g - 1)
    if want_count:
        out["ntested"] = cnt.value
    return out


def rhs_euler2d(U, dx, dy, R, bc=BC_TRANSMISSIVE, gamma=1.4, forced=None, want_sel=False,
                want_win=False, want_count=False):
    U = _f64(U)
    assert U.shape[0] == 4
    ny, nx = U.shape[1], U.shape[2]
    g = (R + 1) // 2
    W = 2 * g - 1
    rhs = np.zeros_like(U)
    ax = np.zeros((ny, 4))
    ay = np.zeros((nx, 4))
    nsx = 8 * ny * (nx + 1)
    nsy = 8 * nx * (ny + 1)
    sel = np.zeros(nsx + nsy, dtype=np.uint8) if want_sel else None
    win = np.zeros((nsx + nsy) * W) if want_win else None
    fz = None if forced is None else np.ascontiguousarray(forced, dtype=np.uint8)
    cnt = ctypes.c_long(0)
    _check(_load().orc_rhs_euler2d(nx, ny, _p(U), dx, dy, R, bc, gamma, _p(fz), _p(sel),
                                   _p(win), _p(rhs), _p(ax), _p(ay), ctypes.byref(cnt)))
    out = {"rhs": rhs, "alpha_x": ax, "alpha_y": ay}
    if want_sel:
        out["sel_x"] = sel[:nsx].reshape(2, 4, ny, nx + 1)
        out["sel_y"] = sel[nsx:].reshape(2, 4, nx, ny + 1)
        out["sel"] = sel
    if want_win:
        out["win_x"] = win[:nsx * W].reshape(2, 4, ny, nx + 1, W)
        out["win_y"] = win[nsx * W:].reshape(2, 4, nx, ny + 1, W)
    if want_count:
        out["ntested"] = cnt.value
    return out


def rhs_euler1d_frozen(U, h, R, forced, amax=None, bc=BC_TRANSMISSIVE, gamma=1.4):
    """1D Euler RHS with the stencils forced and the alpha maximisers given
    (amax, 3 ints); with amax None returns (rhs, the plain scheme's amax)."""
    U = _f64(U)
    N = U.shape[1]
    rhs = np.zeros_like(U)
    fz = np.ascontiguousarray(forced, dtype=np.uint8)
    ain = None if amax is None else np.ascontiguousarray(amax, dtype=np.int32)
    aout = np.zeros(3, dtype=np.int32)
    _check(_load().orc_rhs_euler1d_frozen(N, _p(U), h, R, bc, gamma, _p(fz), _p(ain), _p(aout),
                                          _p(rhs)))
    return rhs if amax is not None else (rhs, aout)


def rhs_euler2d_frozen(U, dx, dy, R, forced, amax=None, bc=BC_TRANSMISSIVE, gamma=1.4):
    """2D Euler RHS with the stencils forced and the per-line alpha
    maximisers given (amax = (amx [ny,4], amy [nx,4]))."""
    U = _f64(U)
    ny, nx = U.shape[1], U.shape[2]
    rhs = np.zeros_like(U)
    fz = np.ascontiguousarray(forced, dtype=np.uint8)
    if amax is None:
        ax, ay = np.zeros((ny, 4), dtype=np.int32), np.zeros((nx, 4), dtype=np.int32)
        _check(_load().orc_rhs_euler2d_frozen(nx, ny, _p(U), dx, dy, R, bc, gamma, _p(fz), None,
                                              None, _p(ax), _p(ay), _p(rhs)))
        return rhs, (ax, ay)
    ax = np.ascontiguousarray(amax[0], dtype=np.int32)
    ay = np.ascontiguousarray(amax[1], dtype=np.int32)
    _check(_load().orc_rhs_euler2d_frozen(nx, ny, _p(U), dx, dy, R, bc, gamma, _p(fz), _p(ax),
                                          _p(ay), None, None, _p(rhs)))
    return rhs


def rhs_euler2d_alpha(U, dx, dy, R, forced, alpha_x, alpha_y, bc=BC_TRANSMISSIVE, gamma=1.4):
    """2D Euler RHS with forced stencils and given split speeds
    (alpha_x [ny,4], alpha_y [nx,4])."""
    U = _f64(U)
    ny, nx = U.shape[1], U.shape[2]
    rhs = np.zeros_like(U)
    fz = np.ascontiguousarray(forced, dtype=np.uint8)
    _check(_load().orc_rhs_euler2d_alpha(nx, ny, _p(U), dx, dy, R, bc, gamma, _p(fz),
                                         _p(_f64(alpha_x)), _p(_f64(alpha_y)), _p(rhs)))
    return rhs


def euler_eigen(UL, UR, gamma=1.4):
    UL = _f64(UL)
    UR = _f64(UR)
    c = UL.shape[0]
    Rm = np.zeros(c * c)
    Lm = np.zeros(c * c)
    lam = np.zeros(4)
    _check(_load().orc_euler_eigen(c, gamma, _p(UL), _p(UR), _p(Rm), _p(Lm), _p(lam)))
    return Rm.reshape(c, c), Lm.reshape(c, c), lam[:c].copy()


# --------------------------------------------------------------------------
# Time integration
# --------------------------------------------------------------------------
class Problem:
    """eq in {EQ_ADVECTION, EQ_EULER1D, EQ_EULER2D, EQ_BURGERS}; U layouts: (N,),
    (3,N), (4,ny,nx), (N,)."""

    def __init__(self, eq, R, nx, ny=1, dx=1.0, dy=1.0, bc=BC_PERIODIC, gamma=1.4, a=1.0):
        self.eq, self.R, self.nx, self.ny = eq, R, nx, ny
        self.dx, self.dy, self.bc, self.gamma, self.a = dx, dy, bc, gamma, a

    def _args(self):
        return (self.eq, self.nx, self.ny, self.dx, self.dy, self.R, self.bc, self.gamma,
                self.a)

    def rhs(self, U):
        U = _f64(U)
        out = np.zeros_like(U)
        _check(_load().orc_rhs(*self._args(), _p(U), _p(out)))
        return out

    def cfl_dt(self, U, cfl):
        U = _f64(U)
        dt = ctypes.c_double()
        _check(_load().orc_cfl_dt(self.eq, self.nx, self.ny, self.dx, self.dy, self.gamma,
                                  self.a, _p(U), cfl, ctypes.byref(dt)))
        return dt.value

    def step_ssprk3(self, U, dt):
        U = _f64(U).copy()
        _check(_load().orc_step_ssprk3(*self._args(), _p(U), dt))
        return U

    def step_lssp(self, U, dt, m):
        U = _f64(U).copy()
        _check(_load().orc_step_lssp(m, *self._args(), _p(U), dt))
        return U

    def run_ssprk3(self, U, t_final, cfl, max_steps=10 ** 7):
        """March to t_final with the CFL step; the last step is clipped."""
        t = 0.0
        n = 0
        U = _f64(U).copy()
        while t < t_final and n < max_steps:
            dt = self.cfl_dt(U, cfl)
            if t + dt > t_final:
                dt = t_final - t
            U = self.step_ssprk3(U, dt)
            t += dt
            n += 1
        return U, n


def lssp_coeffs(m: int):
    out = np.zeros(m)
    _check(_load().orc_lssp_coeffs(m, _p(out)))
    return out
