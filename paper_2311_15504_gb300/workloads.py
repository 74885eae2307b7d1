"""Seeded synthetic inputs shaped like the paper's test problems.

This module holds initial conditions and random test data only.  It contains
none of the ENO-MR arithmetic and is shared by the tests, the benchmark and
the oracle-side checks.

Grids (paper Sec. 2.1 defines nodes x_j = x_L + (j-1) h, h = (x_R-x_L)/N):
  periodic     -- N unknowns at x_L + j h, j = 0..N-1 (node N+1 is node 1);
  transmissive -- cell centres x_L + (j + 1/2) h.
"""
from __future__ import annotations

import numpy as np

GAMMA = 1.4


def periodic_grid(xl: float, xr: float, n: int):
    h = (xr - xl) / n
    return xl + h * np.arange(n), h


def centred_grid(xl: float, xr: float, n: int):
    h = (xr - xl) / n
    return xl + h * (np.arange(n) + 0.5), h


def conserved_1d(rho, u, p, gamma=GAMMA):
    """(rho, u, p) -> U = [rho, rho u, rho e], e = p/(rho(gamma-1)) + u^2/2."""
    rho = np.asarray(rho, dtype=np.float64)
    u = np.broadcast_to(np.asarray(u, dtype=np.float64), rho.shape)
    p = np.broadcast_to(np.asarray(p, dtype=np.float64), rho.shape)
    return np.stack([rho, rho * u, p / (gamma - 1.0) + 0.5 * rho * u * u])


def conserved_2d(rho, u, v, p, gamma=GAMMA):
    rho = np.asarray(rho, dtype=np.float64)
    u = np.broadcast_to(np.asarray(u, dtype=np.float64), rho.shape)
    v = np.broadcast_to(np.asarray(v, dtype=np.float64), rho.shape)
    p = np.broadcast_to(np.asarray(p, dtype=np.float64), rho.shape)
    return np.stack([rho, rho * u, rho * v,
                     p / (gamma - 1.0) + 0.5 * rho * (u * u + v * v)])


# ---------------------------------------------------------------------------
# Scalar advection (Sec. 4.1)
# ---------------------------------------------------------------------------
def advection_sine(n: int, power: int = 1, lam: float = 1.0):
    """u0 = lam * sin^power(pi x) on [-1, 1], periodic."""
    x, h = periodic_grid(-1.0, 1.0, n)
    return lam * np.sin(np.pi * x) ** power, h


def advection_step(n: int):
    """u0 = 1 on [-0.5, 0.5], else 0, on [-1, 1], periodic."""
    x, h = periodic_grid(-1.0, 1.0, n)
    return np.where(np.abs(x) <= 0.5, 1.0, 0.0), h


# ---------------------------------------------------------------------------
# Inviscid Burgers (Sec. 4.2)
# ---------------------------------------------------------------------------
def burgers_sine3(n: int, lam: float = 1.0):
    """u0 = lam (1 + 0.5 sin^3(pi x)) on [0, 2], periodic; n unknowns."""
    x, h = periodic_grid(0.0, 2.0, n)
    return lam * (1.0 + 0.5 * np.sin(np.pi * x) ** 3), h


def burgers_dt(order: int, h: float, lam: float = 1.0):
    """Time step of the Burgers accuracy test (Sec. 4.2): proportional to
    h^(R/3)/lam so that the SSP-RK3 error matches the order in space."""
    c = {5: 1.0, 9: 1e2, 13: 1e4, 17: 1e6}[order]
    return c * h ** (order / 3.0) / lam


# ---------------------------------------------------------------------------
# 1D Euler
# ---------------------------------------------------------------------------
def shock_entropy(n: int, gamma=GAMMA):
    """Shock / entropy-wave interaction on [-5, 5]: x < -4 gets
    (3.857143, 2.629369, 10.33333), else rho = 1 + 0.2 sin(5x), u = 0, p = 1."""
    x, h = centred_grid(-5.0, 5.0, n)
    left = x < -4.0
    rho = np.where(left, 3.857143, 1.0 + 0.2 * np.sin(5.0 * x))
    u = np.where(left, 2.629369, 0.0)
    p = np.where(left, 10.33333, 1.0)
    return conserved_1d(rho, u, p, gamma), h


def lax_tube(n: int, gamma=GAMMA):
    """Lax shock tube on [0, 2] (Sec. 4.3)."""
    x, h = centred_grid(0.0, 2.0, n)
    left = x < 1.0
    rho = np.where(left, 0.445, 0.5)
    u = np.where(left, 0.698, 0.0)
    p = np.where(left, 3.528, 0.571)
    return conserved_1d(rho, u, p, gamma), h


def density_wave_1d(n: int, gamma=GAMMA):
    """rho = 1 + 0.2 sin(pi x), u = 1, p = 1 on [-1, 1], periodic.
    Exact solution rho(x - t)."""
    x, h = periodic_grid(-1.0, 1.0, n)
    return conserved_1d(1.0 + 0.2 * np.sin(np.pi * x), 1.0, 1.0, gamma), h


def riemann_batch(nprob: int, seed: int = 0, nmin: int = 128, nmax: int = 8192,
                  gamma=GAMMA):
    """Independent 1D Riemann problems on [0, 1], diaphragm at 0.5.
    Sizes log-uniform in [nmin, nmax]; rho ~ U[0.1,2], u ~ U[-1,1],
    p ~ U[0.1,10] on each side.  Returns (sizes, list of U arrays, h list)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    sizes = np.rint(np.exp(rng.uniform(np.log(nmin), np.log(nmax), nprob))).astype(np.int64)
    states = rng.uniform([0.1, -1.0, 0.1, 0.1, -1.0, 0.1], [2.0, 1.0, 10.0, 2.0, 1.0, 10.0],
                         size=(nprob, 6))
    Us, hs = [], []
    for k in range(nprob):
        x, h = centred_grid(0.0, 1.0, int(sizes[k]))
        left = x < 0.5
        rl, ul, pl, rr, ur, pr = states[k]
        Us.append(conserved_1d(np.where(left, rl, rr), np.where(left, ul, ur),
                               np.where(left, pl, pr), gamma))
        hs.append(h)
    return sizes, Us, np.array(hs)


# ---------------------------------------------------------------------------
# 2D Euler
# ---------------------------------------------------------------------------
def quadrant_states(seed: int):
    rng = np.random.Generator(np.random.PCG64(seed))
    lo = np.array([0.1, -1.0, -1.0, 0.02])
    hi = np.array([2.0, 1.0, 1.0, 2.0])
    return rng.uniform(lo, hi, size=(4, 4))


def riemann2d(nx: int, ny: int | None = None, seed: int = 0, xc=0.8, yc=0.8, gamma=GAMMA):
    """Four-quadrant Riemann problem on [0,1]^2 with the interface at
    (xc, yc); per-quadrant (rho, u, v, p) drawn from rho in [0.1,2],
    u, v in [-1,1], p in [0.02,2].  Quadrants: 0 = x>xc,y>yc; 1 = x<xc,y>yc;
    2 = x<xc,y<yc; 3 = x>xc,y<yc.  Returns U [4][ny][nx], dx, dy."""
    ny = nx if ny is None else ny
    x, dx = centred_grid(0.0, 1.0, nx)
    y, dy = centred_grid(0.0, 1.0, ny)
    st = quadrant_states(seed)
    X, Y = np.meshgrid(x, y)
    q = np.where(Y > yc, np.where(X > xc, 0, 1), np.where(X < xc, 2, 3))
    prim = st[q]  # [ny, nx, 4]
    return conserved_2d(prim[..., 0], prim[..., 1], prim[..., 2], prim[..., 3], gamma), dx, dy


def _quadrants(n: int, states, gamma=GAMMA):
    """Four constant states on [-1,1]^2 split at x = 0 and y = 0 (cell
    centres; keys 'll', 'lu', 'uu', 'ul' = (x side, y side))."""
    x, dx = centred_grid(-1.0, 1.0, n)
    X, Y = np.meshgrid(x, x)
    out = np.zeros((4, n, n))
    for key, (r, u, v, p) in states.items():
        m = ((X < 0) if key[0] == "l" else (X >= 0)) & ((Y < 0) if key[1] == "l" else (Y >= 0))
        out[:, m] = conserved_2d(np.array([r]), u, v, p, gamma)[:, 0][:, None]
    return out, dx, dx


def riemann2d_rp1(n: int, gamma=GAMMA):
    """The paper's first 2D Riemann configuration on [-1,1]^2 (Sec. 4.4):
    four shocks; symmetric about the diagonal x = y (with u <-> v)."""
    return _quadrants(n, {"ll": (0.138, 1.206, 1.206, 0.029), "lu": (0.5323, 1.206, 0.0, 0.3),
                          "uu": (1.5, 0.0, 0.0, 1.5), "ul": (0.5323, 0.0, 1.206, 0.3)}, gamma)


def riemann2d_rp2(n: int, gamma=GAMMA):
    """The paper's second 2D Riemann configuration (Sec. 4.4): four contact
    discontinuities."""
    return _quadrants(n, {"ll": (1.0, -0.75, 0.5, 1.0), "lu": (2.0, 0.75, 0.5, 1.0),
                          "uu": (1.0, 0.75, -0.5, 1.0), "ul": (3.0, -0.75, -0.5, 1.0)}, gamma)


def double_mach(nx: int = 1200, ny: int = 300, gamma=GAMMA):
    """Double Mach reflection (Sec. 4.4) on [0, 4] x [0, 1], cell centres: a
    Mach 10 shock at 60 degrees through (1/6, 0).  Returns U, dx, dy and the
    boundary sides (x low, x high, y low, y high) as tuples
    (kind_lo, state_lo, kind_hi, state_hi, split0, rate) with kinds
    'transmissive', 'reflective', 'inflow' and conserved states:
    post-shock inflow on the left; transmissive on the right; at the
    bottom transmissive for x < 1/6 and reflective beyond; at the top the
    exact shock position 1/6 + (1 + 20 t)/sqrt(3) separates post- from
    pre-shock inflow."""
    x, dx = centred_grid(0.0, 4.0, nx)
    y, dy = centred_grid(0.0, 1.0, ny)
    X, Y = np.meshgrid(x, y)
    s60, c60 = np.sin(np.pi / 3), np.cos(np.pi / 3)
    post = conserved_2d(np.array([8.0]), 8.25 * s60, -8.25 * c60, 116.5, gamma)[:, 0]
    pre = conserved_2d(np.array([1.4]), 0.0, 0.0, 1.0, gamma)[:, 0]
    behind = X < 1.0 / 6.0 + Y / np.sqrt(3.0)
    U = np.where(behind[None], post[:, None, None], pre[:, None, None])
    sides = (("inflow", post, "inflow", post, np.inf, 0.0),
             ("transmissive", None, "transmissive", None, np.inf, 0.0),
             ("transmissive", None, "reflective", None, 1.0 / 6.0, 0.0),
             ("inflow", post, "inflow", pre, 1.0 / 6.0 + 1.0 / np.sqrt(3.0), 20.0 / np.sqrt(3.0)))
    return np.ascontiguousarray(U), dx, dy, sides


def rayleigh_taylor(nx: int = 128, ny: int = 512, gamma=5.0 / 3.0):
    """Rayleigh-Taylor instability (Sec. 4.4) on [0, 0.25] x [0, 1], gamma
    5/3, body force (0, 1): heavy fluid (rho = 2) below y = 0.5, light
    (rho = 1) above, p = 2y + 1 below and y + 1.5 above, v = -0.025 c
    cos(8 pi x).  Sides: reflective left and right; inflow of the rest
    states (2, 0, 0, 1) at the bottom and (1, 0, 0, 2.5) at the top."""
    x, dx = centred_grid(0.0, 0.25, nx)
    y, dy = centred_grid(0.0, 1.0, ny)
    X, Y = np.meshgrid(x, y)
    low = Y < 0.5
    rho = np.where(low, 2.0, 1.0)
    p = np.where(low, 2.0 * Y + 1.0, Y + 1.5)
    v = -0.025 * np.sqrt(gamma * p / rho) * np.cos(8.0 * np.pi * X)
    U = conserved_2d(rho, 0.0, v, p, gamma)
    bottom = conserved_2d(np.array([2.0]), 0.0, 0.0, 1.0, gamma)[:, 0]
    top = conserved_2d(np.array([1.0]), 0.0, 0.0, 2.5, gamma)[:, 0]
    sides = (("reflective", None, "reflective", None, np.inf, 0.0),
             ("reflective", None, "reflective", None, np.inf, 0.0),
             ("inflow", bottom, "inflow", bottom, np.inf, 0.0),
             ("inflow", top, "inflow", top, np.inf, 0.0))
    return np.ascontiguousarray(U), dx, dy, sides


def isentropic_vortex(n: int, strength=5.0, gamma=GAMMA, L=10.0, centre=None):
    """Isentropic vortex on [0,L]^2, periodic, centre (L/2, L/2) unless
    given, free stream (rho, u, v, p) = (1, 1, 1, 1)."""
    x, h = periodic_grid(0.0, L, n)
    X, Y = np.meshgrid(x + 0.5 * h, x + 0.5 * h)
    xc, yc = (0.5 * L, 0.5 * L) if centre is None else centre
    r2 = (X - xc) ** 2 + (Y - yc) ** 2
    du = -strength / (2 * np.pi) * np.exp(0.5 * (1 - r2)) * (Y - yc)
    dv = strength / (2 * np.pi) * np.exp(0.5 * (1 - r2)) * (X - xc)
    T = 1.0 - (gamma - 1.0) * strength ** 2 / (8 * gamma * np.pi ** 2) * np.exp(1 - r2)
    rho = T ** (1.0 / (gamma - 1.0))
    p = rho ** gamma
    return conserved_2d(rho, 1.0 + du, 1.0 + dv, p, gamma), h, h


def density_wave_2d(n: int, gamma=GAMMA):
    """rho = 1 + 0.2 sin(pi(x+y)), u = v = 1, p = 1 on [-1,1]^2 periodic."""
    x, h = periodic_grid(-1.0, 1.0, n)
    X, Y = np.meshgrid(x, x)
    return conserved_2d(1.0 + 0.2 * np.sin(np.pi * (X + Y)), 1.0, 1.0, 1.0, gamma), h, h


def smooth_random_euler2d(nx: int, ny: int, seed: int = 0, amp=0.1, gamma=GAMMA):
    """A smooth periodic random field around a uniform state (for parity)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    x = np.arange(nx) / nx
    y = np.arange(ny) / ny
    X, Y = np.meshgrid(x, y)
    fields = []
    for base in (1.0, 0.3, -0.2, 1.0):
        f = np.full((ny, nx), base)
        for _ in range(3):
            kx, ky = rng.integers(1, 4, size=2)
            ph = rng.uniform(0, 2 * np.pi)
            f = f + amp * rng.uniform(0.2, 1.0) * np.sin(2 * np.pi * (kx * X + ky * Y) + ph)
        fields.append(f)
    return conserved_2d(fields[0], fields[1], fields[2], fields[3], gamma)


def random_window(rng, n, kind="float"):
    """Random test windows: 'float' N(0,1), 'int' small integers, 'step'."""
    if kind == "float":
        return rng.standard_normal(n)
    if kind == "int":
        return rng.integers(-4, 5, size=n).astype(np.float64)
    if kind == "step":
        k = rng.integers(1, n)
        return np.where(np.arange(n) < k, 0.0, 1.0) * rng.choice([-1.0, 1.0]) * 10 ** rng.uniform(-3, 3)
    raise ValueError(kind)
