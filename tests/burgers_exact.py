"""Exact solution of the Burgers accuracy test before the shock forms, and
the error norms of Table 8.

u(x, t) = u0(xi) where xi solves xi + t u0(xi) = x (characteristics);
u0 = lam (1 + 0.5 sin^3(pi x)).  Newton's method from xi = x converges for
t below the breaking time 1 / max(-u0') (about 0.55/lam)."""
from __future__ import annotations

import numpy as np

from paper_2311_15504_gb300 import workloads as wl


def exact(x, t, lam=1.0):
    xi = np.array(x, dtype=np.float64)
    for _ in range(60):
        s, c = np.sin(np.pi * xi), np.cos(np.pi * xi)
        u0 = lam * (1.0 + 0.5 * s ** 3)
        du0 = lam * 1.5 * np.pi * s * s * c
        step = (xi + t * u0 - x) / (1.0 + t * du0)
        xi = xi - step
        if np.abs(step).max() < 1e-16:
            break
    return lam * (1.0 + 0.5 * np.sin(np.pi * xi) ** 3)


def dt_schedule(order, h, t_final, lam=1.0):
    """Steps of the paper's dt up to t_final, the last one clipped."""
    dt = wl.burgers_dt(order, h, lam)
    n = int(np.floor(t_final / dt * (1.0 + 1e-14)))
    steps = [dt] * n
    rest = t_final - n * dt
    if rest > 1e-14 * t_final:
        steps.append(rest)
    return steps


def errors(u, h, t, lam=1.0):
    """(L1, Linf) against the exact solution; L1 over the N+1 nodes of
    Sec. 2.1 (the periodic endpoint counted twice)."""
    n = u.shape[0]
    x = h * np.arange(n)
    e = np.abs(u - exact(x, t, lam))
    return (e.sum() + e[0]) / (n + 1), e.max()



def _u0(xi):
    return 1.0 + 0.5 * np.sin(np.pi * xi) ** 3


def _U0(xi):
    """A primitive of u0 (sin^3 = sin - sin cos^2)."""
    c = np.cos(np.pi * xi)
    return xi - 0.5 / np.pi * (c - c ** 3 / 3.0)


def exact_entropy(x, t, m=20001):
    """Entropy solution for lam = 1 at any t, shocks included, by the
    Hopf-Lax formula for the convex flux u^2/2: u(x, t) = u0(xi*) with xi*
    the minimiser of U0(xi) + (x - xi)^2 / (2 t), U0 a primitive of u0.  The
    minimiser lies in [x - 1.5 t, x - 0.5 t] (the range of u0); it is taken
    on a grid of m points there, then refined by Newton's method on
    u0(xi) - (x - xi) / t = 0 (the first-order condition)."""
    x = np.atleast_1d(np.asarray(x, dtype=np.float64))
    out = np.empty_like(x)
    grid = np.linspace(-1.5 * t, -0.5 * t, m)
    for i, xx in enumerate(x):
        xi = xx + grid
        G = _U0(xi) + (xx - xi) ** 2 / (2.0 * t)
        z = xi[np.argmin(G)]
        for _ in range(30):
            s_, c_ = np.sin(np.pi * z), np.cos(np.pi * z)
            f = _u0(z) - (xx - z) / t
            df = 1.5 * np.pi * s_ * s_ * c_ + 1.0 / t
            if df <= 0.0:
                break
            step = f / df
            z -= step
            if abs(step) < 1e-15:
                break
        out[i] = _u0(z)
    return out
