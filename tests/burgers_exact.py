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
