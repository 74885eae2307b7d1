"""Exact solution of the Riemann problem of the 1D Euler equations for an
ideal gas, by the textbook construction: the star pressure p* is the root of
f_L(p) + f_R(p) + u_R - u_L = 0, where f_K is the Rankine-Hugoniot relation
(p > p_K, a shock) or the isentropic Riemann-invariant relation (p <= p_K, a
rarefaction) linking the state K to the star region; the solution is then
sampled along x/t.  Test infrastructure only: it gives the reference
solution of the shock tubes (Sec. 4.3) against which the oracle is pinned.
"""
import math

import numpy as np


def _f(p, rho, pk, c, g):
    """f_K(p) and its derivative."""
    if p > pk:  # shock
        A = 2.0 / ((g + 1.0) * rho)
        B = (g - 1.0) / (g + 1.0) * pk
        s = math.sqrt(A / (p + B))
        return (p - pk) * s, s * (1.0 - 0.5 * (p - pk) / (p + B))
    e = (g - 1.0) / (2.0 * g)  # rarefaction
    r = (p / pk) ** e
    return 2.0 * c / (g - 1.0) * (r - 1.0), (p / pk) ** (-(g + 1.0) / (2.0 * g)) / (rho * c)


def star_state(left, right, g=1.4):
    """(p*, u*) of the Riemann problem left = (rho, u, p), right = (rho, u, p)."""
    rl, ul, pl = left
    rr, ur, pr = right
    cl, cr = math.sqrt(g * pl / rl), math.sqrt(g * pr / rr)
    if 2.0 * (cl + cr) / (g - 1.0) <= ur - ul:
        raise ValueError("the data create a vacuum")
    p = max(1e-12, 0.5 * (pl + pr) - 0.125 * (ur - ul) * (rl + rr) * (cl + cr))
    for _ in range(100):
        fl, dl = _f(p, rl, pl, cl, g)
        fr, dr = _f(p, rr, pr, cr, g)
        step = (fl + fr + ur - ul) / (dl + dr)
        pn = max(p - step, 1e-14 * p)
        if abs(pn - p) <= 1e-15 * (pn + p):
            p = pn
            break
        p = pn
    fl, _ = _f(p, rl, pl, cl, g)
    fr, _ = _f(p, rr, pr, cr, g)
    return p, 0.5 * (ul + ur) + 0.5 * (fr - fl)


def sample(left, right, xi, g=1.4):
    """(rho, u, p) at the similarity coordinates xi = (x - x0) / t."""
    rl, ul, pl = left
    rr, ur, pr = right
    cl, cr = math.sqrt(g * pl / rl), math.sqrt(g * pr / rr)
    ps, us = star_state(left, right, g)
    gm, gp = (g - 1.0) / (g + 1.0), (g + 1.0) / (2.0 * g)
    out = np.empty((3, len(xi)))
    for i, s in enumerate(np.asarray(xi, dtype=np.float64)):
        if s <= us:  # left of the contact
            if ps > pl:  # left shock
                S = ul - cl * math.sqrt(gp * ps / pl + (g - 1.0) / (2.0 * g))
                if s <= S:
                    out[:, i] = (rl, ul, pl)
                else:
                    out[:, i] = (rl * (ps / pl + gm) / (gm * ps / pl + 1.0), us, ps)
            else:  # left rarefaction
                cs = cl * (ps / pl) ** ((g - 1.0) / (2.0 * g))
                if s <= ul - cl:
                    out[:, i] = (rl, ul, pl)
                elif s >= us - cs:
                    out[:, i] = (rl * (ps / pl) ** (1.0 / g), us, ps)
                else:
                    u = 2.0 / (g + 1.0) * (cl + 0.5 * (g - 1.0) * ul + s)
                    c = 2.0 / (g + 1.0) * (cl + 0.5 * (g - 1.0) * (ul - s))
                    out[:, i] = (rl * (c / cl) ** (2.0 / (g - 1.0)), u,
                                 pl * (c / cl) ** (2.0 * g / (g - 1.0)))
        else:  # right of the contact
            if ps > pr:  # right shock
                S = ur + cr * math.sqrt(gp * ps / pr + (g - 1.0) / (2.0 * g))
                if s >= S:
                    out[:, i] = (rr, ur, pr)
                else:
                    out[:, i] = (rr * (ps / pr + gm) / (gm * ps / pr + 1.0), us, ps)
            else:  # right rarefaction
                cs = cr * (ps / pr) ** ((g - 1.0) / (2.0 * g))
                if s >= ur + cr:
                    out[:, i] = (rr, ur, pr)
                elif s <= us + cs:
                    out[:, i] = (rr * (ps / pr) ** (1.0 / g), us, ps)
                else:
                    u = 2.0 / (g + 1.0) * (-cr + 0.5 * (g - 1.0) * ur + s)
                    c = 2.0 / (g + 1.0) * (cr - 0.5 * (g - 1.0) * (ur - s))
                    out[:, i] = (rr * (c / cr) ** (2.0 / (g - 1.0)), u,
                                 pr * (c / cr) ** (2.0 * g / (g - 1.0)))
    return out


def cell_average(left, right, x0, t, edges, g=1.4, sub=64):
    """Cell averages of (rho, m, E) over the cells between edges, by the
    midpoint rule on `sub` points per cell (the conserved variables, so that
    their totals are those of the exact solution up to quadrature)."""
    edges = np.asarray(edges, dtype=np.float64)
    h = np.diff(edges)
    pts = (edges[:-1, None] + h[:, None] * (np.arange(sub) + 0.5) / sub).ravel()
    rho, u, p = sample(left, right, (pts - x0) / t, g)
    U = np.stack([rho, rho * u, p / (g - 1.0) + 0.5 * rho * u * u])
    return U.reshape(3, len(h), sub).mean(axis=2)
