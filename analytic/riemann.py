"""Exact solution of the 1-D Riemann problem of an ideal gas (a reference solution).

Used as the analytic reference of the Sod shock tube (Sect. "Sod test": left
state (n_l, p_l), right state (0.125 n_l, 0.1 p_l), both at rest).  The
method follows the textbook construction (Toro, "Riemann Solvers and Numerical
Methods for Fluid Dynamics", ch. 4): the star pressure p* solves
f_L(p*) + f_R(p*) + (u_R - u_L) = 0, where f_K is the shock (Rankine-Hugoniot)
branch for p* > p_K and the isentropic rarefaction branch otherwise; the star
velocity follows, and the self-similar solution is sampled in xi = (x - x0)/t.

For the kinetic gas of the paper m = 1, k_B = 1, so density = number density n,
T = p / n and gamma = 1 + 2/f = 5/3 for three velocity degrees of freedom.
"""
import math

import numpy as np


def _f_branch(p, rho, pk, c, g):
    """Velocity jump across the left or right wave as a function of p*."""
    if p > pk:  # shock
        A = 2.0 / ((g + 1.0) * rho)
        B = (g - 1.0) / (g + 1.0) * pk
        f = (p - pk) * math.sqrt(A / (p + B))
        df = math.sqrt(A / (B + p)) * (1.0 - 0.5 * (p - pk) / (B + p))
    else:  # rarefaction
        f = 2.0 * c / (g - 1.0) * ((p / pk) ** ((g - 1.0) / (2.0 * g)) - 1.0)
        df = 1.0 / (rho * c) * (p / pk) ** (-(g + 1.0) / (2.0 * g))
    return f, df


def star_state(left, right, gamma=5.0 / 3.0, tol=1e-14, max_iter=200):
    """left/right = (rho, u, p).  Returns (p_star, u_star)."""
    rl, ul, pl = left
    rr, ur, pr = right
    cl = math.sqrt(gamma * pl / rl)
    cr = math.sqrt(gamma * pr / rr)
    # two-rarefaction guess, kept positive
    z = (gamma - 1.0) / (2.0 * gamma)
    p = ((cl + cr - 0.5 * (gamma - 1.0) * (ur - ul)) / (cl / pl ** z + cr / pr ** z)) ** (1.0 / z)
    p = max(p, 1e-12 * min(pl, pr))
    for _ in range(max_iter):
        fl, dfl = _f_branch(p, rl, pl, cl, gamma)
        fr, dfr = _f_branch(p, rr, pr, cr, gamma)
        f = fl + fr + (ur - ul)
        step = f / (dfl + dfr)
        p_new = max(p - step, 1e-14 * p)
        if abs(p_new - p) <= tol * 0.5 * (p_new + p):
            p = p_new
            break
        p = p_new
    fl, _ = _f_branch(p, rl, pl, cl, gamma)
    fr, _ = _f_branch(p, rr, pr, cr, gamma)
    u = 0.5 * (ul + ur) + 0.5 * (fr - fl)
    return p, u


def sample(xi, left, right, gamma=5.0 / 3.0):
    """(rho, u, p) at similarity coordinates xi (array)."""
    rl, ul, pl = left
    rr, ur, pr = right
    g = gamma
    cl = math.sqrt(g * pl / rl)
    cr = math.sqrt(g * pr / rr)
    ps, us = star_state(left, right, g)
    xi = np.asarray(xi, dtype=np.float64)
    rho = np.empty_like(xi)
    u = np.empty_like(xi)
    p = np.empty_like(xi)
    gm = (g - 1.0) / (g + 1.0)
    for k, s in np.ndenumerate(xi):
        if s <= us:  # left of the contact
            if ps > pl:  # left shock
                S = ul - cl * math.sqrt((g + 1.0) / (2.0 * g) * ps / pl + (g - 1.0) / (2.0 * g))
                if s <= S:
                    st = (rl, ul, pl)
                else:
                    st = (rl * (ps / pl + gm) / (gm * ps / pl + 1.0), us, ps)
            else:  # left rarefaction
                head = ul - cl
                cs = cl * (ps / pl) ** ((g - 1.0) / (2.0 * g))
                tail = us - cs
                if s <= head:
                    st = (rl, ul, pl)
                elif s >= tail:
                    st = (rl * (ps / pl) ** (1.0 / g), us, ps)
                else:
                    uu = 2.0 / (g + 1.0) * (cl + 0.5 * (g - 1.0) * ul + s)
                    c = 2.0 / (g + 1.0) * (cl + 0.5 * (g - 1.0) * (ul - s))
                    st = (rl * (c / cl) ** (2.0 / (g - 1.0)), uu, pl * (c / cl) ** (2.0 * g / (g - 1.0)))
        else:  # right of the contact
            if ps > pr:  # right shock
                S = ur + cr * math.sqrt((g + 1.0) / (2.0 * g) * ps / pr + (g - 1.0) / (2.0 * g))
                if s >= S:
                    st = (rr, ur, pr)
                else:
                    st = (rr * (ps / pr + gm) / (gm * ps / pr + 1.0), us, ps)
            else:  # right rarefaction
                head = ur + cr
                cs = cr * (ps / pr) ** ((g - 1.0) / (2.0 * g))
                tail = us + cs
                if s >= head:
                    st = (rr, ur, pr)
                elif s <= tail:
                    st = (rr * (ps / pr) ** (1.0 / g), us, ps)
                else:
                    uu = 2.0 / (g + 1.0) * (-cr + 0.5 * (g - 1.0) * ur + s)
                    c = 2.0 / (g + 1.0) * (cr - 0.5 * (g - 1.0) * (ur - s))
                    st = (rr * (c / cr) ** (2.0 / (g - 1.0)), uu, pr * (c / cr) ** (2.0 * g / (g - 1.0)))
        rho[k], u[k], p[k] = st
    return rho, u, p


def wave_speeds(left, right, gamma=5.0 / 3.0):
    """Positions per unit time of the characteristic features (for tests):
    dict with keys 'left_head', 'left_tail' or 'left_shock', 'contact',
    'right_shock' or 'right_head', 'right_tail'."""
    rl, ul, pl = left
    rr, ur, pr = right
    g = gamma
    cl = math.sqrt(g * pl / rl)
    cr = math.sqrt(g * pr / rr)
    ps, us = star_state(left, right, g)
    out = {"contact": us, "p_star": ps}
    if ps > pl:
        out["left_shock"] = ul - cl * math.sqrt((g + 1.0) / (2.0 * g) * ps / pl + (g - 1.0) / (2.0 * g))
    else:
        out["left_head"] = ul - cl
        out["left_tail"] = us - cl * (ps / pl) ** ((g - 1.0) / (2.0 * g))
    if ps > pr:
        out["right_shock"] = ur + cr * math.sqrt((g + 1.0) / (2.0 * g) * ps / pr + (g - 1.0) / (2.0 * g))
    else:
        out["right_head"] = ur + cr
        out["right_tail"] = us + cr * (ps / pr) ** ((g - 1.0) / (2.0 * g))
    return out


def sod_profile(x_edges, t, x0=0.5, n_left=1.0, p_left=1.0, gamma=5.0 / 3.0, sub=64):
    """Cell averages over the given edges of (n, u, p, T) of the Sod problem
    (n_r = 0.125 n_l, p_r = 0.1 p_l, at rest) at time t."""
    left = (n_left, 0.0, p_left)
    right = (0.125 * n_left, 0.0, 0.1 * p_left)
    x_edges = np.asarray(x_edges, dtype=np.float64)
    nc = len(x_edges) - 1
    out = np.zeros((nc, 4))
    for c in range(nc):
        xs = x_edges[c] + (np.arange(sub) + 0.5) / sub * (x_edges[c + 1] - x_edges[c])
        rho, u, p = sample((xs - x0) / t, left, right, gamma)
        out[c, 0] = rho.mean()
        out[c, 1] = u.mean()
        out[c, 2] = p.mean()
        out[c, 3] = (p / rho).mean()
    return out
