"""Exact solution of the 1D Riemann problem for an ideal gas (Sod's shock tube).

TEST INFRASTRUCTURE ONLY (pins the oracle on the Sod tube of Sec. IV.C.1).
Own implementation of the textbook method (Toro, "Riemann Solvers and
Numerical Methods for Fluid Dynamics", ch. 4): the star pressure is the root
of f_L(p) + f_R(p) + (u_R - u_L) = 0, found by Newton's method; the solution
is then sampled along x/t. Units: p = rho T, sound speed c = sqrt(gamma p / rho).
"""
import math

import numpy as np


def _f_and_df(p, rho, pk, gamma):
    c = math.sqrt(gamma * pk / rho)
    if p > pk:  # shock
        A = 2.0 / ((gamma + 1.0) * rho)
        B = (gamma - 1.0) / (gamma + 1.0) * pk
        sq = math.sqrt(A / (p + B))
        return (p - pk) * sq, sq * (1.0 - 0.5 * (p - pk) / (p + B))
    # rarefaction
    e = (gamma - 1.0) / (2.0 * gamma)
    return (2.0 * c / (gamma - 1.0) * ((p / pk) ** e - 1.0),
            (1.0 / (rho * c)) * (p / pk) ** (-(gamma + 1.0) / (2.0 * gamma)))


def star_state(left, right, gamma=1.4, tol=1e-14, maxit=100):
    """left/right = (rho, u, p). Returns (p_star, u_star)."""
    rl, ul, pl = left
    rr, ur, pr = right
    p = max(1e-12, 0.5 * (pl + pr))
    for _ in range(maxit):
        fl, dfl = _f_and_df(p, rl, pl, gamma)
        fr, dfr = _f_and_df(p, rr, pr, gamma)
        f = fl + fr + (ur - ul)
        dp = f / (dfl + dfr)
        p_new = max(1e-12, p - dp)
        if abs(p_new - p) <= tol * 0.5 * (p_new + p):
            p = p_new
            break
        p = p_new
    fl, _ = _f_and_df(p, rl, pl, gamma)
    fr, _ = _f_and_df(p, rr, pr, gamma)
    u = 0.5 * (ul + ur) + 0.5 * (fr - fl)
    return p, u


def sample(left, right, s, gamma=1.4):
    """Solution (rho, u, p) at similarity coordinates s = x / t (array)."""
    rl, ul, pl = left
    rr, ur, pr = right
    ps, us = star_state(left, right, gamma)
    cl = math.sqrt(gamma * pl / rl)
    cr = math.sqrt(gamma * pr / rr)
    g1 = (gamma - 1.0) / (gamma + 1.0)
    s = np.asarray(s, np.float64)
    rho = np.empty_like(s)
    u = np.empty_like(s)
    p = np.empty_like(s)
    for k, x in np.ndenumerate(s):
        if x <= us:  # left of the contact
            if ps > pl:  # left shock
                r_star = rl * ((ps / pl + g1) / (g1 * ps / pl + 1.0))
                S = ul - cl * math.sqrt((gamma + 1.0) / (2.0 * gamma) * ps / pl
                                        + (gamma - 1.0) / (2.0 * gamma))
                val = (rl, ul, pl) if x <= S else (r_star, us, ps)
            else:  # left rarefaction
                r_star = rl * (ps / pl) ** (1.0 / gamma)
                c_star = cl * (ps / pl) ** ((gamma - 1.0) / (2.0 * gamma))
                head, tail = ul - cl, us - c_star
                if x <= head:
                    val = (rl, ul, pl)
                elif x >= tail:
                    val = (r_star, us, ps)
                else:
                    uu = 2.0 / (gamma + 1.0) * (cl + 0.5 * (gamma - 1.0) * ul + x)
                    cc = 2.0 / (gamma + 1.0) * (cl + 0.5 * (gamma - 1.0) * (ul - x))
                    rr_ = rl * (cc / cl) ** (2.0 / (gamma - 1.0))
                    val = (rr_, uu, pl * (cc / cl) ** (2.0 * gamma / (gamma - 1.0)))
        else:  # right of the contact
            if ps > pr:  # right shock
                r_star = rr * ((ps / pr + g1) / (g1 * ps / pr + 1.0))
                S = ur + cr * math.sqrt((gamma + 1.0) / (2.0 * gamma) * ps / pr
                                        + (gamma - 1.0) / (2.0 * gamma))
                val = (rr, ur, pr) if x >= S else (r_star, us, ps)
            else:  # right rarefaction
                r_star = rr * (ps / pr) ** (1.0 / gamma)
                c_star = cr * (ps / pr) ** ((gamma - 1.0) / (2.0 * gamma))
                head, tail = ur + cr, us + c_star
                if x >= head:
                    val = (rr, ur, pr)
                elif x <= tail:
                    val = (r_star, us, ps)
                else:
                    uu = 2.0 / (gamma + 1.0) * (-cr + 0.5 * (gamma - 1.0) * ur + x)
                    cc = 2.0 / (gamma + 1.0) * (cr - 0.5 * (gamma - 1.0) * (ur - x))
                    rr_ = rr * (cc / cr) ** (2.0 / (gamma - 1.0))
                    val = (rr_, uu, pr * (cc / cr) ** (2.0 * gamma / (gamma - 1.0)))
        rho[k], u[k], p[k] = val
    return rho, u, p


def shock_speed_right(left, right, gamma=1.4):
    rr, ur, pr = right
    ps, _ = star_state(left, right, gamma)
    cr = math.sqrt(gamma * pr / rr)
    return ur + cr * math.sqrt((gamma + 1.0) / (2.0 * gamma) * ps / pr + (gamma - 1.0) / (2.0 * gamma))
