"""Exact solution of the 1D Euler Riemann problem (ideal gas), written from the textbook method
(Toro, "Riemann Solvers and Numerical Methods for Fluid Dynamics", Chapter 4): Newton iteration
for the star pressure with the shock/rarefaction pressure functions, then sampling of the wave
pattern.  Test helper only; it shares nothing with the oracle's HLLC solver."""
import math

import numpy as np


def _fK(p, rho, pK, c, g):
    if p > pK:  # shock
        A = 2.0 / ((g + 1.0) * rho)
        B = (g - 1.0) / (g + 1.0) * pK
        q = math.sqrt(A / (p + B))
        return (p - pK) * q, q * (1.0 - 0.5 * (p - pK) / (B + p))
    pr = p / pK  # rarefaction
    f = 2.0 * c / (g - 1.0) * (pr ** ((g - 1.0) / (2.0 * g)) - 1.0)
    df = 1.0 / (rho * c) * pr ** (-(g + 1.0) / (2.0 * g))
    return f, df


def star_state(L, R, g=1.4):
    rL, uL, pL = L
    rR, uR, pR = R
    cL, cR = math.sqrt(g * pL / rL), math.sqrt(g * pR / rR)
    p = max(1e-8, 0.5 * (pL + pR))
    for _ in range(200):
        fL, dL = _fK(p, rL, pL, cL, g)
        fR, dR = _fK(p, rR, pR, cR, g)
        dp = (fL + fR + uR - uL) / (dL + dR)
        pn = max(1e-10, p - dp)
        if abs(pn - p) <= 1e-15 * (pn + p):
            p = pn
            break
        p = pn
    fL, _ = _fK(p, rL, pL, cL, g)
    fR, _ = _fK(p, rR, pR, cR, g)
    u = 0.5 * (uL + uR) + 0.5 * (fR - fL)
    return p, u


def sample(L, R, s, g=1.4):
    """Primitive (rho, u, p) at x/t = s."""
    rL, uL, pL = L
    rR, uR, pR = R
    cL, cR = math.sqrt(g * pL / rL), math.sqrt(g * pR / rR)
    ps, us = star_state(L, R, g)
    gm = (g - 1.0) / (g + 1.0)
    if s <= us:  # left of the contact
        if ps > pL:
            SL = uL - cL * math.sqrt((g + 1) / (2 * g) * ps / pL + (g - 1) / (2 * g))
            if s <= SL:
                return rL, uL, pL
            return rL * (ps / pL + gm) / (gm * ps / pL + 1.0), us, ps
        csL = cL * (ps / pL) ** ((g - 1) / (2 * g))
        if s <= uL - cL:
            return rL, uL, pL
        if s >= us - csL:
            return rL * (ps / pL) ** (1 / g), us, ps
        u = 2 / (g + 1) * (cL + (g - 1) / 2 * uL + s)
        c = 2 / (g + 1) * (cL + (g - 1) / 2 * (uL - s))
        r = rL * (c / cL) ** (2 / (g - 1))
        return r, u, pL * (c / cL) ** (2 * g / (g - 1))
    if ps > pR:
        SR = uR + cR * math.sqrt((g + 1) / (2 * g) * ps / pR + (g - 1) / (2 * g))
        if s >= SR:
            return rR, uR, pR
        return rR * (ps / pR + gm) / (gm * ps / pR + 1.0), us, ps
    csR = cR * (ps / pR) ** ((g - 1) / (2 * g))
    if s >= uR + cR:
        return rR, uR, pR
    if s <= us + csR:
        return rR * (ps / pR) ** (1 / g), us, ps
    u = 2 / (g + 1) * (-cR + (g - 1) / 2 * uR + s)
    c = 2 / (g + 1) * (cR - (g - 1) / 2 * (uR - s))
    r = rR * (c / cR) ** (2 / (g - 1))
    return r, u, pR * (c / cR) ** (2 * g / (g - 1))


def density_averages(L, R, x0, x1, nx, xs, t, g=1.4, sub=64):
    dx = (x1 - x0) / nx
    out = np.zeros(nx)
    for i in range(nx):
        xs_ = x0 + (i + (np.arange(sub) + 0.5) / sub) * dx
        out[i] = np.mean([sample(L, R, (x - xs) / t, g)[0] for x in xs_])
    return out
