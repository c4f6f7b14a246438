"""Exact solution of the Riemann problem for two ideal gases, one on each
side of the initial discontinuity (the air-helium shock tube of Sec. 4.1.5):
the star pressure from f_L(p) + f_R(p) + u_R - u_L = 0 by Newton's method,
with the classical shock (Rankine-Hugoniot) and rarefaction (isentropic)
branches of f_K, then the self-similar solution sampled at x / t.  Written
for the tests from the gas dynamics; it shares nothing with the oracle."""
import numpy as np


def _f(p, g, r, pk):
    """f_K and its derivative for side K (gamma g, density r, pressure pk)."""
    c = np.sqrt(g * pk / r)
    if p > pk:  # shock
        A, B = 2.0 / ((g + 1.0) * r), (g - 1.0) / (g + 1.0) * pk
        s = np.sqrt(A / (p + B))
        return (p - pk) * s, s * (1.0 - 0.5 * (p - pk) / (B + p))
    e = (g - 1.0) / (2.0 * g)
    return 2.0 * c / (g - 1.0) * ((p / pk) ** e - 1.0), (p / pk) ** (-(g + 1.0) / (2.0 * g)) / (r * c)


def star_state(left, right):
    """(p*, u*) for left = (gamma, rho, u, p), right likewise."""
    gL, rL, uL, pL = left
    gR, rR, uR, pR = right
    p = 0.5 * (pL + pR)
    for _ in range(200):
        fl, dl = _f(p, gL, rL, pL)
        fr, dr = _f(p, gR, rR, pR)
        dp = (fl + fr + uR - uL) / (dl + dr)
        p = max(p - dp, 1e-14 * p)
        if abs(dp) <= 1e-15 * p:
            break
    fl, _ = _f(p, gL, rL, pL)
    fr, _ = _f(p, gR, rR, pR)
    return p, 0.5 * (uL + uR) + 0.5 * (fr - fl)


def sample(xi, left, right):
    """(rho, u, p, side) at xi = (x - x0)/t; side 0 left gas, 1 right gas.
    Only the pattern of the shock tube is handled: a rarefaction into the
    left gas and a shock into the right gas (p_L > p* > p_R)."""
    gL, rL, uL, pL = left
    gR, rR, uR, pR = right
    p, us = star_state(left, right)
    assert pL > p > pR, "left rarefaction / right shock expected"
    cL, cR = np.sqrt(gL * pL / rL), np.sqrt(gR * pR / rR)
    rsl = rL * (p / pL) ** (1.0 / gL)
    csl = cL * (p / pL) ** ((gL - 1.0) / (2.0 * gL))
    q = (gR - 1.0) / (gR + 1.0)
    rsr = rR * (p / pR + q) / (q * p / pR + 1.0)
    sR = uR + cR * np.sqrt((gR + 1.0) / (2.0 * gR) * p / pR + (gR - 1.0) / (2.0 * gR))
    out = np.empty((4, len(xi)))
    for i, s in enumerate(xi):
        if s < us:
            if s <= uL - cL:
                out[:, i] = (rL, uL, pL, 0)
            elif s >= us - csl:
                out[:, i] = (rsl, us, p, 0)
            else:  # inside the fan
                c = 2.0 / (gL + 1.0) * (cL + 0.5 * (gL - 1.0) * (uL - s))
                out[:, i] = (rL * (c / cL) ** (2.0 / (gL - 1.0)),
                             2.0 / (gL + 1.0) * (cL + 0.5 * (gL - 1.0) * uL + s),
                             pL * (c / cL) ** (2.0 * gL / (gL - 1.0)), 0)
        else:
            out[:, i] = (rsr, us, p, 1) if s < sR else (rR, uR, pR, 1)
    return out, dict(p=p, u=us, rho_l=rsl, rho_r=rsr, shock=sR)
