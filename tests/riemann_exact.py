"""Exact solution of the 1-D Euler Riemann problem for an ideal gas (the
textbook wave curves: shock or rarefaction on each side of a contact), used
as the reference of the Sod tests (Sec. 4.1.2, Test 2).  Test helper, not
part of the library or of the oracle."""

import numpy as np


def exact_riemann_density(rhoL, uL, pL, rhoR, uR, pR, gamma, xi):
    """Textbook exact solution of the 1-D Euler Riemann problem (ideal gas),
    density sampled at xi = x/t (two-rarefaction/shock wave curves)."""
    from scipy.optimize import brentq
    cL, cR = np.sqrt(gamma * pL / rhoL), np.sqrt(gamma * pR / rhoR)

    def fK(p, rho, pk, ck):
        if p > pk:
            A = 2.0 / ((gamma + 1) * rho)
            B = (gamma - 1) / (gamma + 1) * pk
            return (p - pk) * np.sqrt(A / (p + B))
        return 2 * ck / (gamma - 1) * ((p / pk) ** ((gamma - 1) / (2 * gamma)) - 1)

    g = lambda p: fK(p, rhoL, pL, cL) + fK(p, rhoR, pR, cR) + uR - uL
    ps = brentq(g, 1e-10, 100.0, xtol=1e-14)
    us = 0.5 * (uL + uR) + 0.5 * (fK(ps, rhoR, pR, cR) - fK(ps, rhoL, pL, cL))
    gm = (gamma - 1) / (gamma + 1)
    out = np.empty_like(xi)
    for k, s in enumerate(xi):
        if s <= us:  # left of contact
            if ps > pL:
                SL = uL - cL * np.sqrt((gamma + 1) / (2 * gamma) * ps / pL + (gamma - 1) / (2 * gamma))
                out[k] = rhoL if s < SL else rhoL * ((ps / pL + gm) / (gm * ps / pL + 1))
            else:
                csL = cL * (ps / pL) ** ((gamma - 1) / (2 * gamma))
                if s < uL - cL:
                    out[k] = rhoL
                elif s > us - csL:
                    out[k] = rhoL * (ps / pL) ** (1 / gamma)
                else:
                    out[k] = rhoL * (2 / (gamma + 1) + gm / cL * (uL - s)) ** (2 / (gamma - 1))
        else:
            if ps > pR:
                SR = uR + cR * np.sqrt((gamma + 1) / (2 * gamma) * ps / pR + (gamma - 1) / (2 * gamma))
                out[k] = rhoR if s > SR else rhoR * ((ps / pR + gm) / (gm * ps / pR + 1))
            else:
                csR = cR * (ps / pR) ** ((gamma - 1) / (2 * gamma))
                if s > uR + cR:
                    out[k] = rhoR
                elif s < us + csR:
                    out[k] = rhoR * (ps / pR) ** (1 / gamma)
                else:
                    out[k] = rhoR * (2 / (gamma + 1) - gm / cR * (uR - s)) ** (2 / (gamma - 1))
    return out
