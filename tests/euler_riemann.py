"""Exact solution of the Riemann problem for the 1D Euler equations of an
ideal polytropic gas (the textbook pressure-function method: Newton
iteration for the star pressure, then sampling the self-similar solution at
S = x/t).  Test helper for the paper's Riemann validation (Sec. 4), where
the lattice Boltzmann moments obey the Euler equations (Eq. Euler) with
pressure P = (gamma - 1) tr[rho] eps and gamma = 1 + 2/d."""
import numpy as np


def _f(p, rho, u, pk, gamma):
    a = np.sqrt(gamma * pk / rho)
    if p > pk:   # shock
        A = 2.0 / ((gamma + 1.0) * rho)
        B = (gamma - 1.0) / (gamma + 1.0) * pk
        q = np.sqrt(A / (p + B))
        return (p - pk) * q, q * (1.0 - 0.5 * (p - pk) / (B + p))
    e = (gamma - 1.0) / (2.0 * gamma)   # rarefaction
    return 2.0 * a / (gamma - 1.0) * ((p / pk) ** e - 1.0), (p / pk) ** (-(gamma + 1.0) / (2.0 * gamma)) / (rho * a)


def star_state(L, R, gamma):
    rl, ul, pl = L
    rr, ur, pr = R
    p = 0.5 * (pl + pr)
    for _ in range(100):
        fl, dl = _f(p, rl, ul, pl, gamma)
        fr, dr = _f(p, rr, ur, pr, gamma)
        dp = (fl + fr + ur - ul) / (dl + dr)
        pn = max(p - dp, 1e-12 * p)
        if abs(pn - p) <= 1e-14 * p:
            p = pn
            break
        p = pn
    fl, _ = _f(p, rl, ul, pl, gamma)
    fr, _ = _f(p, rr, ur, pr, gamma)
    return p, 0.5 * (ul + ur) + 0.5 * (fr - fl)


def sample(L, R, gamma, S):
    """(rho, u, p) of the exact solution at the similarity variables S."""
    rl, ul, pl = L
    rr, ur, pr = R
    ps, us = star_state(L, R, gamma)
    al, ar = np.sqrt(gamma * pl / rl), np.sqrt(gamma * pr / rr)
    g1, g2 = (gamma - 1.0) / (gamma + 1.0), (gamma - 1.0) / (2.0 * gamma)
    out = np.zeros((3, len(S)))
    for k, s in enumerate(np.asarray(S, float)):
        if s <= us:   # left of the contact
            if ps > pl:
                sl = ul - al * np.sqrt((gamma + 1.0) / (2.0 * gamma) * ps / pl + g2)
                w = (rl, ul, pl) if s <= sl else (rl * (ps / pl + g1) / (g1 * ps / pl + 1.0), us, ps)
            else:
                shl, asl = ul - al, al * (ps / pl) ** g2
                stl = us - asl
                if s <= shl:
                    w = (rl, ul, pl)
                elif s >= stl:
                    w = (rl * (ps / pl) ** (1.0 / gamma), us, ps)
                else:
                    c = 2.0 / (gamma + 1.0) + (gamma - 1.0) / ((gamma + 1.0) * al) * (ul - s)
                    w = (rl * c ** (2.0 / (gamma - 1.0)), 2.0 / (gamma + 1.0) * (al + 0.5 * (gamma - 1.0) * ul + s),
                         pl * c ** (2.0 * gamma / (gamma - 1.0)))
        else:         # right of the contact
            if ps > pr:
                sr = ur + ar * np.sqrt((gamma + 1.0) / (2.0 * gamma) * ps / pr + g2)
                w = (rr, ur, pr) if s >= sr else (rr * (ps / pr + g1) / (g1 * ps / pr + 1.0), us, ps)
            else:
                shr, asr = ur + ar, ar * (ps / pr) ** g2
                str_ = us + asr
                if s >= shr:
                    w = (rr, ur, pr)
                elif s <= str_:
                    w = (rr * (ps / pr) ** (1.0 / gamma), us, ps)
                else:
                    c = 2.0 / (gamma + 1.0) - (gamma - 1.0) / ((gamma + 1.0) * ar) * (ur - s)
                    w = (rr * c ** (2.0 / (gamma - 1.0)), 2.0 / (gamma + 1.0) * (-ar + 0.5 * (gamma - 1.0) * ur + s),
                         pr * c ** (2.0 * gamma / (gamma - 1.0)))
        out[:, k] = w
    return out
