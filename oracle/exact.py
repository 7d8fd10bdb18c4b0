"""Reference solutions against which the scheme is checked (Sec. V).

Test infrastructure only (see ``oracle/__init__``).

* ``riemann_sample``   -- exact solution of the 1D Euler Riemann problem, the
  "exact solutions" the shock-tube figures of Sec. V.A compare with. The paper
  names no solver; this is the textbook exact iterative method (pressure
  function, Newton iteration for p*, self-similar sampling; E. F. Toro,
  "Riemann Solvers and Numerical Methods for Fluid Dynamics", ch. 4), written
  for a general gamma and used at gamma = 2 (reading R1 of ``scheme``).
* ``normal_shock`` / ``moving_shock`` / ``oblique_shock`` -- Rankine-Hugoniot
  jump conditions; they reproduce the post-shock states printed for the
  regular reflection (Sec. V.B.a), the Mach reflection (Sec. V.B.b) and the
  shock-bubble problems (Sec. V.C).
* ``couette_u``        -- the analytic Couette velocity series of Sec. V.D.
* ``relative_error``   -- E = sum |num - exa| / sum |exa| of Sec. V.A.
"""
import math

import numpy as np

GAMMA = 2.0


# ----------------------------------------------------------------------------
# Exact Riemann solver
# ----------------------------------------------------------------------------
def _pressure_function(p, rho_k, p_k, gamma):
    """f_K(p) and its derivative: shock branch for p > p_K, rarefaction else."""
    a_k = math.sqrt(gamma * p_k / rho_k)
    if p > p_k:
        A = 2.0 / ((gamma + 1.0) * rho_k)
        B = (gamma - 1.0) / (gamma + 1.0) * p_k
        sq = math.sqrt(A / (p + B))
        return (p - p_k) * sq, sq * (1.0 - 0.5 * (p - p_k) / (B + p))
    g1 = (gamma - 1.0) / (2.0 * gamma)
    return (2.0 * a_k / (gamma - 1.0) * ((p / p_k) ** g1 - 1.0),
            (p / p_k) ** (-(gamma + 1.0) / (2.0 * gamma)) / (rho_k * a_k))


def star_state(left, right, gamma=GAMMA, tol=1e-14, maxit=200):
    """(p*, u*) for primitive states (rho, u, p) on the two sides."""
    rl, ul, pl = left
    rr, ur, pr = right
    al = math.sqrt(gamma * pl / rl)
    ar = math.sqrt(gamma * pr / rr)
    if 2.0 * (al + ar) / (gamma - 1.0) <= ur - ul:
        raise ValueError("vacuum is generated; not handled")
    # two-rarefaction guess, then Newton on f_L + f_R + (u_R - u_L) = 0
    g1 = (gamma - 1.0) / (2.0 * gamma)
    p = ((al + ar - 0.5 * (gamma - 1.0) * (ur - ul))
         / (al / pl ** g1 + ar / pr ** g1)) ** (1.0 / g1)
    p = max(p, 1e-12)
    for _ in range(maxit):
        fl, dl = _pressure_function(p, rl, pl, gamma)
        fr, dr = _pressure_function(p, rr, pr, gamma)
        pn = p - (fl + fr + ur - ul) / (dl + dr)
        pn = max(pn, 1e-14)
        if abs(pn - p) <= tol * 0.5 * (pn + p):
            p = pn
            break
        p = pn
    fl, _ = _pressure_function(p, rl, pl, gamma)
    fr, _ = _pressure_function(p, rr, pr, gamma)
    return p, 0.5 * (ul + ur) + 0.5 * (fr - fl)


def riemann_sample(left, right, xi, gamma=GAMMA):
    """Exact solution (rho, u, p) at similarity coordinates xi = x/t.

    ``left``/``right`` are (rho, u, p); ``xi`` an array. Sampling follows the
    wave pattern: left wave (shock or fan), contact, right wave."""
    rl, ul, pl = left
    rr, ur, pr = right
    ps, us = star_state(left, right, gamma)
    al = math.sqrt(gamma * pl / rl)
    ar = math.sqrt(gamma * pr / rr)
    gm = (gamma - 1.0) / (gamma + 1.0)
    xi = np.asarray(xi, dtype=np.float64)
    rho = np.empty_like(xi)
    u = np.empty_like(xi)
    p = np.empty_like(xi)
    for n, s in np.ndenumerate(xi):
        if s <= us:  # left of the contact
            if ps > pl:  # left shock
                rs = rl * ((ps / pl + gm) / (gm * ps / pl + 1.0))
                sl = ul - al * math.sqrt((gamma + 1.0) / (2.0 * gamma) * ps / pl
                                         + (gamma - 1.0) / (2.0 * gamma))
                val = (rl, ul, pl) if s <= sl else (rs, us, ps)
            else:  # left rarefaction
                rs = rl * (ps / pl) ** (1.0 / gamma)
                asl = al * (ps / pl) ** ((gamma - 1.0) / (2.0 * gamma))
                if s <= ul - al:
                    val = (rl, ul, pl)
                elif s >= us - asl:
                    val = (rs, us, ps)
                else:
                    c = 2.0 / (gamma + 1.0) + gm / al * (ul - s)
                    val = (rl * c ** (2.0 / (gamma - 1.0)),
                           2.0 / (gamma + 1.0) * (al + 0.5 * (gamma - 1.0) * ul + s),
                           pl * c ** (2.0 * gamma / (gamma - 1.0)))
        else:  # right of the contact
            if ps > pr:  # right shock
                rs = rr * ((ps / pr + gm) / (gm * ps / pr + 1.0))
                sr = ur + ar * math.sqrt((gamma + 1.0) / (2.0 * gamma) * ps / pr
                                         + (gamma - 1.0) / (2.0 * gamma))
                val = (rr, ur, pr) if s >= sr else (rs, us, ps)
            else:  # right rarefaction
                rs = rr * (ps / pr) ** (1.0 / gamma)
                asr = ar * (ps / pr) ** ((gamma - 1.0) / (2.0 * gamma))
                if s >= ur + ar:
                    val = (rr, ur, pr)
                elif s <= us + asr:
                    val = (rs, us, ps)
                else:
                    c = 2.0 / (gamma + 1.0) - gm / ar * (ur - s)
                    val = (rr * c ** (2.0 / (gamma - 1.0)),
                           2.0 / (gamma + 1.0) * (-ar + 0.5 * (gamma - 1.0) * ur + s),
                           pr * c ** (2.0 * gamma / (gamma - 1.0)))
        rho[n], u[n], p[n] = val
    return rho, u, p


# ----------------------------------------------------------------------------
# Rankine-Hugoniot relations
# ----------------------------------------------------------------------------
def normal_shock(rho1, un1, p1, gamma=GAMMA):
    """Shock-frame jump for upstream normal velocity un1 > a1: returns
    (rho2, un2, p2)."""
    a1 = math.sqrt(gamma * p1 / rho1)
    M2 = (un1 / a1) ** 2
    rho2 = rho1 * (gamma + 1.0) * M2 / ((gamma - 1.0) * M2 + 2.0)
    p2 = p1 * (1.0 + 2.0 * gamma / (gamma + 1.0) * (M2 - 1.0))
    return rho2, un1 * rho1 / rho2, p2


def moving_shock(rho1, p1, Ms, direction, gamma=GAMMA):
    """Post-shock (rho, u, v, p) behind a shock of Mach number Ms running
    into gas at rest (rho1, p1) along the unit vector ``direction``."""
    a1 = math.sqrt(gamma * p1 / rho1)
    rho2, un2, p2 = normal_shock(rho1, Ms * a1, p1, gamma)
    speed = Ms * a1 - un2  # lab-frame gas speed behind the shock
    return rho2, speed * direction[0], speed * direction[1], p2


def oblique_shock(rho1, u1, v1, p1, beta, gamma=GAMMA):
    """Downstream (rho, u, v, p) for a steady oblique shock whose line makes
    the angle ``beta`` (radians) below the upstream flow direction, the flow
    crossing it from the side it comes from (the geometry of Sec. V.B.a)."""
    th = math.atan2(v1, u1)
    t = (math.cos(th - beta), math.sin(th - beta))   # along the shock line
    n = (-t[1], t[0])                                # normal, pointing downstream
    un = u1 * n[0] + v1 * n[1]
    ut = u1 * t[0] + v1 * t[1]
    rho2, un2, p2 = normal_shock(rho1, un, p1, gamma)
    return rho2, un2 * n[0] + ut * t[0], un2 * n[1] + ut * t[1], p2


# ----------------------------------------------------------------------------
# Couette flow and the error measure
# ----------------------------------------------------------------------------
def couette_u(y, t, U, D, mu, rho, terms=2000):
    """Sec. V.D series: u = 2yU/D - sum_j (-1)^(j+1) 2U/(j pi)
    exp(-4 j^2 pi^2 mu t / (rho D^2)) sin(2 j pi y / D), walls at y = +-D/2."""
    y = np.asarray(y, dtype=np.float64)
    out = 2.0 * y * U / D
    for j in range(1, terms + 1):
        amp = math.exp(-4.0 * j * j * math.pi ** 2 * mu * t / (rho * D * D))
        if amp < 1e-300:
            break
        out = out - (-1.0) ** (j + 1) * 2.0 * U / (j * math.pi) * amp \
            * np.sin(2.0 * j * math.pi * y / D)
    return out


def relative_error(num, exa):
    """Sec. V.A: E = sum_I |num - exa| / sum_I |exa|."""
    num = np.asarray(num, dtype=np.float64)
    exa = np.asarray(exa, dtype=np.float64)
    return float(np.abs(num - exa).sum() / np.abs(exa).sum())
