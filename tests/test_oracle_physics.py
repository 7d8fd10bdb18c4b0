"""Whole-scheme pins of the oracle against the paper's numerical experiments.

* Sod tube, Sec. V.A(a) case 1 (dx = 0.002, dt = 2e-6, t = 0.18, the paper's
  rates): the velocity error E_u against the exact gamma = 2 Riemann solution
  is within 15 % of the printed 3.32 % (E_u does not depend on the unstated
  domain length, since u = 0 outside the wave fan), and the star-region
  plateaus match the exact p* and u*.
* Couette flow, Sec. V.D case 1 geometry (NY = 32, dy = 0.004, walls on the
  ghost nodes) with time rescaled by 20 (dt x 20, s / 20, t / 20; the same
  s dt = 1 and the same mu t / D^2): E_u against the series with
  mu = rho T / s_5 (Eq. 15), summed over the vertical line of NY + 1 nodes
  including the two wall nodes, is within [5 %, 9 %] (printed case 1:
  7.02 %), and a viscosity off by a factor 1.5 either way misses by far.
* Sod tube on 200 x 1 nodes, dx = 0.005, dt = 1e-5 with every rate 1e5
  becomes unphysical (rho <= 0 or non-finite somewhere) after about a
  thousand steps, while the paper's Sod rates scaled to that grid run through
  all 10 000 steps.
"""
import math

import numpy as np
import pytest

import workloads as W
from oracle import exact, scheme


@pytest.mark.slow
def test_sod_paper_case1_velocity_error_and_plateaus():
    w = W.sod_paper_case1()
    f, bad = scheme.run(scheme.init_populations(*w.fields()), w.cfg(), w.nsteps)
    assert bad is None
    rho, u, v, T = (q[0] for q in scheme.macroscopic(f))
    t = w.nsteps * w.dt
    x = (np.arange(w.nx) + 0.5) * w.dx - 0.5
    L, R = (1.0, 0.0, 1.0), (0.125, 0.0, 0.1)
    re, ue, pe = exact.riemann_sample(L, R, x / t)
    E_u = exact.relative_error(u, ue)
    assert abs(E_u - 0.0332) < 0.15 * 0.0332, E_u
    ps, us = exact.star_state(L, R)
    # plateau between the fan tail and the contact, and between contact and shock
    p = rho * T
    sel = (x / t > us - 0.25) & (x / t < us - 0.08)
    assert np.abs(u[sel] - us).max() < 0.02 * us and np.abs(p[sel] - ps).max() < 0.02 * ps
    assert abs(v).max() < 1e-12


@pytest.mark.slow
def test_couette_velocity_profile():
    NY, d, dt, s5 = 32, 0.004, 2e-4, 5e3
    D = NY * d
    w = W.couette(NX=1, NY=NY, d=d, dt=dt, t_end=57.5 / 20, s=W.rates(s5))
    f, bad = scheme.run(scheme.init_populations(*w.fields()), w.cfg(), w.nsteps)
    rho, u, v, T = (q[:, 0] for q in scheme.macroscopic(f))
    y = w.meta["y"]
    t = w.nsteps * dt
    line = lambda a: np.r_[-0.1, a, 0.1]   # walls at y = -D/2, +D/2
    E = {fac: exact.relative_error(line(u), line(exact.couette_u(y, t, 0.1, D, fac / s5, 1.0)))
         for fac in (1 / 1.5, 1.0, 2.0)}
    assert 0.05 < E[1.0] < 0.09, E
    assert E[1 / 1.5] > 0.15 and E[2.0] > E[1.0], E
    # mirror symmetry of the problem: u odd, rho and T even about the centre
    assert np.abs(u + u[::-1]).max() < 1e-12
    assert np.abs(T - T[::-1]).max() < 1e-12 and np.abs(rho - rho[::-1]).max() < 1e-12


def test_sod_all_rates_1e5_becomes_unphysical():
    w = W.sod_config1("literal", ny=1)
    _, bad = scheme.run(scheme.init_populations(*w.fields()), w.cfg(), 2000, check_every=1)
    assert bad is not None and 500 < bad < 2000


@pytest.mark.slow
def test_sod_scaled_rates_run_through():
    w = W.sod_config1("stable", ny=1)
    f, bad = scheme.run(scheme.init_populations(*w.fields()), w.cfg(), w.nsteps, check_every=100)
    assert bad is None and scheme.positive_temperature(f)
    rho, u, v, T = (q[0] for q in scheme.macroscopic(f))
    x = (np.arange(w.nx) + 0.5) * w.dx - 0.5
    re, ue, pe = exact.riemann_sample((1.0, 0.0, 1.0), (0.125, 0.0, 0.1), x / (w.nsteps * w.dt))
    assert exact.relative_error(u, ue) < 0.12   # coarse grid: about 10 %
