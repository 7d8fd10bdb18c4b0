"""Pins of the reference solutions (oracle/exact.py) and of the stored
post-shock boundary states in ``workloads``.

* Rankine-Hugoniot at gamma = 2 reproduces the three post-shock states the
  paper prints (Sec. V.B.a, V.B.b, V.C) -- which also pins gamma = 2.
* The exact Riemann solver reproduces the textbook star state of Sod's
  problem at gamma = 1.4 (p* = 0.30313, u* = 0.92745; Toro, Table 4.2) and
  satisfies the jump conditions across the waves it produces.
* The Couette series starts from rest and ends at the linear profile.
"""
import json
import math
import os

import numpy as np
import pytest

import workloads as W
from oracle import exact


@pytest.fixture(scope="module")
def printed(golden_dir):
    with open(os.path.join(golden_dir, "printed_numbers.json")) as fh:
        return json.load(fh)


def test_regular_reflection_top_state(printed):
    p = printed["regular_reflection_mach5"]
    rho, u, v, T = p["inflow_rho_u_v_T"]
    r2, u2, v2, p2 = exact.oblique_shock(rho, u, v, rho * T, math.radians(p["shock_angle_deg"]))
    got = (r2, u2, v2, p2 / r2)
    for a, b in zip(got, p["top_rho_u_v_T"]):
        assert abs(a - b) <= 6e-6 * max(1.0, abs(b)), (got, p["top_rho_u_v_T"])


def test_mach_reflection_post_shock_state(printed):
    p = printed["mach_reflection_ms15"]
    rho1, _, _, T1 = p["pre_rho_u_v_T"]
    ang = math.radians(p["direction_deg"])
    r2, u2, v2, p2 = exact.moving_shock(rho1, rho1 * T1, p["mach"], (math.cos(ang), math.sin(ang)))
    rho_p, speed_p, T_p = p["post_rho_speed_T"]
    assert abs(r2 - rho_p) < 1e-5
    assert abs(math.hypot(u2, v2) - speed_p) < 1e-6
    assert abs(p2 / r2 - T_p) < 1e-6


def test_bubble_post_shock_state(printed):
    p = printed["bubble_ms122"]
    rho1, _, _, p1 = p["pre_rho_u_v_p"]
    r2, u2, v2, p2 = exact.moving_shock(rho1, p1, p["mach"], (-1.0, 0.0))
    want = p["post_rho_u_v_p"]
    assert abs(r2 - want[0]) < 5e-5 and abs(u2 - want[1]) < 5e-5
    assert v2 == 0.0 and abs(p2 - want[3]) < 5e-5


def test_stored_workload_states_match_rh():
    r2, u2, v2, p2 = exact.oblique_shock(1.0, 2.9 * math.sqrt(2.0), 0.0, 1.0, math.radians(30.0))
    np.testing.assert_allclose(W.REFLECT_M29_TOP, (r2, u2, v2, p2 / r2), rtol=1e-14)
    r2, u2, v2, p2 = exact.moving_shock(1.0, 1.0, 1.22, (-1.0, 0.0))
    np.testing.assert_allclose(W.BUBBLE_POST, (1.28, -0.3774, 0.0, 1.6512 / 1.28))
    assert abs(W.BUBBLE_POST[0] - r2) < 5e-5 and abs(W.BUBBLE_POST[1] - u2) < 5e-5


def test_riemann_textbook_sod_gamma14():
    ps, us = exact.star_state((1.0, 0.0, 1.0), (0.125, 0.0, 0.1), gamma=1.4)
    assert abs(ps - 0.30313) < 1e-5 and abs(us - 0.92745) < 1e-5


@pytest.mark.parametrize("gamma", [1.4, 2.0])
def test_riemann_jump_conditions(gamma):
    """Across the right shock of the sampled solution, mass, momentum and
    energy fluxes balance in the shock frame; the left fan is isentropic."""
    L, R = (1.0, 0.0, 1.0), (0.125, 0.0, 0.1)
    ps, us = exact.star_state(L, R, gamma)
    aR = math.sqrt(gamma * R[2] / R[0])
    S = R[1] + aR * math.sqrt((gamma + 1) / (2 * gamma) * ps / R[2] + (gamma - 1) / (2 * gamma))
    rho, u, p = exact.riemann_sample(L, R, np.array([S - 1e-9, S + 1e-9]), gamma)
    assert abs(u[0] - us) < 1e-12 and abs(p[0] - ps) < 1e-12 and rho[1] == R[0]
    m1 = rho[0] * (u[0] - S)
    m2 = rho[1] * (u[1] - S)
    assert abs(m1 - m2) < 1e-10
    assert abs(m1 * (u[0] - S) + p[0] - (m2 * (u[1] - S) + p[1])) < 1e-10
    h = lambda r, uu, pp: gamma / (gamma - 1) * pp / r + 0.5 * (uu - S) ** 2
    assert abs(h(rho[0], u[0], p[0]) - h(rho[1], u[1], p[1])) < 1e-9
    xi = np.linspace(-math.sqrt(gamma * L[2] / L[0]), us - 0.2, 50)
    rho, u, p = exact.riemann_sample(L, R, xi, gamma)
    np.testing.assert_allclose(p / rho ** gamma, L[2] / L[0] ** gamma, rtol=1e-12)
    # Riemann invariant u + 2a/(gamma-1) is constant through the left fan
    a = np.sqrt(gamma * p / rho)
    np.testing.assert_allclose(u + 2 * a / (gamma - 1),
                               L[1] + 2 * math.sqrt(gamma * L[2] / L[0]) / (gamma - 1), rtol=1e-12)


def test_couette_series_limits():
    D, U = 0.128, 0.1
    y = np.linspace(-D / 2 + D / 64, D / 2 - D / 64, 31)
    np.testing.assert_allclose(exact.couette_u(y, 1e6, U, D, 1e-5, 1.0), 2 * y * U / D, atol=1e-12)
    u0 = exact.couette_u(y, 0.0, U, D, 1e-5, 1.0, terms=200000)
    assert np.abs(u0).max() < 2e-3
    assert abs(exact.couette_u(np.array([D / 2]), 1.0, U, D, 1e-5, 1.0)[0] - U) < 1e-12


def test_relative_error_definition():
    assert exact.relative_error([1.0, 2.0], [1.0, 1.0]) == 0.5
