"""Split sides (reading R22) and the Mach reflection of Sec. V.B.b.

* A split side's ghost line takes the near kind up to s0 + s1 t along the
  side and the far kind beyond, and the split moves with t.
* Mach reflection at the paper's resolution (dx = dy = 0.003, dt = 1e-5,
  rates of Sec. V.B.b) on a 200 x 100 domain with the wedge tip at node 50
  (the set-up is self-similar about the tip): the top side switches from the
  post-shock inflow to extrapolation at g(t), which moves at 1.5 / sin 30 x
  tan 30 = sqrt(3) along the top. The incident shock inside the domain, found
  on the last interior row, must move along with g: its displacement over
  1200 steps within 15 % of g's, and it stays within 2 nodes of g (it trails
  by ~1.1 nodes, the smeared shock's half width).
"""
import math

import numpy as np

import workloads as W
from oracle import scheme


def test_split_side_ghost_follows_position_and_time():
    w = W.random_state(6, 5, seed=3)
    f = scheme.init_populations(*w.fields())
    state = (1.2, 0.1, 0.0, 0.9)
    near = scheme._ghost_line(f, "y+", ("eq", state))
    far = scheme._ghost_line(f, "y+", ("extrap", None))
    h, s0, s1 = 0.1, 0.22, 0.5
    for t, n_near in ((0.0, 2), (0.2, 3), (0.6, 5)):          # s = 0.05, 0.15, ... <= 0.22 + 0.5 t
        line = scheme._ghost_line(f, "y+", ("eq", state, ("extrap", s0, s1)), t, h)
        np.testing.assert_array_equal(line[:, :n_near], near[:, :n_near])
        np.testing.assert_array_equal(line[:, n_near:], far[:, n_near:])


def _top_shock_x(f, w):
    rho = scheme.macroscopic(f)[0][-2]                  # last-but-one interior row
    mid = 0.5 * (W.MACH_PRE[0] + W.MACH_POST[0])
    i = int(np.where(rho < mid)[0][0])
    xa = (i - 0.5) * w.dx
    return xa + (rho[i - 1] - mid) / (rho[i - 1] - rho[i]) * w.dx


def test_mach_reflection_incident_shock_follows_the_moving_top_side():
    w = W.mach_reflection(nx=200, ny=100, dx=0.003, dt=1e-5, foot=50)
    g = lambda t: w.meta["foot"] + math.tan(math.pi / 6) * (w.meta["H"] + 1.5 * t / math.sin(math.pi / 6))
    f = scheme.init_populations(*w.fields())
    x0 = _top_shock_x(f, w)
    n = 1200
    f, bad = scheme.run(f, w.cfg(), n, check_every=100)
    assert bad is None
    t = n * w.dt
    x1 = _top_shock_x(f, w)
    moved, expected = x1 - x0, g(t) - g(0.0)
    assert abs(moved - expected) < 0.15 * expected, (moved, expected)
    assert abs(x1 - g(t)) < 2 * w.dx, (x1, g(t))
