"""The MRT finite-difference LB scheme, step by step, in plain FP64 numpy.

Test infrastructure only (see ``oracle/__init__``).

Passages followed
-----------------
* Eq. 3 (Sec. II): df/dt + v.grad f = -M^-1 S_hat (f_hat - f_hat^eq).
* Eq. 14a-14i (Sec. III.B): equilibria of the non-conserved moments;
  f_hat^eq_12 = f_hat^eq_15 = f_hat^eq_16 = 0 as the text after Eq. 14 chooses.
* Appendix, Eq. A.1a/A.1b: forward-Euler time step and the per-axis
  Lax-Wendroff space term (central difference minus v^2 dt/2 times the second
  difference; no mixed x-y term).
* Sec. V: boundary nodes carry f = f^eq of a boundary state -- fixed
  (Dirichlet), periodic, reflecting (normal velocity reversed, Sec. V.B.a) or
  linearly extrapolated (Sec. V.B.a, V.C).

Readings where the paper is silent or ambiguous
-----------------------------------------------
R1  R = 1, two translational degrees of freedom, no internal ones. The moment
    set fixes e = rho T + rho |u|^2 / 2 (m_4 = |v|^2/2, Eq. 5d, with the
    momentum flux of Eq. 9b and f_hat^eq_5 of Eq. 14a), so
    P = rho T = e - |j|^2 / (2 rho) and gamma = 2. T = e/rho - |u|^2/2.
R2  Velocity-space equilibrium f^eq = M^-1 f_hat^eq (Sec. II mapping); it may
    have small negative entries.
R3  The appendix calls the time step "upwind" but writes forward Euler with the
    Lax-Wendroff space term A.1b; the formula is followed. The collision term
    is evaluated at the node at time n.
R4  Relaxation: Delta m_k = -dt s_k (m_k - m_k^eq); for s_k dt = 1 the moment
    is reset to its equilibrium.
R5  Grid: cell-centred interior nodes plus one ghost node per non-periodic
    side. Ghosts are refreshed every step from the interior at time n. The
    5-point cross stencil never reads corner ghosts (they stay NaN here).
R6  Reflecting side: the ghost state is (rho, u, v, T) of the adjacent
    interior node with the velocity component normal to that side negated.
R7  Extrapolating side: ghost q = 2 q_1 - q_2 for q in (rho, u, v, T), q_1 the
    adjacent node and q_2 the next one in; if that gives rho <= 0 or T <= 0
    (or the grid is one node deep) the ghost takes q_1.
R8  Moving isothermal wall (Couette, Sec. V.D: "constant speed and constant
    temperature"): the ghost state is (rho of the adjacent node, u_w, v_w,
    T_w); the paper does not say what density the wall node carries.
R22 Side split along its length (Mach reflection, Sec. V.B.b): the ghost
    of the node at s = (index + 1/2) h along the side takes the near kind
    where s <= s0 + s1 t and the far kind beyond, t the time of the state
    being advanced (the paper's g(t) for the top, 150 dx for the bottom).
R20 Open side of problems the paper does not pose (2D Riemann quadrants):
    zero-gradient outflow, the ghost state is the adjacent node's state
    (zero-order extrapolation; the first-order one of R7 amplifies waves that
    cross such a side).
"""
import numpy as np

from .lattice import matrices

SIDES = ("x-", "x+", "y-", "y+")


# ----------------------------------------------------------------------------
# Moments and equilibria
# ----------------------------------------------------------------------------
def conserved_from_state(rho, u, v, T):
    """(rho, j_x, j_y, e) of a state (rho, u, v, T) under reading R1."""
    dt = np.result_type(rho, u, v, T, np.float64)   # float64 (or wider)
    rho, u, v, T = (np.asarray(q, dtype=dt) for q in (rho, u, v, T))
    return rho, rho * u, rho * v, rho * T + 0.5 * rho * (u * u + v * v)


def moment_equilibria(rho, jx, jy, e):
    """Eq. 14: the 16 equilibrium moments as a (16, ...) array.

    Rows 1-4 are the conserved moments themselves; rows 12, 15, 16 are zero.
    P = e - |j|^2/(2 rho) by reading R1.
    """
    rho = np.asarray(rho, dtype=np.result_type(rho, np.float64))
    jx2 = jx * jx
    jy2 = jy * jy
    jsq = jx2 + jy2
    P = e - jsq / (2.0 * rho)
    zero = np.zeros_like(rho)
    out = [
        rho,
        jx,
        jy,
        e,
        (jx2 - jy2) / rho,                                    # 14a
        jx * jy / rho,                                        # 14b
        (e + P) * jx / rho,                                   # 14c
        (e + P) * jy / rho,                                   # 14d
        (jx2 - 3.0 * jy2) * jx / rho ** 2,                    # 14e
        (3.0 * jx2 - jy2) * jy / rho ** 2,                    # 14f
        2.0 * e * e / rho - jsq * jsq / (4.0 * rho ** 3),     # 14g
        zero,                                                 # f12 = 0
        (6.0 * rho * e - 2.0 * jx2 - 2.0 * jy2) * (jx2 - jy2) / rho ** 3,  # 14h
        (6.0 * rho * e - 2.0 * jx2 - 2.0 * jy2) * jx * jy / rho ** 3,      # 14i
        zero,                                                 # f15 = 0
        zero,                                                 # f16 = 0
    ]
    return np.stack(np.broadcast_arrays(*out))


def moments(f):
    """f_hat = M f for f of shape (16, ...)."""
    _, M, _ = matrices()
    return np.tensordot(M, f, axes=(1, 0))


def macroscopic(f):
    """(rho, u, v, T) of populations f (16, ...) via rows 1-4 of M (Sec. III.A)
    and reading R1."""
    m = moments(f)
    rho, jx, jy, e = m[0], m[1], m[2], m[3]
    u = jx / rho
    v = jy / rho
    T = e / rho - 0.5 * (u * u + v * v)
    return rho, u, v, T


def equilibrium_populations(rho, u, v, T):
    """f^eq = M^-1 f_hat^eq(rho, j, e) (reading R2)."""
    _, _, Minv = matrices()
    meq = moment_equilibria(*conserved_from_state(rho, u, v, T))
    return np.tensordot(Minv, meq, axes=(1, 0))


def collision(f, s, dt):
    """Eq. 3's right-hand side times dt, i.e. the population change
    Delta f = M^-1 (-dt S_hat (f_hat - f_hat^eq)) at every node (reading R4).

    ``s`` is the 16 diagonal entries of S_hat (s_1..s_4 have no effect: the
    conserved moments equal their equilibria)."""
    _, M, Minv = matrices()
    m = np.tensordot(M, f, axes=(1, 0))
    meq = moment_equilibria(m[0], m[1], m[2], m[3])
    shape = (16,) + (1,) * (f.ndim - 1)
    dm = -dt * np.asarray(s, dtype=np.float64).reshape(shape) * (m - meq)
    return np.tensordot(Minv, dm, axes=(1, 0))


# ----------------------------------------------------------------------------
# Boundary (ghost) nodes
# ----------------------------------------------------------------------------
def _extrapolate(q1, q2):
    """Reading R7 on arrays of states: 2 q1 - q2, q1 where that is unphysical."""
    qe = [2.0 * a - b for a, b in zip(q1, q2)]
    bad = ~((qe[0] > 0.0) & (qe[3] > 0.0))
    return [np.where(bad, a, b) for a, b in zip(q1, qe)]


def _ghost_line(f, side, bc, t=0.0, h=1.0):
    """Ghost populations next to one side, shape (16, n) (n = ny for x sides,
    nx for y sides), from the interior f (16, ny, nx) at time t. ``bc`` is
    (kind, state) or, for a side split along its length (reading R22),
    (kind, state, (far_kind, s0, s1)): the ghost of the node at position
    s = (index + 1/2) h along the side takes ``kind`` where s <= s0 + s1 t
    and ``far_kind`` beyond."""
    if len(bc) > 2 and bc[2] is not None:
        far, s0, s1 = bc[2]
        near_line = _ghost_line(f, side, bc[:2])
        far_line = _ghost_line(f, side, (far, bc[1]))
        s = (np.arange(near_line.shape[1]) + 0.5) * h
        return np.where(s <= s0 + s1 * t, near_line, far_line)
    kind, state = bc
    xs = side[0] == "x"
    lo = side[1] == "-"
    if xs:
        first = f[:, :, 0] if lo else f[:, :, -1]
        second = (f[:, :, 1] if lo else f[:, :, -2]) if f.shape[2] > 1 else first
        opposite = f[:, :, -1] if lo else f[:, :, 0]
        n = f.shape[1]
    else:
        first = f[:, 0, :] if lo else f[:, -1, :]
        second = (f[:, 1, :] if lo else f[:, -2, :]) if f.shape[1] > 1 else first
        opposite = f[:, -1, :] if lo else f[:, 0, :]
        n = f.shape[2]
    if kind == "periodic":
        return opposite.copy()
    if kind == "eq":
        rho, u, v, T = (np.full(n, float(x)) for x in state)
        return equilibrium_populations(rho, u, v, T)
    if kind == "reflect":
        rho, u, v, T = macroscopic(first)
        if xs:
            u = -u
        else:
            v = -v
        return equilibrium_populations(rho, u, v, T)
    if kind == "extrap":
        q1 = list(macroscopic(first))
        q2 = list(macroscopic(second))
        return equilibrium_populations(*_extrapolate(q1, q2))
    if kind == "outflow":
        # zero-gradient open side: the adjacent node's state unchanged
        return equilibrium_populations(*macroscopic(first))
    if kind == "wall":
        rho = macroscopic(first)[0]
        _, uw, vw, Tw = (float(x) for x in state)
        return equilibrium_populations(rho, np.full(n, uw), np.full(n, vw),
                                       np.full(n, Tw))
    raise ValueError("unknown boundary kind %r" % (kind,))


def padded(f, bcs, t=0.0, dx=1.0, dy=1.0):
    """Interior f (16, ny, nx) at time t surrounded by one ring of ghost
    nodes (16, ny+2, nx+2). Corner ghosts are NaN: the cross stencil never
    reads them (reading R5)."""
    q, ny, nx = f.shape
    g = np.full((q, ny + 2, nx + 2), np.nan)
    g[:, 1:-1, 1:-1] = f
    g[:, 1:-1, 0] = _ghost_line(f, "x-", bcs[0], t, dy)
    g[:, 1:-1, -1] = _ghost_line(f, "x+", bcs[1], t, dy)
    g[:, 0, 1:-1] = _ghost_line(f, "y-", bcs[2], t, dx)
    g[:, -1, 1:-1] = _ghost_line(f, "y+", bcs[3], t, dx)
    return g


def check_bcs(bcs):
    for a, b in ((0, 1), (2, 3)):
        if (bcs[a][0] == "periodic") != (bcs[b][0] == "periodic"):
            raise ValueError("periodic must be set on both opposite sides")


# ----------------------------------------------------------------------------
# One time step
# ----------------------------------------------------------------------------
def advection(g, dx, dy, dt):
    """Eq. A.1b: v_i . grad f_i with the Lax-Wendroff second-difference term,
    evaluated at every interior node of the ghost-padded array g."""
    v, _, _ = matrices()
    vx = v[:, 0].reshape(16, 1, 1)
    vy = v[:, 1].reshape(16, 1, 1)
    c = g[:, 1:-1, 1:-1]
    e_ = g[:, 1:-1, 2:]
    w_ = g[:, 1:-1, :-2]
    n_ = g[:, 2:, 1:-1]
    s_ = g[:, :-2, 1:-1]
    return (vx * (e_ - w_) / (2.0 * dx)
            + vy * (n_ - s_) / (2.0 * dy)
            - vx * vx * dt * (e_ - 2.0 * c + w_) / (2.0 * dx * dx)
            - vy * vy * dt * (n_ - 2.0 * c + s_) / (2.0 * dy * dy))


def step(f, cfg, t=0.0):
    """One time step of Eq. 3 discretised by Eq. A.1 from time t:
    f(t+dt) = f - dt * [v.grad f]_A.1b + Delta f_collision, all terms at t.

    ``cfg`` needs keys dx, dy, dt, s (16 rates) and bc (4 pairs (kind, state),
    or split triples, for sides x-, x+, y-, y+)."""
    g = padded(f, cfg["bc"], t, cfg["dx"], cfg["dy"])
    dt = cfg["dt"]
    return f - dt * advection(g, cfg["dx"], cfg["dy"], dt) + collision(f, cfg["s"], dt)


def init_populations(rho, u, v, T):
    """Initial populations: f = f^eq of the initial fields (Sec. V: the
    paper sets f_i = f_i^eq from the initial macroscopic state)."""
    return equilibrium_populations(rho, u, v, T)


def run(f, cfg, nsteps, check_every=0, level0=0):
    """Advance ``nsteps`` steps from time level ``level0`` (time level0 dt).
    Returns (f, first_bad) where first_bad is the first checked time level
    (counted from level0 = the input state) at which some node is
    non-finite or has rho <= 0, checked every ``check_every`` steps
    (0: never); the run stops there."""
    check_bcs(cfg["bc"])
    for n in range(nsteps):
        if check_every and n % check_every == 0 and not physical(f):
            return f, n
        f = step(f, cfg, (level0 + n) * cfg["dt"])
    if check_every and not physical(f):
        return f, nsteps
    return f, None


def physical(f):
    """True when every population is finite and rho > 0 at every node.

    T <= 0 is not part of this test: the scheme's overshoots at
    discontinuities can make T slightly negative for a few steps from which
    it recovers (see ``positive_temperature``)."""
    rho = moments(f)[0]
    return bool(np.isfinite(f).all() and np.all(rho > 0.0))


def positive_temperature(f):
    """True when T > 0 at every node."""
    return bool(np.all(macroscopic(f)[3] > 0.0))


def conserved_totals(f, dx, dy):
    """Grid sums of (rho, j_x, j_y, e) times the cell area (FP64)."""
    m = moments(f)
    return np.array([m[k].sum() for k in range(4)]) * dx * dy
