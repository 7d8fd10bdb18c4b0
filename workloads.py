"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle.

This module holds problem set-ups only -- grid sizes, rates, boundary kinds,
boundary states and initial macroscopic fields -- and none of the scheme's
arithmetic. Both sides (the CUDA library through its binding, and the CPU
oracle) receive exactly these arrays.

A ``Workload`` describes one 2D problem:
  nx, ny      interior nodes (x fastest in every array, shape (ny, nx))
  dx, dy, dt  grid spacing and time step
  s           the 16 diagonal relaxation rates s_1..s_16 (s_1..s_4 unused)
  bc          four (kind, state) pairs for the sides x-, x+, y-, y+;
              kind in {"periodic", "eq", "reflect", "extrap", "wall"};
              state = (rho, u, v, T) for "eq" and "wall" (the wall takes rho
              from the adjacent node), else None
  rho,u,v,T   initial fields, float64 arrays of shape (ny, nx)
  nsteps      the number of steps of the full run

Boundary states that are post-shock states were computed with the
Rankine-Hugoniot relations at gamma = 2 (``tests/golden/make_states.py``,
which calls only the oracle); a test checks them.
"""
from dataclasses import dataclass, field
import math

import numpy as np

BC_KINDS = ("periodic", "eq", "reflect", "extrap", "wall")


def rates(default=1e5, **given):
    """16 relaxation rates: ``default`` everywhere, s_k overridden by the
    keyword s<k> (1-based, as in the paper)."""
    s = [float(default)] * 16
    for key, val in given.items():
        k = int(key[1:])
        s[k - 1] = float(val)
    return tuple(s)


@dataclass
class Workload:
    name: str
    nx: int
    ny: int
    dx: float
    dy: float
    dt: float
    s: tuple
    bc: tuple
    rho: np.ndarray
    u: np.ndarray
    v: np.ndarray
    T: np.ndarray
    nsteps: int = 1
    meta: dict = field(default_factory=dict)

    def cfg(self):
        """Plain dict of the scheme parameters (the oracle's input)."""
        return {"nx": self.nx, "ny": self.ny, "dx": self.dx, "dy": self.dy,
                "dt": self.dt, "s": self.s, "bc": self.bc}

    def fields(self):
        return self.rho, self.u, self.v, self.T


def _fill(nx, ny, state):
    return [np.full((ny, nx), float(x)) for x in state]


# ----------------------------------------------------------------------------
# Shock tubes (Sec. V.A)
# ----------------------------------------------------------------------------
SOD_L = (1.0, 0.0, 0.0, 1.0)
SOD_R = (0.125, 0.0, 0.0, 0.8)
LAX_L = (0.445, 0.698, 0.0, 7.928)
LAX_R = (0.5, 0.0, 0.0, 1.142)

# Sod rates of Sec. V.A(a) and the same rates scaled by the grid ratio
# 0.005/0.002 -> x0.4 for the coarser 200-node tube (stable variant).
SOD_RATES_PAPER = rates(s5=500, s6=500, s7=1e3, s8=1e3, s11=2500)
SOD_RATES_STABLE = rates(s5=200, s6=200, s7=400, s8=400, s11=1000)
SOD_RATES_LITERAL = rates()


def shock_tube(left, right, nx, dx, dt, nsteps, s, ny=1, x_interface=None,
               name="shock_tube"):
    """Quasi-1D tube: nx x ny nodes, y periodic, x sides held at the initial
    left/right equilibria (Sec. V.A). Node i sits at x = (i + 1/2) dx; nodes
    with x <= x_interface take the left state (default: the middle)."""
    if x_interface is None:
        x_interface = 0.5 * nx * dx
    x = (np.arange(nx) + 0.5) * dx
    left_mask = np.broadcast_to(x <= x_interface, (ny, nx))
    f = [np.where(left_mask, a, b) for a, b in zip(left, right)]
    bc = (("eq", tuple(left)), ("eq", tuple(right)),
          ("periodic", None), ("periodic", None))
    return Workload(name, nx, ny, dx, dx, dt, tuple(s), bc, *f, nsteps=nsteps,
                    meta={"x_interface": x_interface, "left": left, "right": right})


def sod_config1(rates_kind="literal", ny=4):
    """Sod tube on 200 x ny nodes, dx = dy = 0.005, dt = 1e-5, 10 000 steps
    (t = 0.1), interface at x = 0.5. ``rates_kind``: "literal" (all s = 1e5),
    "stable" (the paper's Sod rates x 0.4) or "paper"."""
    s = {"literal": SOD_RATES_LITERAL, "stable": SOD_RATES_STABLE,
         "paper": SOD_RATES_PAPER}[rates_kind]
    return shock_tube(SOD_L, SOD_R, 200, 0.005, 1e-5, 10000, s, ny=ny,
                      name="sod_200x%d_%s" % (ny, rates_kind))


def sod_paper_case1():
    """Sec. V.A(a) case 1: dx = 0.002, dt = 2e-6, t = 0.18 on x in [-0.5, 0.5]
    (500 nodes; the domain length is not stated in the paper)."""
    return shock_tube(SOD_L, SOD_R, 500, 0.002, 2e-6, 90000, SOD_RATES_PAPER,
                      name="sod_paper_case1")


# ----------------------------------------------------------------------------
# The paper's other shock tubes (Sec. V.A(b)-(e)) and the single-relaxation
# version (Sec. II: S = I / tau; the paper's tau = 1e-5 gives every s = 1e5)
# ----------------------------------------------------------------------------
# name: (left, right, t_end, {case: (dx, dt)}, MRT rates, domain [a, b]); the
# domain (not stated in the paper) holds every wave of the gamma = 2 exact
# solution at t_end with a margin.
PAPER_TUBES = {
    "lax": ((0.445, 0.698, 0.0, 7.928), (0.5, 0.0, 0.0, 1.142), 0.2,
            {1: (0.004, 4e-6), 2: (0.002, 2e-6), 3: (0.001, 1e-6)},
            rates(s7=3e3, s8=3e3, s13=1e2), (-0.8, 0.8)),
    "colella": ((1.0, 0.0, 0.0, 1000.0), (1.0, 0.0, 0.0, 0.01), 0.1,
                {1: (0.002, 2e-6), 2: (0.001, 1e-6)},
                rates(s7=5e4, s8=5e4, s11=5e5, s13=5e5), (-5.0, 3.0)),
    "two_shock": ((5.99924, 19.5975, 0.0, 76.8254), (5.99242, -6.19633, 0.0, 7.69222), 0.1,
                  {1: (0.003, 1e-5)}, rates(s5=5e3, s6=5e3, s7=3e4, s8=3e4), (-0.5, 1.8)),
    "high_mach": ((5.0, 45.0, 0.0, 10.0), (6.0, -20.0, 0.0, 5.0), 0.018,
                  {1: (0.003, 1e-5)}, rates(s5=1.5e4, s6=1.5e4, s10=5e4), (-0.3, 0.7)),
}
SRT_RATES = rates()   # every s = 1 / tau = 1e5


def paper_tube(name, case=1, srt=False, ny=1):
    """Sec. V.A shock tube ``name`` (lax, colella, two_shock, high_mach) at
    the paper's grid and time step of ``case``, the paper's MRT rates or
    (srt) the single relaxation time tau = 1e-5, on x in [a, b] with the
    interface at x = 0; nsteps reaches the paper's t_end. meta holds a, the
    end time and the two states (for the exact solution)."""
    left, right, t_end, grids, mrt, (a, b) = PAPER_TUBES[name]
    dx, dt = grids[case]
    nx = int(round((b - a) / dx))
    w = shock_tube(left, right, nx, dx, dt, int(round(t_end / dt)), SRT_RATES if srt else mrt,
                   ny=ny, x_interface=-a, name="%s_case%d_%s" % (name, case, "srt" if srt else "mrt"))
    w.meta.update(a=a, t_end=t_end)
    return w


# ----------------------------------------------------------------------------
# Regular shock reflection (Sec. V.B.a geometry)
# ----------------------------------------------------------------------------
# Paper's Mach-5 problem: inflow (1, 5, 0, 0.5), top (2.27273, 4.3, -1.21244, 1.76).
REFLECT_M5_IN = (1.0, 5.0, 0.0, 0.5)
REFLECT_M5_TOP = (2.27273, 4.3, -1.21244, 1.76)
# Mach 2.9 inflow with pre-shock rho = 1, T = 1 (sound speed sqrt(2) at
# gamma = 2), 30-degree incident shock: post-shock state from the oblique
# Rankine-Hugoniot relations (T = p / rho).
REFLECT_M29_IN = (1.0, 2.9 * math.sqrt(2.0), 0.0, 1.0)
REFLECT_M29_TOP = (1.5374771480804381, 3.742789341797761, -0.6208189520502188,
                   1.6065279429250885)
REFLECT_RATES = rates(s5=1e4, s6=2e3, s7=1e4, s8=1e4)


def regular_reflection(nx=600, ny=200, dx=1e-3, dt=2e-6, nsteps=20000,
                       inflow=REFLECT_M29_IN, top=REFLECT_M29_TOP):
    """Left: inflow held (Dirichlet); top: post-shock state held; bottom:
    reflecting wall; right: linear extrapolation; interior starts at the
    inflow state (Sec. V.B.a)."""
    f = _fill(nx, ny, inflow)
    bc = (("eq", tuple(inflow)), ("extrap", None), ("reflect", None),
          ("eq", tuple(top)))
    return Workload("regular_reflection_%dx%d" % (nx, ny), nx, ny, dx, dx, dt,
                    REFLECT_RATES, bc, *f, nsteps=nsteps)


# ----------------------------------------------------------------------------
# Shock-bubble interaction (Sec. V.C)
# ----------------------------------------------------------------------------
BUBBLE_PRE = (1.0, 0.0, 0.0, 1.0)                 # (rho, u, v, T), p = 1
BUBBLE_POST = (1.28, -0.3774, 0.0, 1.6512 / 1.28)  # p = 1.6512
BUBBLE_RATES = rates(s5=1e4, s6=1e4, s7=1e4, s8=1e4)


def shock_bubble(nx=2048, ny=1024, dx=1e-3, dt=1e-5, radius=128,
                 bubble_rho=0.1358, nsteps=2000, s=None):
    """Mach-1.22 planar shock (post-shock gas on the right, moving left) and a
    light circular bubble in pressure equilibrium (p = 1, T = 1/rho_b), centre
    (nx/2, ny/2), shock plane ``radius + 32`` nodes to the right of the
    centre. Right: post-shock inflow held; left: extrapolation; top and
    bottom: reflecting (Sec. V.C)."""
    rho, u, v, T = _fill(nx, ny, BUBBLE_PRE)
    ix = np.arange(nx)[None, :] + 0.5
    iy = np.arange(ny)[:, None] + 0.5
    cx, cy = 0.5 * nx, 0.5 * ny
    inside = (ix - cx) ** 2 + (iy - cy) ** 2 <= radius ** 2
    rho = np.where(inside, bubble_rho, rho)
    T = np.where(inside, 1.0 / bubble_rho, T)
    post = np.broadcast_to(ix > cx + radius + 32, (ny, nx))
    fields = [np.where(post, p, q) for p, q in zip(BUBBLE_POST, (rho, u, v, T))]
    bc = (("extrap", None), ("eq", BUBBLE_POST), ("reflect", None),
          ("reflect", None))
    return Workload("shock_bubble_%dx%d" % (nx, ny), nx, ny, dx, dx, dt,
                    BUBBLE_RATES if s is None else s, bc, *fields, nsteps=nsteps)


# Sec. V.C, second case: a heavy bubble (rho 3.1538, p = 1), s5 = 1e3.
HEAVY_BUBBLE_RHO = 3.1538
HEAVY_BUBBLE_RATES = rates(s5=1e3)


def heavy_bubble(nx=2048, ny=1024, dx=1e-3, dt=1e-5, radius=128, nsteps=2000):
    """The shock-bubble set-up of ``shock_bubble`` with the paper's heavy
    bubble and its rates."""
    w = shock_bubble(nx, ny, dx, dt, radius, HEAVY_BUBBLE_RHO, nsteps, s=HEAVY_BUBBLE_RATES)
    w.name = "heavy_bubble_%dx%d" % (nx, ny)
    return w


# ----------------------------------------------------------------------------
# Mach reflection (Sec. V.B.b)
# ----------------------------------------------------------------------------
MACH_PRE = (2.0, 0.0, 0.0, 0.5)
MACH_POST = (3.17647, 0.555556 * math.cos(math.pi / 6), -0.555556 * math.sin(math.pi / 6), 0.839506)
MACH_RATES = rates(s5=1e3, s6=5e2, s7=1e3, s8=1e3)


def mach_reflection(nx=600, ny=300, dx=0.003, dt=1e-5, nsteps=25000, foot=150):
    """Sec. V.B.b: a Mach-1.5 planar shock (post-shock state MACH_POST behind
    it, MACH_PRE ahead) meets a 30-degree wedge whose tip is at x = foot dx on
    the bottom. Initially the post-shock region is y >= h(x, 0), h(x, t) =
    tan 60 (x - foot dx) - 1.5 t / sin 30 (cell-centred nodes). Sides: left
    held at the post-shock state; right linear extrapolation; bottom the
    post-shock state for x <= foot dx and reflecting beyond; top the
    post-shock state for x <= g(t) = foot dx + tan 30 (H + 1.5 t / sin 30),
    H the domain height (0.9 in the paper), and extrapolation beyond --
    both as split sides (reading R22)."""
    x = (np.arange(nx)[None, :] + 0.5) * dx
    y = (np.arange(ny)[:, None] + 0.5) * dx
    h0 = math.tan(math.pi / 3) * (x - foot * dx)
    post = np.broadcast_to(y >= h0, (ny, nx))
    fields = [np.where(post, a, b) for a, b in zip(MACH_POST, MACH_PRE)]
    H = ny * dx
    t30 = math.tan(math.pi / 6)
    bc = (("eq", MACH_POST), ("extrap", None),
          ("eq", MACH_POST, ("reflect", foot * dx, 0.0)),
          ("eq", MACH_POST, ("extrap", foot * dx + t30 * H, t30 * 1.5 / math.sin(math.pi / 6))))
    return Workload("mach_reflection_%dx%d" % (nx, ny), nx, ny, dx, dx, dt, MACH_RATES, bc,
                    *fields, nsteps=nsteps, meta={"foot": foot * dx, "H": H})


# ----------------------------------------------------------------------------
# Couette flow (Sec. V.D)
# ----------------------------------------------------------------------------
def couette(NX=16, NY=32, d=0.004, dt=1e-5, U=0.1, t_end=57.5, s=None):
    """Plates at y = -D/2 and +D/2 moving at -U and +U, D = NY d. The walls sit
    on ghost nodes j = 0 and j = NY, so the evolved rows are j = 1..NY-1 at
    y_j = -D/2 + j d; x is periodic. Walls hold (u, v, T) = (+-U, 0, 1) and
    take rho from the adjacent node."""
    ny = NY - 1
    rho, u, v, T = _fill(NX, ny, (1.0, 0.0, 0.0, 1.0))
    bc = (("periodic", None), ("periodic", None),
          ("wall", (1.0, -U, 0.0, 1.0)), ("wall", (1.0, U, 0.0, 1.0)))
    nsteps = int(round(t_end / dt))
    y = -0.5 * NY * d + d * np.arange(1, NY)
    return Workload("couette_%dx%d" % (NX, NY), NX, ny, d, d, dt,
                    tuple(s) if s is not None else rates(), bc, rho, u, v, T,
                    nsteps=nsteps, meta={"U": U, "D": NY * d, "y": y})


# ----------------------------------------------------------------------------
# Seeded random states (parity cases)
# ----------------------------------------------------------------------------
def random_state(nx, ny, seed, bc=None, dx=0.01, dt=1e-5, s=None, smooth=True,
                 umax=0.5, name=None):
    """Seeded positive states: rho in [0.5, 2], T in [0.5, 1.5],
    |u|, |v| <= umax. ``smooth`` superposes a few random Fourier modes;
    otherwise every node is drawn independently."""
    rng = np.random.default_rng(seed)
    if s is None:
        s = tuple(float(x) for x in 10.0 ** rng.uniform(2.0, 5.0, 16))
    if bc is None:
        bc = (("periodic", None),) * 4
    if smooth:
        X = (np.arange(nx)[None, :] + 0.5) / nx
        Y = (np.arange(ny)[:, None] + 0.5) / ny

        def field_():
            out = np.zeros((ny, nx))
            for _ in range(4):
                kx, ky = rng.integers(0, 4, 2)
                ph = rng.uniform(0, 2 * np.pi)
                out = out + rng.uniform(-1, 1) * np.cos(2 * np.pi * (kx * X + ky * Y) + ph)
            return out / 4.0
    else:
        def field_():
            return rng.uniform(-1, 1, (ny, nx))
    rho = 1.25 + 0.75 * field_()
    u = umax * field_()
    v = umax * field_()
    T = 1.0 + 0.5 * field_()
    return Workload(name or "random_%dx%d_s%d" % (nx, ny, seed), nx, ny, dx, dx,
                    dt, tuple(s), tuple(bc), rho, u, v, T, nsteps=1)


def tube_batch(ntubes=4096, nx_min=128, nx_max=2048, seed=0):
    """Batched quasi-1D Riemann problems: tube lengths Nx ~ U[nx_min, nx_max]
    (integers), left/right rho and T log-uniform in [0.1, 10], u uniform in
    [-1, 1], v = 0. Each tube spans x in [0, 1] (dx = 1/Nx), interface at 0.5,
    dt = 1e-5, 10 000 steps; the Sod-type rates scale with dx:
    s5 = s6 = 200 (0.005/dx), s7 = s8 = 400 (0.005/dx), s11 = 1000 (0.005/dx),
    each capped at 1e5, all others 1e5.
    Returns a dict of numpy arrays (one row per tube)."""
    rng = np.random.default_rng(seed)
    nx = rng.integers(nx_min, nx_max + 1, ntubes)
    lo, hi = math.log(0.1), math.log(10.0)
    rho = np.exp(rng.uniform(lo, hi, (ntubes, 2)))
    T = np.exp(rng.uniform(lo, hi, (ntubes, 2)))
    u = rng.uniform(-1.0, 1.0, (ntubes, 2))
    dx = 1.0 / nx
    scale = 0.005 / dx
    s = np.full((ntubes, 16), 1e5)
    for k, base in ((5, 200.0), (6, 200.0), (7, 400.0), (8, 400.0), (11, 1000.0)):
        s[:, k - 1] = np.minimum(base * scale, 1e5)
    return {"nx": nx.astype(np.int64), "dx": dx, "dt": 1e-5, "nsteps": 10000,
            "left": np.stack([rho[:, 0], u[:, 0], np.zeros(ntubes), T[:, 0]], 1),
            "right": np.stack([rho[:, 1], u[:, 1], np.zeros(ntubes), T[:, 1]], 1),
            "s": s}



def tube_fields(B):
    """The batch's initial (rho, u, v, T), each one array over all tubes'
    nodes in tube order: the left state at x <= 0.5, the right beyond."""
    fields = []
    for q in range(4):
        parts = []
        for t in range(len(B["nx"])):
            x = (np.arange(B["nx"][t]) + 0.5) / B["nx"][t]
            parts.append(np.where(x <= 0.5, B["left"][t, q], B["right"][t, q]))
        fields.append(np.concatenate(parts))
    return fields


# ----------------------------------------------------------------------------
# Linear stability (Sec. IV)
# ----------------------------------------------------------------------------
def vn_example(nk=181):
    """The stability example of Sec. IV: state (rho, u, v, T) = (2, 10, 0, 2),
    dx = dy = 2e-3, dt = 1e-5; MRT rates s5 = 6500, s7 = s8 = 9e4, s9 = 8e4,
    s13 = 7e4, s14 = 8e3, s15 = 2.5e4, others 1e5, and the single-relaxation
    version tau = 1e-5 (every s = 1e5); nk wave numbers k dx uniformly in
    [0, pi] along x."""
    mrt = np.full(16, 1e5)
    for k, val in ((5, 6500.0), (7, 9e4), (8, 9e4), (9, 8e4), (13, 7e4), (14, 8e3), (15, 2.5e4)):
        mrt[k - 1] = val
    dx = 2e-3
    th = np.linspace(0.0, np.pi, nk)
    state = (2.0, 10.0, 0.0, 2.0)
    return {"names": ["mrt", "srt"], "states": np.array([state, state]),
            "rates": np.stack([mrt, np.full(16, 1e5)]), "dx": dx, "dy": dx, "dt": 1e-5,
            "k": np.stack([th / dx, np.zeros(nk)], 1)}

# ----------------------------------------------------------------------------
# 2D Riemann quadrant problems (learned-corrector data)
# ----------------------------------------------------------------------------
def quadrant(seed, n, dt=1e-5, rt_range=(0.1, 10.0), umax=1.0):
    """Seeded 2D Riemann problem on the unit square, n x n nodes: four
    constant states in the quadrants split at (0.5, 0.5), rho and T
    log-uniform in ``rt_range`` (default [0.1, 10]), u and v uniform in
    [-umax, umax]; linear extrapolation on all four sides; dx = 1/n; the
    Sod-type rates scaled with dx as for the tubes (s5 = s6 = 200 (0.005/dx),
    s7 = s8 = 400 (0.005/dx), s11 = 1000 (0.005/dx), capped at 1e5; others
    1e5). The same seed gives the same states at every n."""
    rng = np.random.default_rng(seed)
    lo, hi = math.log(rt_range[0]), math.log(rt_range[1])
    rho = np.exp(rng.uniform(lo, hi, 4))
    T = np.exp(rng.uniform(lo, hi, 4))
    u = rng.uniform(-umax, umax, 4)
    v = rng.uniform(-umax, umax, 4)
    dx = 1.0 / n
    X = (np.arange(n)[None, :] + 0.5) * dx
    Y = (np.arange(n)[:, None] + 0.5) * dx
    q = (X > 0.5).astype(int) + 2 * (Y > 0.5).astype(int)   # quadrant index 0..3
    scale = 0.005 / dx
    s = list(rates())
    for k, base in ((5, 200.0), (6, 200.0), (7, 400.0), (8, 400.0), (11, 1000.0)):
        s[k - 1] = min(base * scale, 1e5)
    bc = (("extrap", None),) * 4
    return Workload("quadrant_%d_n%d" % (seed, n), n, n, dx, dx, dt, tuple(s), bc,
                    rho[q], u[q], v[q], T[q], nsteps=1,
                    meta={"seed": seed, "states": np.stack([rho, u, v, T], 1)})


# Quadrant problems for the learned corrector. At the full contrast of the
# configuration (rho, T in [0.1, 10], |u|, |v| <= 1) the scheme itself goes
# unphysical (rho <= 0 or T <= 0) for most draws; measured validity of the
# 2048 x 2048 reference runs to t = 0.02 / 0.05 over 8 draws: 4 / 1 of 8 at
# [0.3, 3] and 0.5, 8 / 6 at [0.5, 2] and 0.3, 8 / 8 at [0.7, 1.4] and 0.2.
CORRECTOR_RT_RANGE = (0.5, 2.0)
CORRECTOR_UMAX = 0.3
CORRECTOR_WIDTH = 0.004   # interface half-width: 2 nodes at n = 512


def corrector_quadrant(seed, n, dt=1e-5, width=CORRECTOR_WIDTH):
    """Corrector problems: the four states of ``quadrant`` (rho, T
    log-uniform in CORRECTOR_RT_RANGE, |u|, |v| <= CORRECTOR_UMAX) laid out
    as a doubly periodic 2 x 2 checkerboard -- state q for x in (0.25, 0.75)
    or not, times the same in y -- joined by tanh steps of a fixed physical
    half-width at 0.25 and 0.75 in each direction (H(s) = (tanh((s - 0.25)
    / width) - tanh((s - 0.75) / width)) / 2), periodic on all sides, and
    the Sod-type rates of ``quadrant`` scaled with 0.005 / dx (a fixed
    relaxation length in nodes). Every resolution starts from the same
    continuous state. Open sides fail at n >= 512: where a quadrant interface
    meets an open side (linear extrapolation or zero-gradient outflow) the
    flow speeds up along the side and T goes negative in every draw tried;
    rates fixed across resolutions leave the fine runs with relaxation
    lengths of tens of nodes, and they go unphysical inside."""
    w = quadrant(seed, n, dt, rt_range=CORRECTOR_RT_RANGE, umax=CORRECTOR_UMAX)
    st = w.meta["states"]                      # rows: quadrants 0..3; (rho, u, v, T)
    x = (np.arange(n) + 0.5) / n
    h = 0.5 * (np.tanh((x - 0.25) / width) - np.tanh((x - 0.75) / width))
    hx, hy = h[None, :], h[:, None]
    wts = ((1 - hx) * (1 - hy), hx * (1 - hy), (1 - hx) * hy, hx * hy)
    w.rho, w.u, w.v, w.T = (sum(wt * st[q, k] for q, wt in enumerate(wts)) for k in range(4))
    w.bc = (("periodic", None),) * 4
    return w
