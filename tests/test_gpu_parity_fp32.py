"""GPU FP32 path against the FP64 oracle.

The FP32 path stores populations in FP32 and runs the transforms, equilibria
and update in FP32; the reported moments sum the FP32 populations in FP64.
Its error against the FP64 oracle therefore grows with the step count; the
bound used here is derived from FP32 rounding: each step perturbs every
population by about 10 units in the last place (u = 2^-24 ~ 6e-8; the
moment blocks have condition numbers up to ~10^3 after the scaling that the
factorised back-map applies, so a step's error is ~10 u relative), and over
n steps the rounding errors of a damped explicit scheme add at most linearly:
relative L-infinity <= 30 u n^0.5 + 3e-6 is checked, with n the step count,
for smooth flows. With shocks the FP32 rounding perturbs the discrete shock
profile, and the L-infinity difference at the few nodes inside a shock is
larger; for the supersonic reflection the bar is the measured value with a
2x margin (2e-4 after 40 steps), and the L1 error E of Sec. V.A is reported.
"""
import math

import numpy as np
import pytest

import workloads as W
from harness import field_errors, gpu_run, l1_errors, oracle_run, pop_error

pytestmark = pytest.mark.gpu

U32 = 2.0 ** -24


def bound(n):
    return 30 * U32 * math.sqrt(max(n, 1)) + 3e-6


CASES = [
    ("periodic", lambda: W.random_state(70, 19, seed=70, smooth=True), 100, None),
    ("bcs", lambda: W.random_state(64, 17, seed=9, smooth=True,
                                   bc=(("eq", (1.0, 0.3, 0.0, 1.0)), ("extrap", None),
                                       ("reflect", None), ("eq", (1.2, 0.25, -0.1, 1.1)))), 100, None),
    ("sod", lambda: W.sod_config1("stable", ny=4), 1000, None),
    ("reflection", lambda: W.regular_reflection(), 40, 2e-4),
]


@pytest.mark.parametrize("name,make,nsteps,tol", CASES, ids=[c[0] for c in CASES])
def test_fp32_within_bound(name, make, nsteps, tol):
    w = make()
    got, f, status = gpu_run(w, nsteps, "fp32")
    ref, fref = oracle_run(w, nsteps)
    err = field_errors(got, ref)
    perr = pop_error(f, fref)
    tol = bound(nsteps) if tol is None else tol
    where = {k: np.unravel_index(np.abs(got[k] - ref[k]).argmax(), ref[k].shape) for k in err}
    print("fp32 %s n=%d Linf %s pop %.3g L1 %s at %s tol %.3g"
          % (name, nsteps, err, perr, l1_errors(got, ref), where, tol))
    assert max(err.values()) <= tol, (err, tol, where)
    assert status[0] == 0
