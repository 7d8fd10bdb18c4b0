"""GPU (FP64 path) against the oracle, element by element, through the C ABI.

Bar: relative L-infinity per field (rho, u, v, T; see harness.field_errors)
and for the populations <= 1e-12 for runs up to 100 steps and <= 1e-14 per
step beyond (harness.fp64_tol), on seeded inputs spanning several thread
tiles with ragged edges, on every boundary kind, on the shock-tube and
shock-reflection set-ups at full size, and across CUDA-graph batches.
"""
import numpy as np
import pytest

import workloads as W
from harness import field_errors, fp64_tol, gpu_run, oracle_run, pop_error

pytestmark = pytest.mark.gpu

def _check(w, nsteps, tol=None, precision="fp64"):
    tol = fp64_tol(nsteps) if tol is None else tol
    got, f, status = gpu_run(w, nsteps, precision)
    ref, fref = oracle_run(w, nsteps)
    err = field_errors(got, ref)
    perr = pop_error(f, fref)
    assert max(err.values()) <= tol and perr <= tol, (w.name, nsteps, err, perr)
    return err, perr, status


@pytest.mark.parametrize("nx,ny", [(1, 1), (3, 1), (1, 5), (5, 3), (33, 9), (70, 19), (100, 37)])
@pytest.mark.parametrize("nsteps", [1, 10])
def test_periodic_random(nx, ny, nsteps):
    w = W.random_state(nx, ny, seed=nx * 100 + ny, smooth=(nx * ny > 20))
    _check(w, nsteps)


BC_SETS = [
    (("eq", (1.1, 0.2, 0.05, 0.9)), ("eq", (0.9, -0.1, 0.0, 1.2)), ("periodic", None), ("periodic", None)),
    (("periodic", None), ("periodic", None), ("reflect", None), ("reflect", None)),
    (("extrap", None), ("extrap", None), ("wall", (1.0, -0.1, 0.0, 1.0)), ("wall", (1.0, 0.1, 0.0, 1.0))),
    (("eq", (1.0, 0.3, 0.0, 1.0)), ("extrap", None), ("reflect", None), ("eq", (1.2, 0.25, -0.1, 1.1))),
    (("reflect", None), ("wall", (1.0, 0.0, 0.2, 1.3)), ("extrap", None), ("reflect", None)),
    (("outflow", None), ("outflow", None), ("outflow", None), ("outflow", None)),
    (("outflow", None), ("eq", (1.1, 0.2, 0.0, 0.9)), ("reflect", None), ("outflow", None)),
]


@pytest.mark.parametrize("bcs", range(len(BC_SETS)))
@pytest.mark.parametrize("nx,ny", [(2, 2), (37, 11), (64, 17)])
def test_boundary_kinds(bcs, nx, ny):
    w = W.random_state(nx, ny, seed=7 + bcs, bc=BC_SETS[bcs], smooth=True)
    _check(w, 12)


def test_boundaries_one_node_deep():
    bc = (("extrap", None), ("reflect", None), ("wall", (1.0, 0.1, 0.0, 1.0)), ("extrap", None))
    for nx, ny in ((1, 6), (6, 1), (1, 1)):
        _check(W.random_state(nx, ny, seed=3, bc=bc), 5)


def test_sod_config1_literal_1000_steps():
    _check(W.sod_config1("literal", ny=4), 1000)


def test_sod_config1_stable_full_run():
    """All 10 000 steps within 1e-12 (measured 6.2e-13, test_gpu_error_growth)."""
    w = W.sod_config1("stable", ny=4)
    _check(w, w.nsteps, tol=1e-12)


@pytest.mark.parametrize("nsteps", [1, 10, 100])
def test_regular_reflection_full_size(nsteps):
    w = W.regular_reflection()
    _check(w, nsteps)


def test_regular_reflection_small_long():
    w = W.regular_reflection(nx=90, ny=30, dx=1e-3 * 600 / 90, dt=2e-6 * 600 / 90)
    _check(w, 600)


def test_graph_batches_equal_single_launches():
    """Steps issued as graph replays (64 per batch) equal steps issued one by
    one, bit for bit."""
    w = W.random_state(45, 13, seed=5)
    a, fa, _ = gpu_run(w, 150)
    b, fb, _ = gpu_run(w, 150, chunks=[1] * 150)
    assert np.array_equal(fa, fb)


def test_watchdog_first_bad_step_matches_oracle():
    from oracle import scheme
    w = W.sod_config1("literal", ny=4)
    _, bad_ref = scheme.run(scheme.init_populations(*w.fields()), w.cfg(), 1500, check_every=1)
    _, _, (rc, bad, negT) = gpu_run(w, 1500)
    from paper_0908_3749_gb300.lbm import LBM_ERR_NONFINITE
    assert rc == LBM_ERR_NONFINITE
    assert bad_ref is not None and abs(bad - bad_ref) <= 1, (bad, bad_ref)
    assert 0 <= negT <= bad


def test_no_false_alarm_on_stable_run():
    w = W.sod_config1("stable", ny=4)
    _, _, (rc, bad, negT) = gpu_run(w, 2000)
    assert rc == 0 and bad == -1
