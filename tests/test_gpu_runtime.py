"""GPU tests of the runtime around the step: audits, checkpoint/resume,
device-pointer I/O, streams, and the Couette experiment of Sec. V.D."""
import numpy as np
import pytest

import workloads as W
from harness import field_errors, gpu_run, oracle_run

pytestmark = pytest.mark.gpu


def _ctx(w, precision="fp64", audit_every=0, stream=None):
    from paper_0908_3749_gb300 import lbm
    cfg = lbm.make_config(w.nx, w.ny, w.dx, w.dy, w.dt, w.s, w.bc, precision, audit_every)
    ctx = lbm.lbm_create(cfg, stream)
    lbm.lbm_set_init(ctx, *[np.ascontiguousarray(a) for a in w.fields()])
    return lbm, ctx


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_audit_matches_oracle_totals_and_is_conserved(precision):
    from oracle import scheme
    w = W.random_state(77, 29, seed=12, smooth=False)
    lbm, ctx = _ctx(w, precision, audit_every=5)
    try:
        t0 = np.array(lbm.lbm_audit(ctx))
        f0 = scheme.init_populations(*w.fields())
        ref = scheme.conserved_totals(f0, w.dx, w.dy)
        tol = 1e-13 if precision == "fp64" else 1e-6
        np.testing.assert_allclose(t0, ref, rtol=tol, atol=tol * np.abs(ref).max())
        lbm.lbm_step(ctx, 100)
        log, steps = lbm.lbm_audit_log(ctx)
        assert steps == list(range(0, 100, 5))
        np.testing.assert_allclose(log[0], t0, rtol=1e-15 if precision == "fp64" else 1e-6)
        drift = np.abs(np.array(log) - t0).max(axis=0) / np.abs(t0).max()
        assert drift.max() < (1e-13 if precision == "fp64" else 2e-6), drift
        # bitwise reproducible
        assert lbm.lbm_audit(ctx) == lbm.lbm_audit(ctx)
    finally:
        lbm.lbm_destroy(ctx)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_checkpoint_resume_is_bitwise(precision):
    w = W.regular_reflection(nx=70, ny=23)
    lbm, ctx = _ctx(w, precision)
    try:
        lbm.lbm_step(ctx, 30)
        dt = np.float64 if precision == "fp64" else np.float32
        ck = np.empty((16, w.ny, w.nx), dtype=dt)
        step = lbm.lbm_get_populations(ctx, ck)
        assert step == 30 and lbm.lbm_step_count(ctx) == 30
        lbm.lbm_step(ctx, 77)
        a = np.empty_like(ck)
        lbm.lbm_get_populations(ctx, a)
        lbm.lbm_set_populations(ctx, ck, step)
        lbm.lbm_step(ctx, 77)
        b = np.empty_like(ck)
        assert lbm.lbm_get_populations(ctx, b) == 107
        assert np.array_equal(a, b)
    finally:
        lbm.lbm_destroy(ctx)


def _state(lbm, ctx, shape, dt):
    f = np.empty(shape, dtype=dt)
    step = lbm.lbm_get_populations(ctx, f)
    log, steps = lbm.lbm_audit_log(ctx)
    return f, step, log, steps, lbm.lbm_status(ctx)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_block_count_changes_no_result(precision):
    """Tiles reach the persistent step's blocks through a counter; every block
    count (one block doing all tiles, a few, the default) gives bitwise the
    same populations, audit log and watchdog state."""
    w = W.regular_reflection(nx=300, ny=100)
    dt = np.float64 if precision == "fp64" else np.float32
    states = []
    for blocks in (1, 7, 64, 0):
        lbm, ctx = _ctx(w, precision, audit_every=7)
        try:
            lbm.lbm_set_step_blocks(ctx, blocks)
            assert lbm.lbm_step_blocks(ctx) >= 1
            lbm.lbm_step(ctx, 150)      # two graph replays and 22 single launches
            states.append(_state(lbm, ctx, (16, w.ny, w.nx), dt))
        finally:
            lbm.lbm_destroy(ctx)
    f0, step0, log0, steps0, st0 = states[0]
    assert step0 == 150 and steps0 == list(range(0, 150, 7)) and st0[0] == 0
    for f, step, log, steps, st in states[1:]:
        assert np.array_equal(f, f0)
        assert (step, log, steps, st) == (step0, log0, steps0, st0)


def test_autotune_leaves_state_and_counters_alone():
    from paper_0908_3749_gb300 import lbm as L
    w = W.regular_reflection(nx=200, ny=64)
    shape = (16, w.ny, w.nx)
    lbm, ctx = _ctx(w, "fp32", audit_every=5)
    lbm, ref = _ctx(w, "fp32", audit_every=5)
    try:
        lbm.lbm_step(ctx, 12)
        lbm.lbm_step(ref, 12)
        before = _state(lbm, ctx, shape, np.float32)
        g = lbm.lbm_autotune(ctx, 5)
        assert 1 <= g == lbm.lbm_step_blocks(ctx)
        after = _state(lbm, ctx, shape, np.float32)
        assert np.array_equal(before[0], after[0]) and before[1:] == after[1:]
        lbm.lbm_step(ctx, 70)
        lbm.lbm_step(ref, 70)
        a, b = _state(lbm, ctx, shape, np.float32), _state(lbm, ref, shape, np.float32)
        assert np.array_equal(a[0], b[0]) and a[1:] == b[1:]
    finally:
        lbm.lbm_destroy(ctx)
        lbm.lbm_destroy(ref)
    tc, tctx = _ctx(w, "tc_tf32x3")
    try:
        assert tc.lbm_autotune(tctx, 3) == tc.lbm_step_blocks(tctx)
        with pytest.raises(L.LBMError) as ei:
            tc.lbm_set_step_blocks(tctx, 4)
        assert ei.value.code == L.LBM_ERR_UNSUPPORTED
    finally:
        tc.lbm_destroy(tctx)


def test_device_pointers_and_streams():
    import torch
    w = W.random_state(50, 20, seed=4)
    s = torch.cuda.Stream()
    lbm, ctx = _ctx(w, "fp64", stream=s)
    try:
        dev = [torch.tensor(a, device="cuda") for a in w.fields()]
        with torch.cuda.stream(s):
            lbm.lbm_set_init(ctx, *dev)
            lbm.lbm_step(ctx, 20)
            outd = [torch.empty((w.ny, w.nx), dtype=torch.float64, device="cuda") for _ in range(4)]
            lbm.lbm_moments(ctx, *outd)
        s.synchronize()
        outh = [np.empty((w.ny, w.nx)) for _ in range(4)]
        lbm.lbm_moments(ctx, *outh)
        for a, b in zip(outd, outh):
            assert np.array_equal(a.cpu().numpy(), b)
        ref, _ = oracle_run(w, 20)
        err = field_errors(dict(zip(("rho", "u", "v", "T"), outh)), ref)
        assert max(err.values()) < 1e-12
    finally:
        lbm.lbm_destroy(ctx)


def test_invalid_and_unsupported_configs_raise():
    from paper_0908_3749_gb300 import lbm
    w = W.random_state(4, 4, seed=1)
    for kw, code in (({"internal_dof": 3}, lbm.LBM_ERR_UNSUPPORTED),
                     ({"precision": "tc_bf16x3"}, lbm.LBM_ERR_UNSUPPORTED)):
        cfg = lbm.make_config(w.nx, w.ny, w.dx, w.dy, w.dt, w.s, w.bc, **kw)
        with pytest.raises(lbm.LBMError) as ei:
            lbm.lbm_create(cfg)
        assert ei.value.code == code


def test_zero_steps_is_a_no_op():
    w = W.random_state(9, 4, seed=2)
    a, fa, _ = gpu_run(w, 0)
    ref, fref = oracle_run(w, 0)
    assert np.abs(fa - fref).max() <= 1e-15 * np.abs(fref).max()


@pytest.mark.slow
def test_couette_paper_case1_velocity_error():
    """Sec. V.D case 1 at the paper's parameters (16 x 32, dx = 0.004,
    dt = 1e-5, all s = 1e5, t = 57.5: 5.75 million steps). The printed
    velocity error is 7.02 %; the GPU run must land within 10 % of it with
    mu = rho T / s_5 in the analytic series, E summed over the vertical line
    of NY + 1 nodes including the two wall nodes (which move at -U, +U)."""
    from oracle import exact
    w = W.couette(NX=16, NY=32, d=0.004, dt=1e-5)
    got, _, status = gpu_run(w, w.nsteps)
    assert status[0] == 0
    y = w.meta["y"]
    u = got["u"][:, 0]
    assert np.abs(got["u"] - got["u"][:, :1]).max() < 1e-12   # uniform in x
    ue = exact.couette_u(y, w.nsteps * w.dt, 0.1, w.meta["D"], 1.0 / 1e5, 1.0)
    E = exact.relative_error(np.r_[-0.1, u, 0.1], np.r_[-0.1, ue, 0.1])
    assert abs(E - 0.0702) < 0.1 * 0.0702, E


def test_moments_into_one_host_array_equal_separate_arrays():
    """lbm_moments with the four fields as consecutive blocks of one host
    array (one device-to-host copy) gives what four separate arrays get."""
    from paper_0908_3749_gb300 import lbm
    w = W.random_state(45, 13, seed=8)
    cfg = lbm.make_config(w.nx, w.ny, w.dx, w.dy, w.dt, w.s, w.bc, "fp64", 0)
    ctx = lbm.lbm_create(cfg)
    try:
        lbm.lbm_set_init(ctx, *w.fields())
        lbm.lbm_step(ctx, 7)
        block = np.empty((4, w.ny, w.nx))
        lbm.lbm_moments(ctx, *block)
        sep = [np.empty((w.ny, w.nx)) for _ in range(4)]
        lbm.lbm_moments(ctx, *sep)
    finally:
        lbm.lbm_destroy(ctx)
    for k in range(4):
        assert np.array_equal(block[k], sep[k])


def test_c_program_on_the_abi(tmp_path):
    """tests/abi_example.c, built with gcc against include/lbm.h and the
    library, runs 200 FP64 steps on a periodic grid and checks conservation
    and the watchdog by itself."""
    import subprocess
    from test_abi import _build_c_example
    exe, env = _build_c_example(tmp_path)
    res = subprocess.run([exe], capture_output=True, text=True, env=env, timeout=120)
    assert res.returncode == 0 and "abi example ok" in res.stdout, (res.returncode, res.stderr)


def test_fma_probe_rates_are_physical_and_repeatable():
    """The roofline denominators: every rate is positive and below the most
    any device could retire (its multiprocessors x 128 FP32 lanes x 2.5 GHz;
    64 FP64 lanes), the paired FP32 form retires the FP32 lane rate (the same
    FP32 units), and a second measurement agrees within 10 %."""
    import torch
    from paper_0908_3749_gb300 import lbm
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    r = {k: lbm.lbm_probe_fma_rate(k, 20.0) for k in ("fp64", "fp32", "fp32x2")}
    assert 0 < r["fp64"] <= sms * 64 * 2.5e9, r
    assert 0 < r["fp32"] <= sms * 128 * 2.5e9, r
    assert abs(r["fp32x2"] / r["fp32"] - 1) < 0.15, r
    again = lbm.lbm_probe_fma_rate("fp64", 20.0)
    assert abs(again / r["fp64"] - 1) < 0.1, (again, r)
