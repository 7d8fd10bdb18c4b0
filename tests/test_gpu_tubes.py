"""GPU tests of the batched quasi-1D tubes (include/lbm_batch.h): parity of
every tube with the FP64 oracle run on the same tube as a one-node-deep 2D
grid, tiling invariance, graph batches, per-tube watchdog and audit, the
bounded grid barrier's timeout path, and the autotuner."""
import math
import os
import time

import numpy as np
import pytest

import workloads as W
from harness import field_errors, oracle_run

pytestmark = pytest.mark.gpu

U32 = 2.0 ** -24


def fp32_bound(n):
    return 30 * U32 * math.sqrt(max(n, 1)) + 3e-6


def _batch(nx, seed=0, rates=None, dt=1e-5):
    rng = np.random.default_rng(seed)
    nt = len(nx)
    nx = np.asarray(nx, dtype=np.int64)
    dx = 1.0 / np.maximum(nx, 200)          # keep 6 dt / dx <= 1
    lo, hi = math.log(0.5), math.log(2.0)
    left = np.stack([np.exp(rng.uniform(lo, hi, nt)), rng.uniform(-0.5, 0.5, nt), np.zeros(nt),
                     np.exp(rng.uniform(lo, hi, nt))], 1)
    right = np.stack([np.exp(rng.uniform(lo, hi, nt)), rng.uniform(-0.5, 0.5, nt), np.zeros(nt),
                      np.exp(rng.uniform(lo, hi, nt))], 1)
    if rates is None:
        s = np.full((nt, 16), 1e5)
        scale = 0.005 / dx
        for k, base in ((5, 200.0), (6, 200.0), (7, 400.0), (8, 400.0), (11, 1000.0)):
            s[:, k - 1] = np.minimum(base * scale, 1e5)
    else:
        s = np.asarray(rates, dtype=np.float64)
    return {"nx": nx, "dx": dx, "dt": dt, "s": s, "left": left, "right": right}


def _fields(B):
    return W.tube_fields(B)


def _tube_workload(B, t):
    n = int(B["nx"][t])
    x = (np.arange(n) + 0.5) / n
    m = (x <= 0.5)[None, :]
    f = [np.where(m, B["left"][t, q], B["right"][t, q]) for q in range(4)]
    bc = (("eq", tuple(B["left"][t])), ("eq", tuple(B["right"][t])), ("periodic", None), ("periodic", None))
    return W.Workload("tube%d" % t, n, 1, B["dx"][t], B["dx"][t], B["dt"], tuple(B["s"][t]), bc, *f)


def _run(B, nsteps, tiling=None, chunks=None):
    from paper_0908_3749_gb300 import lbm
    b = lbm.lbm_batch_create(B["nx"], B["dx"], B["dt"], B["s"], B["left"], B["right"])
    try:
        if tiling:
            lbm.lbm_batch_set_tiling(b, *tiling)
        lbm.lbm_batch_set_init(b, *_fields(B))
        for n in (chunks or [nsteps]):
            lbm.lbm_batch_step(b, n)
        tot = lbm.lbm_batch_total_nodes(b)
        out = [np.empty(tot) for _ in range(4)]
        lbm.lbm_batch_moments(b, *out)
        status = lbm.lbm_batch_status(b, len(B["nx"]))
        audit = lbm.lbm_batch_audit(b, len(B["nx"]))
        steps = lbm.lbm_batch_step_count(b)
    finally:
        lbm.lbm_batch_destroy(b)
    return out, status, audit, steps


def _split(B, arr):
    offs = np.concatenate([[0], np.cumsum(B["nx"])])
    return [arr[offs[t]:offs[t + 1]] for t in range(len(B["nx"]))]


NX = [2, 3, 31, 32, 33, 64, 127, 129, 200, 257, 300, 513]


def test_every_tube_matches_oracle():
    B = _batch(NX, seed=1)
    n = 30
    out, (rc, bad, nbad, to), audit, steps = _run(B, n)
    assert rc == 0 and nbad == 0 and to == 0 and steps == n
    parts = [_split(B, a) for a in out]
    for t in range(len(NX)):
        w = _tube_workload(B, t)
        ref, fref = oracle_run(w, n)
        got = {k: parts[q][t][None, :] for q, k in enumerate(("rho", "u", "v", "T"))}
        err = field_errors(got, ref)
        assert max(err.values()) <= fp32_bound(n), (t, NX[t], err)
        from oracle import scheme
        tot = scheme.conserved_totals(fref, w.dx, 1.0)
        np.testing.assert_allclose(audit[t], tot, rtol=2e-6, atol=2e-6 * np.abs(tot).max())


@pytest.mark.parametrize("tiling", [(128, 64), (512, 128), (1024, 512), (1024, 128)])
def test_tiling_does_not_change_results(tiling):
    B = _batch(NX, seed=2)
    a = _run(B, 25, tiling=(256, 128))[0]
    b = _run(B, 25, tiling=tiling)[0]
    for x, y in zip(a, b):
        assert np.array_equal(x, y)


def test_graph_batches_equal_single_steps():
    B = _batch(NX, seed=3)
    a, _, _, sa = _run(B, 12)
    b, _, _, sb = _run(B, 12, chunks=[1] * 12)
    c, _, _, sc = _run(B, 12, chunks=[5, 7])
    assert sa == sb == sc == 12
    for x, y, z in zip(a, b, c):
        assert np.array_equal(x, y) and np.array_equal(x, z)


def test_unstable_tube_is_flagged_alone():
    nx = [200, 150, 256]
    B = _batch(nx, seed=4)
    B["s"][0, :] = 1e5                        # all rates 1e5 on the 200-node Sod tube
    B["dx"][0] = 0.005
    B["left"][0] = W.SOD_L
    B["right"][0] = W.SOD_R
    from oracle import scheme
    w = _tube_workload(B, 0)
    _, bad_ref = scheme.run(scheme.init_populations(*w.fields()), w.cfg(), 1500, check_every=1)
    _, (rc, bad, nbad, to), _, _ = _run(B, 1500)
    assert rc == 0 and to == 0 and nbad == 1
    assert bad_ref is not None and abs(bad[0] - bad_ref) <= 5, (bad[0], bad_ref)
    assert bad[1] == -1 and bad[2] == -1


def test_barrier_timeout_is_reported_not_hung():
    from paper_0908_3749_gb300 import lbm
    B = _batch([300] * 40, seed=5)
    b = lbm.lbm_batch_create(B["nx"], B["dx"], B["dt"], B["s"], B["left"], B["right"])
    try:
        lbm.lbm_batch_set_init(b, *_fields(B))
        _, _, blocks = lbm.lbm_batch_get_tiling(b)
        assert blocks >= 2
        lbm.lbm_batch_debug_skip_arrival(b, blocks - 1, 2)
        t0 = time.time()
        lbm.lbm_batch_step(b, 5)
        rc, _, _, to = lbm.lbm_batch_status(b, 40)
        assert rc == lbm.LBM_ERR_TIMEOUT and to == 1
        assert time.time() - t0 < 30
        # a fresh initial state clears the barrier and the batch runs again
        lbm.lbm_batch_set_init(b, *_fields(B))
        lbm.lbm_batch_step(b, 3)
        rc, _, nbad, to = lbm.lbm_batch_status(b, 40)
        assert rc == 0 and to == 0 and lbm.lbm_batch_step_count(b) == 3
    finally:
        lbm.lbm_batch_destroy(b)


def test_autotuner_picks_a_candidate_and_caches_it(tmp_path):
    from paper_0908_3749_gb300 import lbm
    B = _batch([700] * 64, seed=6)
    cache = str(tmp_path / "tune.json")
    b = lbm.lbm_batch_create(B["nx"], B["dx"], B["dt"], B["s"], B["left"], B["right"])
    try:
        lbm.lbm_batch_set_init(b, *_fields(B))
        before = [np.empty(lbm.lbm_batch_total_nodes(b)) for _ in range(4)]
        lbm.lbm_batch_moments(b, *before)
        chosen = lbm.lbm_batch_autotune(b, 5, cache)
        assert chosen == lbm.lbm_batch_get_tiling(b)[:2]
        assert os.path.exists(cache) and str(chosen[0]) in open(cache).read()
        after = [np.empty_like(before[0]) for _ in range(4)]
        lbm.lbm_batch_moments(b, *after)
        for x, y in zip(before, after):       # state restored after the trials
            assert np.array_equal(x, y)
        assert lbm.lbm_batch_step_count(b) == 0
        t0 = time.time()
        assert lbm.lbm_batch_autotune(b, 5, cache) == chosen   # from the cache
    finally:
        lbm.lbm_batch_destroy(b)
