"""The largest grids: when 16 x pitch x ny reaches 2^32 population elements the
step switches to 64-bit element offsets. A 16384 x 16448 doubly periodic grid
(4.31e9 elements per population buffer) is initialised on the device from an
analytic smooth state, stepped once in the benchmark's launch forms (FP32 one
block per tile and persistent; FP64 one block per tile), and its moments are
compared at sampled nodes -- the four corners, the last row and column, and
seeded interior nodes, where 32-bit offsets would have wrapped -- with the
oracle's step of the same state on each node's 3 x 3 neighbourhood (periodic
wrap taken explicitly). FP64 also checks the audit of the initial state
against a torch FP64 sum of the analytic conserved fields.

Bars: FP64 1e-12 (one step); FP32 30 u + 3e-6 (the single-step FP32 bound,
u = 2^-24; the FP32 populations start from the FP64 equilibrium rounded to
FP32). Memory: FP64 about 86 GB on the device, FP32 about 43 GB.
"""
import math

import numpy as np
import pytest

import workloads as W
from oracle import scheme

pytestmark = pytest.mark.gpu

NX, NY = 16384, 16448
DX = DY = 1e-3
DT = 1e-5
U32 = 2.0 ** -24
BARS = {"fp64": 1e-12, "fp32": 30 * U32 + 3e-6}


def _state(i, j, lib):
    """Analytic periodic state at node indices (i, j); lib = numpy or torch."""
    t1 = 2 * math.pi * (1024 * i / NX + 517 * j / NY)
    t2 = 2 * math.pi * (333 * i / NX - 1028 * j / NY)
    t3 = 2 * math.pi * (2048 * i / NX + 2056 * j / NY)
    rho = 1.0 + 0.2 * lib.sin(t1)
    u = 0.3 * lib.cos(t2)
    v = 0.2 * lib.sin(t3)
    T = 1.0 + 0.3 * lib.cos(t1 + t2)
    return rho, u, v, T


def _oracle_node(i, j, s):
    """(rho, u, v, T) at node (i, j) after one oracle step."""
    ii = np.array([(i - 1) % NX, i, (i + 1) % NX], dtype=np.float64)[None, :]
    jj = np.array([(j - 1) % NY, j, (j + 1) % NY], dtype=np.float64)[:, None]
    f = scheme.equilibrium_populations(*[np.broadcast_to(q, (3, 3)) for q in _state(ii, jj, np)])
    per = ("periodic", None)
    f1 = scheme.step(f, {"dx": DX, "dy": DY, "dt": DT, "s": s, "bc": (per, per, per, per)})
    return [float(q[1, 1]) for q in scheme.macroscopic(f1)]


def _samples():
    rng = np.random.default_rng(4321)
    pts = [(0, 0), (NX - 1, 0), (0, NY - 1), (NX - 1, NY - 1), (NX // 2, NY - 1),
           (NX - 1, NY // 2), (NX - 2, NY - 2), (31, NY - 1), (NX - 33, 7)]
    pts += [(int(a), int(b)) for a, b in zip(rng.integers(0, NX, 24), rng.integers(0, NY, 24))]
    return pts


@pytest.mark.parametrize("precision,blocks", [("fp32", 0), ("fp32", 456), ("fp64", 0)])
def test_wide_grid_one_step_sampled(precision, blocks):
    import torch
    from paper_0908_3749_gb300 import lbm
    s = np.array(W.BUBBLE_RATES, dtype=np.float64)
    per = ("periodic", None)
    cfg = lbm.make_config(NX, NY, DX, DY, DT, s, (per, per, per, per), precision, 0)
    stream = torch.cuda.current_stream()
    ctx = lbm.lbm_create(cfg, stream)
    try:
        i = torch.arange(NX, dtype=torch.float64, device="cuda")[None, :]
        j = torch.arange(NY, dtype=torch.float64, device="cuda")[:, None]
        fields = [q.expand(NY, NX).contiguous() for q in _state(i, j, torch)]
        lbm.lbm_set_init(ctx, *fields)
        if precision == "fp64":
            rho, u, v, T = fields
            e = rho * T + 0.5 * rho * (u * u + v * v)
            want = [float(q.sum()) * DX * DY for q in (rho, rho * u, rho * v, e)]
            got = lbm.lbm_audit(ctx)
            for g, w_ in zip(got, want):
                assert abs(g - w_) <= 1e-12 * max(abs(w_), 1.0), (got, want)
            del rho, u, v, T, e
        del fields
        torch.cuda.empty_cache()
        if blocks:
            lbm.lbm_set_step_blocks(ctx, blocks)
        lbm.lbm_step(ctx, 1)
        out = [torch.empty((NY, NX), dtype=torch.float64, device="cuda") for _ in range(4)]
        lbm.lbm_moments(ctx, *out)
        rc, bad, _ = lbm.lbm_status(ctx)
        assert rc == lbm.LBM_OK and bad == -1
        pts = _samples()
        ii = torch.tensor([p[0] for p in pts], device="cuda")
        jj = torch.tensor([p[1] for p in pts], device="cuda")
        got = np.stack([o[jj, ii].cpu().numpy() for o in out], 1)
        del out
    finally:
        lbm.lbm_destroy(ctx)
        torch.cuda.empty_cache()
    ref = np.array([_oracle_node(a, b, s) for a, b in pts])
    scale = [np.abs(ref[:, 0]).max(), np.hypot(ref[:, 1], ref[:, 2]).max(),
             np.hypot(ref[:, 1], ref[:, 2]).max(), np.abs(ref[:, 3]).max()]
    err = max(float(np.abs(got[:, q] - ref[:, q]).max() / scale[q]) for q in range(4))
    print("%dx%d %s blocks %d: worst sampled field error %.3g" % (NX, NY, precision, blocks, err))
    assert err <= BARS[precision]
