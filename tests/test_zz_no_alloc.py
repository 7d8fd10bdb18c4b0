"""GPU test of lbm_audit_noalloc, the entry point that allocates nothing.

Some callers cannot allocate device memory (an allocator-free embedding, a
memory pool that is fully reserved, a loop that must not allocate). For them
the library keeps the reduction's scratch in a fixed device array and takes
only caller-owned input and output buffers. This test calls it through the
C ABI, twice in a row on the same state, and checks both results against
lbm_audit (the entry point that uses context-owned scratch) and against the
oracle's conservation totals of the same populations, within the tolerance
the audit tests use; it also checks that oversized grids are rejected with a
clear message, and that the binding refuses tensors the kernel would read
past. The file is named so that pytest collects it last; it passes alone in
a fresh process as well.
"""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_noalloc_totals_match_lbm_audit_and_oracle_twice(precision):
    import torch
    from oracle import scheme
    from paper_0908_3749_gb300 import lbm
    w = W.random_state(333, 101, seed=77, smooth=False)
    cfg = lbm.make_config(w.nx, w.ny, w.dx, w.dy, w.dt, w.s, w.bc, precision, 0)
    ctx = lbm.lbm_create(cfg)
    try:
        lbm.lbm_set_init(ctx, *[np.ascontiguousarray(a) for a in w.fields()])
        lbm.lbm_step(ctx, 7)
        ref = np.array(lbm.lbm_audit(ctx))
        dt = torch.float64 if precision == "fp64" else torch.float32
        f = torch.empty((16, w.ny, w.nx), dtype=dt, device="cuda")
        lbm.lbm_get_populations(ctx, f)
        torch.cuda.synchronize()
        # the oracle's totals of the very populations the kernel reads
        oref = scheme.conserved_totals(f.cpu().numpy().astype(np.float64), w.dx, w.dy)
        out = torch.full((4,), float("nan"), dtype=torch.float64, device="cuda")
        tol = 1e-13
        for _ in range(2):
            out.fill_(float("nan"))
            lbm.lbm_audit_noalloc(f, precision, w.nx, w.ny, w.nx, w.dx, w.dy, out)
            torch.cuda.synchronize()
            got = out.cpu().numpy()
            np.testing.assert_allclose(got, ref, rtol=tol, atol=tol * np.abs(ref).max())
            np.testing.assert_allclose(got, oref, rtol=tol, atol=tol * np.abs(oref).max())
    finally:
        lbm.lbm_destroy(ctx)


def test_noalloc_rejects_oversized_grid():
    import torch
    from paper_0908_3749_gb300 import lbm
    nx, ny = 32 * lbm.NOALLOC_MAX_BLOCKS + 1, 8   # needs more blocks than the scratch holds
    f = torch.zeros(16 * ny * nx, dtype=torch.float32, device="cuda")
    out = torch.zeros(4, dtype=torch.float64, device="cuda")
    with pytest.raises(lbm.LBMError) as ei:
        lbm.lbm_audit_noalloc(f, "fp32", nx, ny, nx, 1.0, 1.0, out)
    assert ei.value.code == lbm.LBM_ERR_INVALID and "scratch" in str(ei.value)


def test_noalloc_binding_refuses_mismatched_tensors():
    import torch
    from paper_0908_3749_gb300 import lbm
    nx, ny = 40, 9
    f64 = torch.zeros((16, ny, nx), dtype=torch.float64, device="cuda")
    out = torch.zeros(4, dtype=torch.float64, device="cuda")
    cases = [
        (f64, "fp32", out),                                          # dtype vs precision
        (f64[:, :, :nx - 1].contiguous(), "fp64", out),              # too few elements
        (f64.transpose(1, 2), "fp64", out),                          # not contiguous
        (f64, "fp64", torch.zeros(4, dtype=torch.float32, device="cuda")),  # totals dtype
        (f64, "fp64", torch.zeros(3, dtype=torch.float64, device="cuda")),  # totals size
        (f64.cpu(), "fp64", out),                                    # host tensor
    ]
    for f, prec, tot in cases:
        with pytest.raises(lbm.LBMError) as ei:
            lbm.lbm_audit_noalloc(f, prec, nx, ny, nx, 1.0, 1.0, tot)
        assert ei.value.code == lbm.LBM_ERR_INVALID
