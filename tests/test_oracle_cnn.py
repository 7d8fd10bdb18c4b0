"""Pins of the corrector network's CPU reference (oracle/cnn.py).

* conv3x3 equals a sum of scipy 2D cross-correlations with zero fill (a
  library routine), channel by channel;
* every gradient equals central finite differences of the loss;
* restriction of a uniform field returns it; restriction conserves the
  block totals of rho, j, e exactly.
"""
import numpy as np
import pytest

from oracle import cnn


def _params(rng, chans):
    return [(rng.standard_normal((3, 3, a, b)) * 0.2, rng.standard_normal(b) * 0.1)
            for a, b in zip(chans[:-1], chans[1:])]


def test_conv_matches_scipy_correlate():
    signal = pytest.importorskip("scipy.signal")
    rng = np.random.default_rng(0)
    x = rng.standard_normal((7, 9, 3))
    w = rng.standard_normal((3, 3, 3, 2))
    b = rng.standard_normal(2)
    y = cnn.conv3x3(x, w, b)
    for o in range(2):
        ref = b[o] + sum(signal.correlate2d(x[:, :, k], w[:, :, k, o], mode="same",
                                            boundary="fill", fillvalue=0.0) for k in range(3))
        np.testing.assert_allclose(y[:, :, o], ref, rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("loss_kind,scale", [("mse", None), ("l1", None), ("mse", (0.5, 2.0, 1.0, 0.25)),
                                              ("l1", (0.5, 2.0, 1.0, 0.25))])
def test_gradients_match_finite_differences(loss_kind, scale):
    """Backward pass of the squared and absolute losses, with and without a
    per-channel output scale, against central differences (the absolute
    loss is differentiable away from out = target, which random data avoid
    at this step size)."""
    rng = np.random.default_rng(1)
    chans = [4, 5, 5, 4]
    params = _params(rng, chans)
    x = rng.standard_normal((6, 5, 4))
    t = rng.standard_normal((6, 5, 4))
    kw = dict(scale=scale, loss=loss_kind)
    loss, grads = cnn.loss_and_grads(x, t, params, **kw)
    h = 1e-6
    for l, (w, b) in enumerate(params):
        for arr, g in ((w, grads[l][0]), (b, grads[l][1])):
            flat = arr.reshape(-1)
            gflat = g.reshape(-1)
            for idx in rng.choice(flat.size, size=min(6, flat.size), replace=False):
                old = flat[idx]
                flat[idx] = old + h
                lp, _ = cnn.loss_and_grads(x, t, params, **kw)
                flat[idx] = old - h
                lm, _ = cnn.loss_and_grads(x, t, params, **kw)
                flat[idx] = old
                fd = (lp - lm) / (2 * h)
                assert abs(fd - gflat[idx]) <= 1e-6 * max(1.0, abs(fd)), (l, idx, fd, gflat[idx])


def test_restriction():
    rng = np.random.default_rng(2)
    H = W = 8
    rho = np.exp(rng.uniform(-1, 1, (H, W)))
    u, v = rng.uniform(-1, 1, (2, H, W))
    T = np.exp(rng.uniform(-1, 1, (H, W)))
    R, U, V, TT = cnn.restrict(rho, u, v, T, 4)
    e = rho * T + 0.5 * rho * (u * u + v * v)
    E = R * TT + 0.5 * R * (U * U + V * V)
    np.testing.assert_allclose(R.sum() * 16, rho.sum(), rtol=1e-13)
    np.testing.assert_allclose((R * U).sum() * 16, (rho * u).sum(), rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(E.sum() * 16, e.sum(), rtol=1e-12)
    ones = [np.full((H, W), c) for c in (1.3, 0.2, -0.1, 0.7)]
    for a, c in zip(cnn.restrict(*ones, 2), (1.3, 0.2, -0.1, 0.7)):
        np.testing.assert_allclose(a, c, rtol=1e-14)


def test_bf16_rounding():
    one = 1.0
    assert cnn.bf16(one + 2.0 ** -8) == 1.0              # tie -> even (down)
    assert cnn.bf16(one + 3 * 2.0 ** -8) == 1.0 + 2.0 ** -6   # tie -> even (up)
    assert cnn.bf16(one + 2.0 ** -8 + 2.0 ** -12) == 1.0 + 2.0 ** -7
    assert cnn.bf16(-3.0) == -3.0 and cnn.bf16(0.0) == 0.0
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(5)
    x = (rng.standard_normal(1000) * 10.0 ** rng.uniform(-5, 5, 1000)).astype(np.float32)
    ref = torch.tensor(x).to(torch.bfloat16).to(torch.float64).numpy()
    np.testing.assert_array_equal(cnn.bf16(x), ref)


def test_rounded_pipeline_reduces_to_exact_without_rounding():
    rng = np.random.default_rng(3)
    params = _params(rng, [4, 6, 4])
    x = rng.standard_normal((5, 4, 4))
    t = rng.standard_normal((5, 4, 4))
    l1, g1 = cnn.loss_and_grads(x, t, params)
    l2, g2 = cnn.loss_and_grads(x, t, params, store=lambda a: a)
    assert l1 == l2
    l3, g3 = cnn.loss_and_grads(x, t, params, store=cnn.bf16)
    assert abs(l3 - l1) < 1e-2 * l1
