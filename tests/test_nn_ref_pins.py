"""Pins of the FP64 reference of the surrogate network (oracle/nn_ref.py):
the convolution against scipy's N-d correlation, the gradients against
central finite differences, and the bfloat16 rounding against exact
representable values."""
import numpy as np
import pytest

from oracle import nn_ref

scipy_signal = pytest.importorskip("scipy.signal")


def test_conv3d_matches_library_correlation():
    rng = np.random.default_rng(0)
    x = rng.normal(size=(5, 4, 6, 3))
    W = rng.normal(size=(27, 2, 3))
    b = rng.normal(size=2)
    y = nn_ref.conv3d(x, W, b)
    for o in range(2):
        ref = np.full(x.shape[:3], b[o])
        for i in range(3):
            k = W[:, o, i].reshape(3, 3, 3)
            ref += scipy_signal.correlate(x[..., i], k, mode="same", method="direct")
        np.testing.assert_allclose(y[..., o], ref, rtol=1e-12, atol=1e-12)


def test_gradients_match_finite_differences():
    rng = np.random.default_rng(1)
    chans = [3, 4, 2]
    params = [(0.3 * rng.normal(size=(27, chans[l + 1], chans[l])), 0.1 * rng.normal(size=chans[l + 1]))
              for l in range(2)]
    x = rng.normal(size=(3, 4, 3, 3))
    target = rng.normal(size=(3, 4, 3, 2))
    mask = rng.uniform(size=(3, 4, 3)) > 0.3

    def loss_of(ps):
        return nn_ref.mse(nn_ref.forward(x, ps)[-1], target, mask)[0]

    acts = nn_ref.forward(x, params)
    _, dy = nn_ref.mse(acts[-1], target, mask)
    grads = nn_ref.backward(acts, params, dy)
    h = 1e-6
    for l in range(2):
        for which in (0, 1):
            arr = params[l][which]
            flat = arr.reshape(-1)
            for idx in rng.choice(flat.size, size=min(12, flat.size), replace=False):
                old = flat[idx]
                flat[idx] = old + h
                lp = loss_of(params)
                flat[idx] = old - h
                lm = loss_of(params)
                flat[idx] = old
                fd = (lp - lm) / (2 * h)
                np.testing.assert_allclose(grads[l][which].reshape(-1)[idx], fd, rtol=1e-5, atol=1e-9)


def test_bf16_rounding():
    # bfloat16 keeps 7 explicit mantissa bits: 1 + 2^-7 is the next value after 1
    v = np.array([1.0, 1.0 + 2 ** -7, 1.0 + 2 ** -8, 1.0 + 3 * 2 ** -8, -2.5, 3.140625])
    r = nn_ref.round_bf16(v)
    # 1 + 2^-8 is a tie -> even (1); 1 + 3*2^-8 is a tie -> even (1 + 2^-6)
    np.testing.assert_array_equal(r, [1.0, 1.0 + 2 ** -7, 1.0, 1.0 + 2 ** -6, -2.5, 3.140625])
