"""Pins of the FP64 reference of the elimination proposal network: the
convolution against scipy's textbook 2-D correlation, GELU's derivative and
the full gradient against central finite differences, and a planted mistake
in the input gradient that the finite-difference check catches."""
import numpy as np
import pytest
from scipy.signal import correlate2d

import oracle.cnn as cnn
import scenegen


def test_conv3x3_is_zero_padded_correlation():
    s = scenegen.Stream(1, 1)
    x = s.normal(2 * 3 * 7 * 9).reshape(2, 3, 7, 9)
    W = s.normal(4 * 3 * 9).reshape(4, 3, 3, 3)
    b = s.normal(4)
    out = cnn.conv3x3(x, W, b)
    for bi in range(2):
        for o in range(4):
            ref = b[o] + sum(correlate2d(x[bi, c], W[o, c], mode="same", boundary="fill") for c in range(3))
            assert np.allclose(out[bi, o], ref, atol=1e-12)


def test_gelu_derivative():
    z = np.linspace(-5, 5, 101)
    h = 1e-6
    fd = (cnn.gelu(z + h) - cnn.gelu(z - h)) / (2 * h)
    assert np.allclose(cnn.gelu_grad(z), fd, atol=1e-8)
    assert np.allclose(cnn.gelu(np.array([0.0, 1e3, -1e3])), [0.0, 1e3, 0.0])


def _problem(seed=3, H=6, W=7, B=2):
    s = scenegen.Stream(seed, 2)
    p = scenegen.cnn_init(seed, scale=0.8).astype(np.float64)
    p[cnn.num_params() - 33:] = s.normal(33) * 0.5       # head not at zero
    x = s.normal(B * 6 * H * W).reshape(B, 6, H, W)
    y = (s.uniform(B * H * W) < 0.3).astype(np.float64).reshape(B, H, W)
    return p, x, y


def _fd_check(mod, idx, h=1e-5):
    p, x, y = _problem()
    loss, g = mod.loss_and_grad(p, x, y, pos_weight=2.5)
    for i in idx:
        pp, pm = p.copy(), p.copy()
        pp[i] += h
        pm[i] -= h
        fd = (mod.loss_and_grad(pp, x, y, 2.5)[0] - mod.loss_and_grad(pm, x, y, 2.5)[0]) / (2 * h)
        if abs(fd - g[i]) > 1e-7 * max(1.0, abs(fd)) + 1e-9:
            return False
    return True


def test_gradient_matches_finite_differences():
    n = cnn.num_params()
    assert n == 38785
    s = scenegen.Stream(5, 3)
    # indices in every block (W1, b1, W3, W5, b5, Wh, bh) plus random ones
    fixed = [0, 1000, 1728, 1740, 1760 + 9248 + 17, n - 1000, n - 40, n - 20, n - 1]
    idx = fixed + list(s.integers(20, n))
    assert _fd_check(cnn, idx)


def test_finite_differences_catch_a_flipped_input_gradient():
    import types
    bad = types.SimpleNamespace(**{k: getattr(cnn, k) for k in dir(cnn) if not k.startswith("__")})

    def wrong_input_grad(dz, W):          # forgets to flip the kernel offsets
        B, O, H, Wd = dz.shape
        dzp = np.pad(dz, ((0, 0), (0, 0), (1, 1), (1, 1)))
        dx = np.zeros((B, W.shape[1], H, Wd))
        for ky in range(3):
            for kx in range(3):
                dx += np.einsum("oc,bohw->bchw", W[:, :, ky, kx], dzp[:, :, ky:ky + H, kx:kx + Wd])
        return dx

    src = cnn.loss_and_grad.__code__
    g = dict(cnn.__dict__)
    g["conv3x3_input_grad"] = wrong_input_grad
    bad.loss_and_grad = types.FunctionType(src, g)
    assert not _fd_check(bad, [0, 5, 100, 1000, 1500])
