"""Pins of the FP64 convolutional preconditioner oracle (CPU only)."""
import numpy as np

from oracle import cnn


def test_conv_against_hand_stencil():
    """A single-channel kernel with only the centre and right taps is a 2-point stencil."""
    x = np.random.default_rng(0).standard_normal((1, 1, 5, 6))
    W = np.zeros((1, 1, 3, 3))
    W[0, 0, 1, 1] = 2.0
    W[0, 0, 1, 2] = -1.0
    y = cnn.conv3x3(x, W)
    ref = 2 * x.copy()
    ref[..., :-1] -= x[..., 1:]
    assert np.abs(y - ref).max() < 1e-14


def test_gradients_by_central_differences():
    rng = np.random.default_rng(1)
    ch = (1, 4, 4, 1)
    ws = cnn.init_weights(2, channels=ch)
    r = rng.standard_normal((2, 1, 7, 6))
    e = rng.standard_normal((2, 1, 7, 6))
    L, grads, gr = cnn.loss_and_grads(ws, r, e)
    h = 1e-6
    for li, idx in [(0, (1, 0, 0, 2)), (1, (2, 3, 1, 1)), (2, (0, 2, 2, 0))]:
        wp = [w.copy() for w in ws]
        wm = [w.copy() for w in ws]
        wp[li][idx] += h
        wm[li][idx] -= h
        fd = (cnn.loss_and_grads(wp, r, e)[0] - cnn.loss_and_grads(wm, r, e)[0]) / (2 * h)
        assert abs(fd - grads[li][idx]) <= 1e-6 * max(1.0, abs(fd))
    rp = r.copy()
    rm = r.copy()
    rp[1, 0, 3, 2] += h
    rm[1, 0, 3, 2] -= h
    fd = (cnn.loss_and_grads(ws, rp, e)[0] - cnn.loss_and_grads(ws, rm, e)[0]) / (2 * h)
    assert abs(fd - gr[1, 0, 3, 2]) <= 1e-6 * max(1.0, abs(fd))


def test_positive_homogeneity():
    ws = cnn.init_weights(3, channels=(1, 8, 8, 1))
    x = np.random.default_rng(4).standard_normal((1, 1, 9, 9))
    y1, _ = cnn.forward(ws, x)
    y2, _ = cnn.forward(ws, 7.5 * x)
    assert np.abs(y2 - 7.5 * y1).max() < 1e-12 * np.abs(y2).max()
