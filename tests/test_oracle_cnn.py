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


def _small_operator(H, W, seed):
    """A nonsymmetric sparse operator on an H x W grid (5-point, random coefficients)."""
    import scipy.sparse as sp
    rng = np.random.default_rng(seed)
    m = H * W
    rows, cols, vals = [], [], []
    for i in range(H):
        for j in range(W):
            p = i * W + j
            rows.append(p); cols.append(p); vals.append(4.0 + rng.random())
            for di, dj in ((0, 1), (0, -1), (1, 0), (-1, 0)):
                if 0 <= i + di < H and 0 <= j + dj < W:
                    rows.append(p); cols.append((i + di) * W + j + dj); vals.append(-rng.random())
    return sp.csr_matrix((vals, (rows, cols)), shape=(m, m))


def test_residual_loss_gradients_by_central_differences():
    rng = np.random.default_rng(11)
    ch = (1, 4, 4, 1)
    ws = cnn.init_weights(12, channels=ch)
    A = _small_operator(6, 5, 13)
    x = rng.standard_normal((2, 1, 6, 5))
    r = rng.standard_normal((2, 1, 6, 5))
    L, grads, gx, _ = cnn.residual_loss_and_grads(ws, x, r, A)
    h = 1e-6
    f = lambda ww, xx: cnn.residual_loss_and_grads(ww, xx, r, A)[0]
    for li, idx in [(0, (2, 0, 1, 2)), (1, (1, 3, 0, 1)), (2, (0, 1, 2, 2))]:
        wp = [w.copy() for w in ws]
        wm = [w.copy() for w in ws]
        wp[li][idx] += h
        wm[li][idx] -= h
        fd = (f(wp, x) - f(wm, x)) / (2 * h)
        assert abs(fd - grads[li][idx]) <= 1e-6 * max(1.0, abs(fd))
    xp = x.copy()
    xm = x.copy()
    xp[0, 0, 2, 3] += h
    xm[0, 0, 2, 3] -= h
    fd = (f(ws, xp) - f(ws, xm)) / (2 * h)
    assert abs(fd - gx[0, 0, 2, 3]) <= 1e-6 * max(1.0, abs(fd))


def linear_network(c, channels=(1, 4, 4, 1)):
    """Weights with net(x) = c x exactly: relu(x) - relu(-x) carried by channels 0 and 1."""
    ws = [np.zeros((co, ci, 3, 3)) for ci, co in zip(channels[:-1], channels[1:])]
    ws[0][0, 0, 1, 1] = 1.0
    ws[0][1, 0, 1, 1] = -1.0
    for W in ws[1:-1]:
        W[0, 0, 1, 1] = 1.0
        W[1, 1, 1, 1] = 1.0
    ws[-1][0, 0, 1, 1] = c
    ws[-1][0, 1, 1, 1] = -c
    return ws


def test_linear_network_closed_forms():
    """net(x) = c x and A = a I: the residual loss with r = x is (a (1 + c) - 1)^2, the
    regression loss with e = g r is (c - g)^2 / g^2, and M(w) = (1 + c) D^{-1} w."""
    import scipy.sparse as sp
    c, a, g = 0.75, 0.6, 1.5
    ws = linear_network(c)
    x = np.random.default_rng(14).standard_normal((3, 1, 5, 4))
    y, _ = cnn.forward(ws, x)
    assert np.abs(y - c * x).max() < 1e-14
    A = a * sp.identity(20, format="csr")
    L = cnn.residual_loss_and_grads(ws, x, x.copy(), A)[0]
    assert abs(L - (a * (1 + c) - 1) ** 2) < 1e-13
    Lr = cnn.loss_and_grads(ws, x, g * x)[0]
    assert abs(Lr - (c - g) ** 2 / g ** 2) < 1e-13
    Ah = _small_operator(5, 4, 15)
    dinv = cnn.inverse_diagonal(Ah)
    assert np.allclose(dinv * Ah.diagonal(), 1.0, rtol=0, atol=1e-15)
    w = np.random.default_rng(16).standard_normal(20)
    z = cnn.jacobi_network_preconditioner(ws, w, dinv, 5, 4)
    assert np.abs(z - (1 + c) * dinv * w).max() < 1e-13 * np.abs(z).max()


def test_zero_network_is_jacobi():
    ws = [np.zeros_like(W) for W in cnn.init_weights(0)]
    Ah = _small_operator(4, 6, 17)
    dinv = cnn.inverse_diagonal(Ah)
    w = np.random.default_rng(18).standard_normal(24)
    assert np.array_equal(cnn.jacobi_network_preconditioner(ws, w, dinv, 4, 6), w * dinv)
