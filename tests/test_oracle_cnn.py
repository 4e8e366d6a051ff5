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


# ---- the BF16-storage variants (what the GPU kernels are compared against) ----------------

from fractions import Fraction  # noqa: E402


def _bf16_rational(q):
    """Round an exact rational to the nearest bfloat16 value (8 significant bits, ties to
    even): written on rationals, independently of the bit-level rounding of the oracle."""
    q = Fraction(q)
    if q == 0:
        return Fraction(0)
    a = abs(q)
    e = 0
    while Fraction(2) ** e > a:
        e -= 1
    while Fraction(2) ** (e + 1) <= a:
        e += 1
    ulp = Fraction(2) ** (e - 7)
    t = a / ulp
    n = t.numerator // t.denominator
    rem = t - n
    if rem > Fraction(1, 2) or (rem == Fraction(1, 2) and n % 2 == 1):
        n += 1
    return (1 if q > 0 else -1) * n * ulp


def _chain_weights(ws_center, seed):
    """Three 1 -> 1 channel layers with the given centre taps; the off-centre taps are
    random, and on a 1 x 1 image they only ever multiply the zero padding."""
    rng = np.random.default_rng(seed)
    ws = []
    for c in ws_center:
        W = rng.standard_normal((1, 1, 3, 3))
        W[0, 0, 1, 1] = float(c)
        ws.append(W)
    return ws


# centre taps, input and target chosen so that every BF16 rounding point changes its value
_W = (1 + Fraction(3, 2 ** 9), Fraction(213, 128) + Fraction(1, 2 ** 10),
      1 + Fraction(1, 2 ** 7) + Fraction(1, 2 ** 12))
_X, _E = 1 + Fraction(1, 2 ** 8), Fraction(4)


def _chain_expected():
    """The 1 x 1-image network in closed form on rationals, with the storage roundings of
    the GPU: BF16 weights, BF16 hidden activations (after the ReLU), BF16 hidden-layer
    gradients dL/dz; input, output and output gradient unrounded."""
    bf = _bf16_rational
    wb = [bf(w) for w in _W]
    z1 = wb[0] * _X
    h1 = bf(max(z1, 0))
    z2 = wb[1] * h1
    h2 = bf(max(z2, 0))
    y = wb[2] * h2
    gy = 2 * (y - _E) / (_E * _E)                  # B = 1: dL/dy of (y - e)^2 / e^2
    gz2 = bf(gy * wb[2] * (1 if z2 > 0 else 0))
    gz1 = bf(gz2 * wb[1] * (1 if z1 > 0 else 0))
    out = dict(y=y, L=(y - _E) ** 2 / (_E * _E), gy=gy, dW=[gz1 * _X, gz2 * h1, gy * h2],
               dx=gz1 * wb[0], h=(h1, h2))
    # every rounding point of this case matters: leaving one out changes the result
    assert all(bf(w) != w for w in _W)
    assert bf(z1) != z1 and bf(z2) != z2 and bf(y) != y and bf(gy) != gy
    assert bf(gy * wb[2]) != gy * wb[2] and bf(gz2 * wb[1]) != gz2 * wb[1]
    return out


def test_bf16_storage_forward_closed_form():
    ex = _chain_expected()
    ws = _chain_weights(_W, 30)
    x = np.full((1, 1, 1, 1), float(_X))
    y, acts = cnn.forward_bf16_storage(ws, x)
    assert y[0, 0, 0, 0] == float(ex["y"])
    assert acts[1][0, 0, 0, 0] == float(ex["h"][0]) and acts[2][0, 0, 0, 0] == float(ex["h"][1])
    assert acts[0][0, 0, 0, 0] == float(_X)                 # the input is not rounded
    # the FP64 network (no rounding) gives a different output on this case
    assert cnn.forward(ws, x)[0][0, 0, 0, 0] != float(ex["y"])
    # a negative input: the ReLU after layer 1 zeroes the output
    assert cnn.forward_bf16_storage(ws, -x)[0][0, 0, 0, 0] == 0.0


def test_bf16_storage_gradients_closed_form():
    ex = _chain_expected()
    ws = _chain_weights(_W, 31)
    x = np.full((1, 1, 1, 1), float(_X))
    e = np.full((1, 1, 1, 1), float(_E))
    L, grads, y = cnn.loss_and_grads_bf16_storage(ws, x, e)
    assert L == float(ex["L"]) and y[0, 0, 0, 0] == float(ex["y"])
    for li in range(3):
        assert grads[li][0, 0, 1, 1] == float(ex["dW"][li]), li
        off = grads[li].copy()
        off[0, 0, 1, 1] = 0.0
        assert not off.any()                 # off-centre taps only see the zero padding
    # backward() with bf16=True: the same weight gradients and dL/dx = w1 dL/dz1
    _, acts = cnn.forward_bf16_storage(ws, x)
    g2, gx = cnn.backward(ws, acts, np.full((1, 1, 1, 1), float(ex["gy"])), bf16=True)
    assert [g[0, 0, 1, 1] for g in g2] == [float(v) for v in ex["dW"]]
    assert gx[0, 0, 0, 0] == float(ex["dx"])
    # without the BF16 hidden-gradient rounding the layer-1 and layer-2 gradients differ
    g64, _ = cnn.backward(ws, acts, np.full((1, 1, 1, 1), float(ex["gy"])), bf16=False)
    assert g64[0][0, 0, 1, 1] != float(ex["dW"][0]) and g64[1][0, 0, 1, 1] != float(ex["dW"][1])


def _dyadic_case(seed, ch=(1, 3, 3, 1), H=4, W=5):
    """Weights in {0, +-1/2, +-1} and inputs in {0, +-1/2, +-1}: every activation and
    gradient below is a dyadic rational with few bits, so BF16 storage rounds nothing."""
    rng = np.random.default_rng(seed)
    ws = []
    for ci, co in zip(ch[:-1], ch[1:]):
        W_ = rng.choice([-1.0, -0.5, 0.5, 1.0], size=(co, ci, 3, 3))
        W_ *= rng.random((co, ci, 3, 3)) < 0.35
        ws.append(W_)
    x = rng.choice([-1.0, -0.5, 0.0, 0.5, 1.0], size=(1, 1, H, W))
    return ws, x


def _all_bf16(a):
    return np.array_equal(cnn._round_bf16(a), a)


def _hidden_grads_bf16(ws, acts, gy):
    """True when every hidden-layer gradient dL/dz of the FP64 backward pass from dL/dy =
    gy is a BF16 value (the premise of the bit-for-bit comparison)."""
    g = gy
    ok = True
    for li in range(len(ws) - 1, -1, -1):
        if li < len(ws) - 1:
            g = g * (acts[li + 1] > 0.0)
            ok = ok and _all_bf16(g) and g.any()
        _, g = cnn.conv3x3_backward(acts[li], ws[li], g)
    return ok


def test_bf16_storage_equals_fp64_when_nothing_rounds():
    """With exactly representable values the BF16-storage forward, loss gradients, backward
    and residual-loss gradients equal the FP64 ones bit for bit (the premise is checked on
    every intermediate), so their structure matches the finite-difference-pinned FP64
    functions."""
    import scipy.sparse as sp
    ws, x = _dyadic_case(47)
    y64, acts64 = cnn.forward(ws, x)
    assert all(_all_bf16(a) for a in acts64[1:-1]) and any(a.any() for a in acts64[1:-1])
    yb, actsb = cnn.forward_bf16_storage(ws, x)
    assert np.array_equal(yb, y64) and all(np.array_equal(a, b) for a, b in zip(acts64, actsb))
    e = np.zeros_like(x)
    e[0, 0, 0, 0], e[0, 0, 1, 3], e[0, 0, 3, 2], e[0, 0, 2, 4] = 1.0, -1.0, 1.0, 1.0  # ||e||^2 = 4
    assert _hidden_grads_bf16(ws, acts64, (y64 - e) / 2.0)
    L64, g64, _ = cnn.loss_and_grads(ws, x, e)
    Lb, gb, _ = cnn.loss_and_grads_bf16_storage(ws, x, e)
    assert Lb == L64 and all(np.array_equal(a, b) for a, b in zip(g64, gb))
    gy = (y64 - e) / 2.0
    G64, X64 = cnn.backward(ws, acts64, gy)
    Gb, Xb = cnn.backward(ws, actsb, gy, bf16=True)
    assert all(np.array_equal(a, b) for a, b in zip(G64, Gb)) and np.array_equal(X64, Xb)
    A = 2.0 * sp.identity(x.size, format="csr")
    assert _hidden_grads_bf16(ws, acts64, 2.0 * (x + y64) - e)   # dL/dy, A = 2 I, ||r||^2 = 4
    R64 = cnn.residual_loss_and_grads(ws, x, e, A)
    Rb = cnn.residual_loss_and_grads(ws, x, e, A, bf16=True)
    assert R64[0] == Rb[0] and all(np.array_equal(a, b) for a, b in zip(R64[1], Rb[1]))
    assert np.array_equal(R64[2], Rb[2]) and np.array_equal(R64[3], Rb[3])
