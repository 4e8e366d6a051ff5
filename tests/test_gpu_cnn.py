"""GPU parity of the convolutional preconditioner and of flexible GMRES.

The network stores BF16 weights, activations and hidden gradients and accumulates in
FP32; the oracle counterpart applies the same BF16 rounding points in FP64
(oracle.cnn.forward_bf16_storage / loss_and_grads_bf16_storage).  Remaining differences
come from the FP32 accumulation, which moves a sum across a BF16 rounding boundary for a
small fraction of the hidden values; each such value then differs by one BF16 unit
(2^-8 relative) and the difference travels through the later layers.  The comparison is
element by element: max |y - y_o| <= TOL_Y max |y_o| over every output pixel and
max |g - g_o| <= TOL_G max |g_o| over every entry of each layer's weight gradient.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import cnn  # noqa: E402
from oracle.gmres import gmres as orc_gmres  # noqa: E402
from synth import convdiff_csr, gaussian_vector, varcoef_fields_2d  # noqa: E402

# A flipped BF16 rounding changes a hidden value by one BF16 unit, 2^-8 of it; measured,
# the largest output and weight-gradient differences stay below 5e-3 of the largest value
# (0.3e-3 .. 4.9e-3 over the cases below), so the bound is 1e-2, about 2.5 BF16 units.
TOL_Y = 1e-2       # outputs: max-abs error over max-abs value
TOL_G = 1e-2       # weight gradients, per layer


def elementwise(a, ref):
    """max |a - ref| / max |ref| (element by element)."""
    return float(np.abs(np.asarray(a, dtype=np.float64) - ref).max() / np.abs(ref).max())


@pytest.fixture(scope="module")
def kc():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_2104_01253_gb300 as kc
    return kc


@pytest.fixture(scope="module")
def ctx(kc):
    return kc.Context(0)


def pack(ws):
    return np.concatenate([w.transpose(0, 2, 3, 1).reshape(-1) for w in ws]).astype(np.float32)


def unpack(flat, template):
    out, off = [], 0
    for w in template:
        co, ci = w.shape[0], w.shape[1]
        n = co * 9 * ci
        out.append(flat[off:off + n].reshape(co, 3, 3, ci).transpose(0, 3, 1, 2).astype(np.float64))
        off += n
    return out


def test_tcgen05_conv_single_tile(kc, ctx):
    """The tcgen05 convolution on one 16 x 8 tile (one MMA group) against the oracle."""
    B, H, W = 1, 16, 8
    ws = cnn.init_weights(21)
    w32 = pack(ws)
    x = np.random.default_rng(22).standard_normal((B, 1, H, W)).astype(np.float32)
    ctx.set_conv_kernel(ctx.CONV_TCGEN05)
    yd = torch.zeros((B, 1, H, W), dtype=torch.float32, device="cuda")
    kc.kc_cnn_forward(ctx, torch.as_tensor(w32, device="cuda"),
                      torch.as_tensor(x, device="cuda"), yd, B, H, W)
    torch.cuda.synchronize()
    assert ctx.read_status() == 0
    yo, _ = cnn.forward_bf16_storage(unpack(w32, ws), x.astype(np.float64))
    y = yd.cpu().numpy().astype(np.float64)
    assert elementwise(y, yo) <= TOL_Y


@pytest.mark.parametrize("conv", [0, 1])
@pytest.mark.parametrize("B,H,W", [(2, 40, 40), (1, 37, 50), (3, 8, 33)])
def test_forward_matches_oracle(kc, ctx, B, H, W, conv):
    ws = cnn.init_weights(3)
    w32 = pack(ws)
    assert w32.size == kc.kc_cnn_param_count()
    x = np.random.default_rng(4).standard_normal((B, 1, H, W)).astype(np.float32)
    wd = torch.as_tensor(w32, device="cuda")
    xd = torch.as_tensor(x, device="cuda")
    yd = torch.zeros_like(xd)
    ctx.set_conv_kernel(conv)
    try:
        kc.kc_cnn_forward(ctx, wd, xd, yd, B, H, W)
    finally:
        ctx.set_conv_kernel(ctx.CONV_TCGEN05)
    y = yd.cpu().numpy().astype(np.float64)
    yo, _ = cnn.forward_bf16_storage(unpack(w32, ws), x.astype(np.float64))
    err = elementwise(y, yo)
    print("forward %s conv %d: %.2e" % ((B, H, W), conv, err))
    assert err <= TOL_Y


@pytest.mark.parametrize("conv", [0, 1])
@pytest.mark.parametrize("B,H,W", [(2, 24, 40), (3, 13, 37)])
def test_gradients_match_oracle(kc, ctx, conv, B, H, W):
    ws = cnn.init_weights(5)
    w32 = pack(ws)
    rng = np.random.default_rng(6)
    x = rng.standard_normal((B, 1, H, W)).astype(np.float32)
    e = rng.standard_normal((B, 1, H, W)).astype(np.float32)
    wd = torch.as_tensor(w32, device="cuda")
    grad = torch.zeros_like(wd)
    yd = torch.zeros((B, 1, H, W), dtype=torch.float32, device="cuda")
    ctx.set_conv_kernel(conv)
    try:
        loss = kc.kc_cnn_train_step(ctx, wd, None, None, 0, 0.0, torch.as_tensor(x, device="cuda"),
                                    torch.as_tensor(e, device="cuda"), B, H, W, yd, grad)
    finally:
        ctx.set_conv_kernel(ctx.CONV_TCGEN05)
    Lo, go, _ = cnn.loss_and_grads_bf16_storage(unpack(w32, ws), x.astype(np.float64),
                                                e.astype(np.float64))
    assert abs(loss - Lo) <= 1e-3 * Lo
    g = unpack(grad.cpu().numpy(), ws)
    for li in range(6):
        rel = elementwise(g[li], go[li])
        print("gradient %s conv %d layer %d: %.2e" % ((B, H, W), conv, li, rel))
        assert rel <= TOL_G, (li, rel)
    # and the BF16-storage gradients are close to the exact FP64 gradients
    _, gx, _ = cnn.loss_and_grads(unpack(w32, ws), x.astype(np.float64), e.astype(np.float64))
    for li in range(6):
        assert np.linalg.norm(g[li] - gx[li]) / np.linalg.norm(gx[li]) <= 0.25


@pytest.mark.parametrize("conv", [1, 0])
@pytest.mark.parametrize("B,H,W", [(1, 256, 256), (1, 64, 1024)])
def test_forward_matches_oracle_at_size(kc, ctx, conv, B, H, W):
    """Whole images of many tiles: 256 x 256 (2048 tcgen05 tiles of 16 x 8, more than the
    persistent CTAs, so each CTA walks several) and a 1024-wide strip (the row length of
    the config-5 grid), every pixel compared."""
    ws = cnn.init_weights(23)
    w32 = pack(ws)
    x = np.random.default_rng(24).standard_normal((B, 1, H, W)).astype(np.float32)
    xd = torch.as_tensor(x, device="cuda")
    yd = torch.zeros_like(xd)
    ctx.set_conv_kernel(conv)
    try:
        kc.kc_cnn_forward(ctx, torch.as_tensor(w32, device="cuda"), xd, yd, B, H, W)
    finally:
        ctx.set_conv_kernel(ctx.CONV_TCGEN05)
    torch.cuda.synchronize()
    assert ctx.read_status() == 0
    yo, _ = cnn.forward_bf16_storage(unpack(w32, ws), x.astype(np.float64))
    err = elementwise(yd.cpu().numpy(), yo)
    print("forward %s conv %d: %.2e" % ((B, H, W), conv, err))
    assert err <= TOL_Y


def test_forward_matches_oracle_on_the_1024_grid(kc, ctx):
    """The config-5 size, 1024 x 1024, through the tcgen05 kernel: the oracle recomputes
    sampled windows.  An output pixel depends only on the 13 x 13 input pixels around it
    (six 3 x 3 layers), so the oracle run on a crop gives the exact full-image values at
    the crop pixels that lie at least 6 pixels inside it (or at an image border, where the
    crop's zero padding is the image's)."""
    H = W = 1024
    ws = cnn.init_weights(25)
    w32 = pack(ws)
    x = np.random.default_rng(26).standard_normal((1, 1, H, W)).astype(np.float32)
    xd = torch.as_tensor(x, device="cuda")
    yd = torch.zeros_like(xd)
    kc.kc_cnn_forward(ctx, torch.as_tensor(w32, device="cuda"), xd, yd, 1, H, W)
    torch.cuda.synchronize()
    assert ctx.read_status() == 0
    y = yd.cpu().numpy()[0, 0].astype(np.float64)
    wo = unpack(w32, ws)
    R = 6
    # windows: two corners, an edge, the middle and one straddling tile boundaries
    for (r0, c0, h, w) in [(0, 0, 40, 40), (984, 984, 40, 40), (0, 500, 30, 64),
                           (496, 504, 48, 40), (251, 123, 37, 29)]:
        lo_r, lo_c = max(r0 - R, 0), max(c0 - R, 0)
        hi_r, hi_c = min(r0 + h + R, H), min(c0 + w + R, W)
        crop = x[:, :, lo_r:hi_r, lo_c:hi_c].astype(np.float64)
        yo, _ = cnn.forward_bf16_storage(wo, crop)
        yo = yo[0, 0, r0 - lo_r:r0 - lo_r + h, c0 - lo_c:c0 - lo_c + w]
        err = elementwise(y[r0:r0 + h, c0:c0 + w], yo)
        print("1024^2 window %s: %.2e" % ((r0, c0, h, w), err))
        assert err <= TOL_Y


@pytest.mark.parametrize("conv", [1, 0])
def test_gradients_match_oracle_at_size(kc, ctx, conv):
    """Weight gradients of the regression loss on a 256 x 256 image, every entry."""
    B, H, W = 1, 256, 256
    ws = cnn.init_weights(27)
    w32 = pack(ws)
    rng = np.random.default_rng(28)
    x = rng.standard_normal((B, 1, H, W)).astype(np.float32)
    e = rng.standard_normal((B, 1, H, W)).astype(np.float32)
    wd = torch.as_tensor(w32, device="cuda")
    grad = torch.zeros_like(wd)
    yd = torch.zeros((B, 1, H, W), dtype=torch.float32, device="cuda")
    ctx.set_conv_kernel(conv)
    try:
        loss = kc.kc_cnn_train_step(ctx, wd, None, None, 0, 0.0,
                                    torch.as_tensor(x, device="cuda"),
                                    torch.as_tensor(e, device="cuda"), B, H, W, yd, grad)
    finally:
        ctx.set_conv_kernel(ctx.CONV_TCGEN05)
    Lo, go, yo = cnn.loss_and_grads_bf16_storage(unpack(w32, ws), x.astype(np.float64),
                                                 e.astype(np.float64))
    assert abs(loss - Lo) <= 1e-3 * Lo
    assert elementwise(yd.cpu().numpy(), yo) <= TOL_Y
    g = unpack(grad.cpu().numpy(), ws)
    for li in range(6):
        rel = elementwise(g[li], go[li])
        print("gradient 256^2 conv %d layer %d: %.2e" % (conv, li, rel))
        assert rel <= TOL_G, (li, rel)


def test_adam_steps_reduce_the_loss(kc, ctx):
    B, H, W = 4, 32, 32
    ws = cnn.init_weights(7)
    wd = torch.as_tensor(pack(ws), device="cuda")
    m = torch.zeros_like(wd)
    v = torch.zeros_like(wd)
    rng = np.random.default_rng(8)
    x = torch.as_tensor(rng.standard_normal((B, 1, H, W)).astype(np.float32), device="cuda")
    e = x.clone() * 0.5                       # learnable target: a scaled identity
    yd = torch.zeros_like(x)
    first = kc.kc_cnn_train_step(ctx, wd, m, v, 1, 1e-3, x, e, B, H, W, yd)
    for t in range(2, 200):
        last = kc.kc_cnn_train_step(ctx, wd, m, v, t, 1e-3, x, e, B, H, W, yd)
    assert last < 0.3 * first


def test_residual_loss_gradients_match_oracle(kc, ctx):
    """kc_cnn_train_step_residual against the oracle's residual loss with the GPU's BF16
    storage rounding, on a variable-coefficient convection-diffusion operator."""
    N, B = 24, 3
    Ah = _varcoef(N, 40)
    A = kc.DeviceCSR(Ah)
    ws = cnn.init_weights(41)
    w32 = pack(ws)
    rng = np.random.default_rng(42)
    x = rng.standard_normal((B, 1, N, N)).astype(np.float32)
    r = rng.standard_normal((B, 1, N, N)).astype(np.float32)
    wd = torch.as_tensor(w32, device="cuda")
    grad = torch.zeros_like(wd)
    yd = torch.zeros((B, 1, N, N), dtype=torch.float32, device="cuda")
    loss = kc.kc_cnn_train_step_residual(ctx, wd, None, None, 0, 0.0, A,
                                         torch.as_tensor(x, device="cuda"),
                                         torch.as_tensor(r, device="cuda"), B, N, N, yd, grad)
    Lo, go, _, yo = cnn.residual_loss_and_grads(unpack(w32, ws), x.astype(np.float64),
                                                r.astype(np.float64), Ah.to_scipy(), bf16=True)
    assert abs(loss - Lo) <= 2e-3 * Lo
    assert elementwise(yd.cpu().numpy(), yo) <= TOL_Y
    g = unpack(grad.cpu().numpy(), ws)
    for li in range(6):
        rel = elementwise(g[li], go[li])
        print("residual-loss gradient layer %d: %.2e" % (li, rel))
        assert rel <= TOL_G, (li, rel)


def test_residual_training_reduces_the_loss(kc, ctx):
    """Adam on the residual loss with A = 2 I and r = x: the network can reach zero loss
    (net(x) = -x / 2), so 200 steps must cut the loss well down."""
    import scipy.sparse as sp
    from synth.operators import CSR
    N, B = 16, 4
    S = (2.0 * sp.identity(N * N, format="csr")).tocsr()
    A = kc.DeviceCSR(CSR(N * N, S.indptr.astype(np.int32), S.indices.astype(np.int32),
                         S.data.astype(np.float64)))
    wd = torch.as_tensor(pack(cnn.init_weights(43)), device="cuda")
    m = torch.zeros_like(wd)
    v = torch.zeros_like(wd)
    x = torch.as_tensor(np.random.default_rng(44).standard_normal((B, 1, N, N))
                        .astype(np.float32), device="cuda")
    yd = torch.zeros_like(x)
    first = kc.kc_cnn_train_step_residual(ctx, wd, m, v, 1, 1e-3, A, x, x, B, N, N, yd)
    for t in range(2, 200):
        last = kc.kc_cnn_train_step_residual(ctx, wd, m, v, t, 1e-3, A, x, x, B, N, N, yd)
    assert last < 0.3 * first


def _varcoef(N, seed):
    kappa, wind = varcoef_fields_2d(N, seed)
    return convdiff_csr(N, 2, wind, kappa=kappa)


def test_fgmres_identity_equals_gmres(kc, ctx):
    Ah = _varcoef(32, 64)
    b = gaussian_vector(Ah.m, 71)
    A = kc.DeviceCSR(Ah)
    bd = torch.as_tensor(b, device="cuda")
    x1 = torch.zeros_like(bd)
    x2 = torch.zeros_like(bd)
    i1 = kc.gmres_solve(ctx, A, bd, x1, restart=40, rtol=1e-10)
    i2 = kc.fgmres_solve(ctx, A, None, 32, 32, bd, x2, restart=40, rtol=1e-10)
    assert i1["status"] == 0 and i2["status"] == 0
    assert abs(i1["iters"] - i2["iters"]) <= 1
    assert i2["rel_resid_true"] <= 1e-10
    xo, io = orc_gmres(Ah.to_scipy(), b, restart=40, rtol=1e-10, precond=lambda w: w.copy())
    assert abs(io["iters"] - i2["iters"]) <= 1
    assert np.linalg.norm(x2.cpu().numpy() - xo) / np.linalg.norm(xo) <= 1e-8


def near_identity_weights(seed, eps=0.02):
    """net(x) = relu(x) - relu(-x) = x through channels 0 and 1, plus small random weights
    everywhere: a nonlinear preconditioner close to the identity."""
    rng = np.random.default_rng(seed)
    ws = [eps * rng.standard_normal(w.shape) / 3.0 for w in cnn.init_weights(0)]
    ws[0][0, 0, 1, 1] += 1.0
    ws[0][1, 0, 1, 1] -= 1.0
    for l in range(1, 5):
        ws[l][0, 0, 1, 1] += 1.0
        ws[l][1, 1, 1, 1] += 1.0
    ws[5][0, 0, 1, 1] += 1.0
    ws[5][0, 1, 1, 1] -= 1.0
    return ws


@pytest.mark.parametrize("N", [2, 33, 100])
def test_residual_sample_matches_oracle(kc, ctx, N):
    """kc_cnn_residual_sample: r = b - A x, u = D^{-1} r (oracle.cnn.inverse_diagonal),
    s = rms(u), inputs u / s and residuals r / s in FP32 (one FP32 rounding each, so
    2^-24 relative per element, plus the FP64 arithmetic's few units in the last place);
    ||r|| to 1e-13; r = 0 gives zeros."""
    Ah = _varcoef(N, 61)
    As = Ah.to_scipy()
    b = gaussian_vector(Ah.m, 71)
    x = gaussian_vector(Ah.m, 72) * 0.1
    A = kc.DeviceCSR(Ah)
    bd = torch.as_tensor(b, device="cuda")
    xd = torch.as_tensor(x, device="cuda")
    xin = torch.empty(Ah.m, dtype=torch.float32, device="cuda")
    res = torch.empty_like(xin)
    rn = kc.kc_cnn_residual_sample(ctx, A, bd, xd, xin, res)
    r = b - As @ x
    u = r * cnn.inverse_diagonal(As)
    s = np.sqrt(np.mean(u * u))
    assert abs(rn - np.linalg.norm(r)) <= 1e-13 * np.linalg.norm(r)
    for got, want in ((xin, u / s), (res, r / s)):
        g = got.cpu().numpy().astype(np.float64)
        assert np.all(np.abs(g - want) <= 2.0 ** -23 * np.abs(want) + 1e-14 * np.abs(want).max())
    # x solves A x = b exactly when b = A x: r = 0, outputs zero
    bd0 = torch.as_tensor(As @ np.zeros(Ah.m), device="cuda")
    x0 = torch.zeros_like(bd0)
    assert kc.kc_cnn_residual_sample(ctx, A, bd0, x0, xin, res) == 0.0
    assert not xin.any() and not res.any()
    assert ctx.read_status() == 0


def test_fgmres_jacobi_matches_oracle(kc, ctx):
    Ah = _varcoef(32, 66)
    b = gaussian_vector(Ah.m, 73)
    A = kc.DeviceCSR(Ah)
    bd = torch.as_tensor(b, device="cuda")
    x = torch.zeros_like(bd)
    info = kc.fgmres_solve(ctx, A, None, 32, 32, bd, x, restart=40, rtol=1e-10,
                           precond=kc.PREC_JACOBI)
    assert info["status"] == 0 and info["rel_resid_true"] <= 1e-10
    dinv = cnn.inverse_diagonal(Ah.to_scipy())
    xo, io = orc_gmres(Ah.to_scipy(), b, restart=40, rtol=1e-10, precond=lambda w: w * dinv)
    assert abs(io["iters"] - info["iters"]) <= 1
    assert np.linalg.norm(x.cpu().numpy() - xo) / np.linalg.norm(xo) <= 1e-8


def test_gmres_solve_jacobi_option(kc, ctx):
    """gmres_solve with precond=PREC_JACOBI is right Jacobi-preconditioned GMRES: the same
    solve as fgmres_solve with the Jacobi step (same iteration count, same x to rounding),
    against the oracle's Jacobi-preconditioned GMRES; with an FP32 inner solve it is an
    invalid argument."""
    Ah = _varcoef(32, 66)
    b = gaussian_vector(Ah.m, 73)
    A = kc.DeviceCSR(Ah)
    bd = torch.as_tensor(b, device="cuda")
    x1, x2 = torch.zeros_like(bd), torch.zeros_like(bd)
    i1 = kc.gmres_solve(ctx, A, bd, x1, restart=40, rtol=1e-10, precond=kc.PREC_JACOBI)
    i2 = kc.fgmres_solve(ctx, A, None, 32, 32, bd, x2, restart=40, rtol=1e-10,
                         precond=kc.PREC_JACOBI)
    assert i1["status"] == 0 and i1["rel_resid_true"] <= 1e-10
    assert i1["iters"] == i2["iters"]
    assert torch.equal(x1, x2)
    dinv = cnn.inverse_diagonal(Ah.to_scipy())
    xo, io = orc_gmres(Ah.to_scipy(), b, restart=40, rtol=1e-10, precond=lambda w: w * dinv)
    assert abs(io["iters"] - i1["iters"]) <= 1
    assert np.linalg.norm(x1.cpu().numpy() - xo) / np.linalg.norm(xo) <= 1e-8
    with pytest.raises(kc.KrylovError):
        kc.gmres_solve(ctx, A, bd, torch.zeros_like(bd), restart=40, precision=1,
                       A32=kc.DeviceCSR(Ah, dtype=torch.float32), precond=kc.PREC_JACOBI)


def test_fgmres_with_network_converges(kc, ctx):
    """A perturbed linear network (net(x) ~ -x / 2) in the Jacobi-scaled preconditioner is
    nonlinear: flexible GMRES must reach 1e-10 with an iteration count close to the
    oracle's FGMRES on the same BF16-storage network."""
    N = 32
    Ah = _varcoef(N, 65)
    b = gaussian_vector(Ah.m, 72)
    ws = near_identity_weights(9)
    ws[5] *= -0.5
    w32 = pack(ws)
    A = kc.DeviceCSR(Ah)
    bd = torch.as_tensor(b, device="cuda")
    x = torch.zeros_like(bd)
    info = kc.fgmres_solve(ctx, A, torch.as_tensor(w32, device="cuda"), N, N, bd, x,
                           restart=40, rtol=1e-10)
    assert info["status"] == 0 and info["rel_resid_true"] <= 1e-10
    wo = unpack(w32, ws)
    dinv = cnn.inverse_diagonal(Ah.to_scipy())
    M = lambda w: cnn.jacobi_network_preconditioner(wo, w, dinv, N, N, bf16=True)
    _, io = orc_gmres(Ah.to_scipy(), b, restart=40, rtol=1e-10, precond=M)
    assert io["rel_resid_true"] <= 1e-10
    assert abs(info["iters"] - io["iters"]) <= max(3, 0.1 * io["iters"])


def test_trained_network_reduces_fgmres_iterations(kc, ctx):
    """Train on the restart residuals of plain GMRES solves on seeded operators 0..11
    (32 x 32 grids) with the residual loss, then solve held-out operators 64..66: the
    learned preconditioner must cut the iteration count of plain GMRES(40) and of the
    Jacobi step alone (the part of M without the network).  The size of the gain is an
    empirical result with no closed form; it is printed."""
    from paper_2104_01253_gb300 import train as tr
    N = 32
    ops, X, R, owner = tr.generate_pairs(ctx, N, range(12), restart=40, max_cycles=20)
    assert X.shape[0] >= 100
    w, hist = tr.train(ctx, ops, X, R, owner, steps=600, batch=16, lr=2e-3, seed=0)
    assert np.mean(hist[-50:]) < 0.8 * np.mean(hist[:20])
    rows = []
    for seed in (64, 65, 66):
        Ah = tr.varcoef_operator(N, seed)
        A = kc.DeviceCSR(Ah)
        b = torch.as_tensor(gaussian_vector(Ah.m, 2000 + seed), device="cuda")
        x1, x2, x3 = (torch.zeros_like(b) for _ in range(3))
        plain = kc.gmres_solve(ctx, A, b, x1, restart=40, rtol=1e-10)
        jac = kc.fgmres_solve(ctx, A, None, N, N, b, x3, restart=40, rtol=1e-10,
                              precond=kc.PREC_JACOBI)
        flex = kc.fgmres_solve(ctx, A, w, N, N, b, x2, restart=40, rtol=1e-10)
        assert plain["status"] == 0 and jac["status"] == 0 and flex["status"] == 0
        assert flex["rel_resid_true"] <= 1e-10
        rows.append((plain["iters"], jac["iters"], flex["iters"]))
    print("held-out iterations (plain, Jacobi, learned):", rows)
    assert all(f < p for p, _, f in rows)
    assert all(f < j for _, j, f in rows)
