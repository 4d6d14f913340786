"""Pins of the learned initialiser's FP64 oracle (oracle/unet.py) to facts
other than itself: brute-force loops and a library correlation for the
convolution, adjoint identities for every linear map and its backward,
central finite differences of the loss for the whole backward pass, the
closed form of the cross entropy, and a library bfloat16 conversion."""
import numpy as np
import pytest

from oracle import unet as N


def _brute_conv(X, W, b):
    C, nx, ny, nz = X.shape
    co_n, _, k = W.shape[:3]
    r = k // 2
    Y = np.zeros((co_n, nx, ny, nz))
    for o in range(co_n):
        for i in range(nx):
            for j in range(ny):
                for l in range(nz):
                    s = b[o]
                    for c in range(C):
                        for a in range(k):
                            for bb in range(k):
                                for d in range(k):
                                    ii, jj, ll = i + a - r, j + bb - r, l + d - r
                                    if 0 <= ii < nx and 0 <= jj < ny and 0 <= ll < nz:
                                        s += W[o, c, a, bb, d] * X[c, ii, jj, ll]
                    Y[o, i, j, l] = s
    return Y


def test_conv_matches_brute_force_loops():
    rng = np.random.default_rng(0)
    X = rng.normal(size=(2, 4, 3, 5))
    W = rng.normal(size=(3, 2, 3, 3, 3))
    b = rng.normal(size=3)
    assert np.allclose(N.conv(X, W, b), _brute_conv(X, W, b), rtol=1e-12, atol=1e-12)
    W1 = rng.normal(size=(2, 2, 1, 1, 1))
    assert np.allclose(N.conv(X, W1, b[:2]), _brute_conv(X, W1, b[:2]), rtol=1e-12, atol=1e-12)


def test_conv_matches_scipy_correlate():
    ndimage = pytest.importorskip("scipy.ndimage")
    rng = np.random.default_rng(1)
    X = rng.normal(size=(3, 8, 6, 7))
    W = rng.normal(size=(2, 3, 3, 3, 3))
    b = np.zeros(2)
    ref = np.zeros((2, 8, 6, 7))
    for o in range(2):
        for c in range(3):
            ref[o] += ndimage.correlate(X[c], W[o, c], mode="constant", cval=0.0)
    assert np.allclose(N.conv(X, W, b), ref, rtol=1e-12, atol=1e-12)


def test_adjoint_identities():
    """<L x, y> = <x, L^T y> for conv (input and weight parts), pool and up."""
    rng = np.random.default_rng(2)
    X = rng.normal(size=(3, 8, 8, 8))
    W = rng.normal(size=(4, 3, 3, 3, 3))
    Y = rng.normal(size=(4, 8, 8, 8))
    dX, dW, db = N.conv_backward(X, W, Y)
    lhs = np.sum(N.conv(X, W, np.zeros(4)) * Y)
    assert np.isclose(lhs, np.sum(X * dX), rtol=1e-12)
    assert np.isclose(lhs, np.sum(W * dW), rtol=1e-12)
    assert np.allclose(db, Y.sum(axis=(1, 2, 3)))
    P = rng.normal(size=(3, 4, 4, 4))
    assert np.isclose(np.sum(N.pool(X) * P), np.sum(X * N.pool_backward(P)), rtol=1e-12)
    assert np.isclose(np.sum(N.up(P) * X), np.sum(P * N.up_backward(X)), rtol=1e-12)
    # pool of a constant field is the constant; up then pool is the identity
    assert np.allclose(N.pool(np.full((1, 4, 4, 4), 2.5)), 2.5)
    assert np.allclose(N.pool(N.up(P)), P)


def test_cross_entropy_closed_form():
    z = np.zeros((2, 2, 2))
    y = np.ones((2, 2, 2))
    loss, dz = N.bce_with_logits(z, y)
    assert loss == pytest.approx(np.log(2.0), rel=1e-15)
    assert np.allclose(dz, -0.5 / 8)
    # confident and right: tiny loss; confident and wrong: about |z|
    assert N.bce_with_logits(np.full(4, 30.0), np.ones(4))[0] < 1e-12
    assert N.bce_with_logits(np.full(4, 30.0), np.zeros(4))[0] == pytest.approx(30.0, rel=1e-12)
    rng = np.random.default_rng(3)
    z = rng.normal(size=10)
    y = (rng.random(10) > 0.5).astype(float)
    _, dz = N.bce_with_logits(z, y)
    h = 1e-6
    for i in range(10):
        zp, zm = z.copy(), z.copy()
        zp[i] += h
        zm[i] -= h
        fd = (N.bce_with_logits(zp, y)[0] - N.bce_with_logits(zm, y)[0]) / (2 * h)
        assert dz[i] == pytest.approx(fd, rel=1e-6, abs=1e-10)


def test_bf16_rounding_matches_torch():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(4)
    x = np.concatenate([rng.normal(size=1000) * 10.0 ** rng.integers(-5, 5, 1000),
                        [1.0, 1.0 + 2 ** -8, 1.0 + 3 * 2 ** -9, -2.0 - 2 ** -7, 0.0]])
    ref = torch.from_numpy(x.astype(np.float32)).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(N.bf16_round(x), ref)
    assert N.bf16_round([1.0 + 2 ** -8])[0] == 1.0          # tie to even
    assert N.bf16_round([1.0 + 3 * 2 ** -9])[0] == 1.0 + 2 ** -7


def test_parameter_layout():
    F = 3
    shapes = N.layer_shapes(F)
    assert [s[0] for s in shapes] == ["e0", "e1", "e2", "e3", "d2", "d1", "d0", "head"]
    assert [(s[1], s[2]) for s in shapes] == [(3, 32), (32, 64), (64, 128), (128, 128),
                                              (256, 64), (128, 32), (64, 32), (32, 1)]
    P = N.param_count(F)
    assert P == sum(co * ci * k ** 3 + co for _, ci, co, k in shapes)
    theta = np.arange(P, dtype=np.float64)
    assert np.array_equal(N.pack(N.unpack(theta, F), F), theta)


def test_backward_matches_finite_differences():
    """The whole backward pass against central differences of the FP64
    loss, on sampled weights and every bias-bearing layer."""
    rng = np.random.default_rng(5)
    F = 3
    n = (8, 8, 16)
    theta = N.init_params(F, seed=6)
    # nonzero biases so that every bias gradient is exercised
    P = N.unpack(theta, F)
    for name in P:
        P[name] = (P[name][0], rng.normal(0.0, 0.05, P[name][1].shape))
    theta = N.pack(P, F)
    x = rng.normal(size=(F,) + n)
    y = (rng.random(n) > 0.5).astype(np.float64)
    loss, g = N.loss_and_grad(theta, x, y)
    assert np.isfinite(loss)
    h = 1e-6
    offs = []
    o = 0
    for _, ci, co, k in N.layer_shapes(F):
        nw = co * ci * k ** 3
        offs += list(o + rng.choice(nw, 4, replace=False)) + [o + nw + rng.integers(co)]
        o += nw + co
    for i in offs:
        tp, tm = theta.copy(), theta.copy()
        tp[i] += h
        tm[i] -= h
        fd = (N.loss_and_grad(tp, x, y)[0] - N.loss_and_grad(tm, x, y)[0]) / (2 * h)
        assert g[i] == pytest.approx(fd, rel=2e-4, abs=1e-8), i


def test_folding_x_neighbours_into_channels_is_exact():
    """The input layer's reading on the GPU: each cell carries the features
    of its x neighbours (offsets -1, 0, +1) as channels dx F + f, zero
    outside the grid, and the 3 x 3 x 3 convolution becomes one over the
    taps at x offset 0 with weights W'[co, dx F + f, 1, b, c] =
    W[co, f, dx, b, c] (all other taps zero).  Both the output and the
    weight gradient must agree with the unfolded layer to rounding."""
    rng = np.random.default_rng(7)
    F, co = 3, 5
    n = (5, 4, 6)
    X = rng.normal(size=(F,) + n)
    W = rng.normal(size=(co, F, 3, 3, 3))
    b = rng.normal(size=co)
    Xf = np.zeros((3 * F,) + n)
    for dx in range(3):
        for i in range(n[0]):
            ii = i + dx - 1
            if 0 <= ii < n[0]:
                Xf[dx * F:(dx + 1) * F, i] = X[:, ii]
    Wf = np.zeros((co, 3 * F, 3, 3, 3))
    for dx in range(3):
        Wf[:, dx * F:(dx + 1) * F, 1] = W[:, :, dx]
    assert np.allclose(N.conv(Xf, Wf, b), N.conv(X, W, b), rtol=1e-12, atol=1e-12)
    dY = rng.normal(size=(co,) + n)
    _, dW, _ = N.conv_backward(X, W, dY)
    _, dWf, _ = N.conv_backward(Xf, Wf, dY)
    for dx in range(3):
        assert np.allclose(dWf[:, dx * F:(dx + 1) * F, 1], dW[:, :, dx], rtol=1e-12, atol=1e-12)


def test_features_invert_to_the_energy_parts():
    """Channel 0 is asinh of the vdW part U - C|E|^2 over the scale, channel
    1 asinh of the CFA part C|E|^2, channel 2 the tight labels: energy
    densities built as scale * sinh(a) + scale * sinh(b) come back as a and
    b (a swapped channel or a missed subtraction fails)."""
    rng = np.random.default_rng(11)
    n = (3, 4, 5)
    a = rng.normal(size=n) * 3.0
    b = rng.normal(size=n) * 3.0
    scale = 0.01
    cfa = scale * np.sinh(b)
    U = scale * np.sinh(a) + cfa
    chi = (rng.random(n) > 0.5).astype(np.uint8)
    x = N.features(U, cfa, chi, scale=scale)
    assert x.shape == (3,) + n
    assert np.allclose(x[0], a, rtol=1e-12, atol=1e-12)
    assert np.allclose(x[1], b, rtol=1e-12, atol=1e-12)
    assert np.array_equal(x[2], chi.astype(np.float64))


def test_bfloat16_storage_only_rounds_the_kept_tensors():
    """store=None is the FP64 network; store=bf16_round keeps every stored
    activation bfloat16-exact and stays within the bfloat16 rounding error
    of the FP64 network, for the logits and for every gradient."""
    rng = np.random.default_rng(7)
    F = 3
    n = (8, 16, 16)
    theta = N.init_params(F, seed=8)
    P = N.unpack(theta, F)
    for name in P:
        P[name] = (P[name][0], N.bf16_round(rng.normal(0.0, 0.05, P[name][1].shape)))
    theta = N.pack(P, F)
    x = N.bf16_round(rng.normal(size=(F,) + n))
    y = (rng.random(n) > 0.5).astype(np.float64)
    z64 = N.forward(theta, x)
    assert np.array_equal(N.forward(theta, x, store=None), z64)
    zq, a, _ = N.forward(theta, x, keep=True, store=N.bf16_round)
    for name in ("e0", "p0", "e1", "p1", "e2", "p2", "e3", "d2", "d1", "d0"):
        assert np.array_equal(N.bf16_round(a[name]), a[name]), name
    # seven stored layers, each rounding to 8 significant bits (2^-8 relative)
    err = np.linalg.norm(zq - z64) / np.linalg.norm(z64)
    assert 0.0 < err < 7 * 2.0 ** -8, err
    l64, g64 = N.loss_and_grad(theta, x, y)
    lq, gq = N.loss_and_grad(theta, x, y, store=N.bf16_round)
    assert lq == pytest.approx(l64, rel=7 * 2.0 ** -8)
    # the gradients go through ReLU masks that the roundings can move on the
    # coarse levels (32 cells at 1/4 resolution here), so they are compared
    # by direction: a dropped term or a transposed operand has cosine ~0
    o = 0
    for name, ci, co, k in N.layer_shapes(F):
        nw = co * ci * k ** 3 + co
        u, v = gq[o:o + nw], g64[o:o + nw]
        cos = float(np.dot(u, v) / (np.linalg.norm(u) * np.linalg.norm(v)))
        assert cos > 0.99, (name, cos)
        o += nw
