"""GPU checks of the learned initialiser's kernels against the FP64 oracle
(oracle/unet.py): logits, loss and the gradient of every layer from the
same bfloat16 weights and inputs, through the C ABI.  The GPU stores
activations and the ReLU-masked gradients in bfloat16, so agreement is
judged on each tensor as a whole: relative L2 error below 5e-2 and cosine
above 0.998 (a transposed weight, a wrong tap or a missing term gives
errors of order one)."""
import numpy as np
import pytest

import oracle as O
from oracle import unet as N
from paper_2208_05524_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _vs():
    from paper_2208_05524_gb300 import vesis
    return vesis


def _dev(a, dtype):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda").to(dtype).contiguous()


def _problem(n, seed, F=3):
    rng = np.random.default_rng(seed)
    theta = N.init_params(F, seed=seed)
    P = N.unpack(theta, F)
    for k in P:   # small biases, exactly representable in FP32
        P[k] = (P[k][0], np.float32(rng.normal(0.0, 0.05, P[k][1].shape)).astype(np.float64))
    theta = N.pack(P, F)
    x = N.bf16_round(rng.normal(size=(F,) + tuple(n)))
    idx = np.indices(n).reshape(3, -1).T
    c = np.array(n) / 2.0
    y = (np.linalg.norm(idx - c, axis=1) < min(n) / 3.0).reshape(n).astype(np.uint8)
    y ^= (rng.random(n) < 0.05).astype(np.uint8)
    return theta, x, y


def _compare(g, go):
    err = np.linalg.norm(g - go) / max(np.linalg.norm(go), 1e-30)
    cos = float(np.dot(g, go) / max(np.linalg.norm(g) * np.linalg.norm(go), 1e-30))
    return err, cos


def _layer_slices(F):
    o, out = 0, []
    for name, ci, co, k in N.layer_shapes(F):
        nw = co * ci * k ** 3
        out.append((name + ".W", slice(o, o + nw)))
        out.append((name + ".b", slice(o + nw, o + nw + co)))
        o += nw + co
    return out


def test_forward_and_gradients_match_oracle():
    vs = _vs()
    n = (16, 16, 24)
    theta, x, y = _problem(n, 1)
    net = vs.Net(3)
    assert net.P == N.param_count(3)
    net.set_params(theta)
    assert np.array_equal(net.get_params().astype(np.float64), theta)
    xd = _dev(x.reshape(3, -1).astype(np.float32), torch.float32)
    yd = _dev(y.reshape(-1), torch.uint8)
    z = torch.empty(int(np.prod(n)), dtype=torch.float32, device="cuda")
    chi = torch.empty(int(np.prod(n)), dtype=torch.uint8, device="cuda")
    net.forward(xd, n, logits=z, chi=chi)
    zo = N.forward(theta, x)
    zg = z.cpu().numpy().reshape(n)
    err, cos = _compare(zg.reshape(-1), zo.reshape(-1))
    assert err < 5e-2 and cos > 0.998, (err, cos)
    assert np.array_equal(chi.cpu().numpy().reshape(n), (zg > 0).astype(np.uint8))
    loss, g = net.loss_grad(xd, yd, n, grad=True)
    lo, go = N.loss_and_grad(theta, x, y.astype(np.float64))
    assert loss == pytest.approx(lo, rel=1e-2)
    for name, sl in _layer_slices(3):
        err, cos = _compare(g[sl].astype(np.float64), go[sl])
        assert err < 5e-2 and cos > 0.998, (name, err, cos)


def test_crop_reads_the_right_window():
    vs = _vs()
    full = (24, 24, 32)
    theta, x, y = _problem(full, 2)
    crop = (8, 0, 8, 16, 24, 16)
    sl = (slice(8, 24), slice(0, 24), slice(8, 24))
    net = vs.Net(3)
    net.set_params(theta)
    xd = _dev(x.reshape(3, -1).astype(np.float32), torch.float32)
    yd = _dev(y.reshape(-1), torch.uint8)
    loss, g = net.loss_grad(xd, yd, full, crop=crop, grad=True)
    lo, go = N.loss_and_grad(theta, x[(slice(None),) + sl], y[sl].astype(np.float64))
    assert loss == pytest.approx(lo, rel=1e-2)
    err, cos = _compare(g.astype(np.float64), go)
    assert err < 5e-2 and cos > 0.998, (err, cos)


def test_training_lowers_the_loss():
    vs = _vs()
    n = (32, 32, 32)
    theta, x, y = _problem(n, 3)
    net = vs.Net(3)
    net.set_params(theta)
    xd = _dev(x.reshape(3, -1).astype(np.float32), torch.float32)
    yd = _dev(y.reshape(-1), torch.uint8)
    l0 = net.loss_grad(xd, yd, n)
    for _ in range(60):
        net.loss_grad(xd, yd, n)
        net.adam_step(lr=2e-3)
    l1 = net.loss_grad(xd, yd, n)
    assert l1 < 0.5 * l0, (l0, l1)


def test_features_match_oracle():
    vs = _vs()
    s = synth.random_cluster(40, 32, 0.5, seed=4, net_charge=1.0)
    S = vs.System(s)
    G = S.G
    U = torch.empty(G, dtype=torch.float32, device="cuda")
    E = torch.empty(3 * G, dtype=torch.float32, device="cuda")
    S.energy_field(U, E)
    chi_t = torch.empty(G, dtype=torch.uint8, device="cuda")
    S.init_labels(chi_t, "tight")
    x = torch.empty(3 * G, dtype=torch.float32, device="cuda")
    S.features(U, E, chi_t, x, scale=0.01)
    Ue = U.cpu().numpy().astype(np.float64)
    Ee = E.cpu().numpy().astype(np.float64).reshape(3, G)
    cfa = O.cfa_prefactor(O.params()) * np.einsum("ig,ig->g", Ee, Ee)
    xo = N.features(Ue, cfa, chi_t.cpu().numpy(), scale=0.01)
    xg = x.cpu().numpy().reshape(3, G)
    assert np.array_equal(xg[2], xo[2])
    for c in range(2):
        assert np.allclose(xg[c], xo[c], rtol=1e-5, atol=1e-5), c


def test_net_arguments():
    vs = _vs()
    net = vs.Net(3)
    x = torch.zeros(3 * 8 * 8 * 12, device="cuda")
    with pytest.raises(vs.VesisError):       # 12 is not a multiple of 8
        net.forward(x, (8, 8, 12))
    with pytest.raises(vs.VesisError):       # crop outside the grid
        net.forward(x, (8, 8, 12), crop=(0, 0, 8, 8, 8, 8))
    with pytest.raises(vs.VesisError):
        net.set_params(np.full(net.P, np.nan, np.float32))


def test_tcgen05_convolutions_match_mma_and_oracle():
    """The tcgen05 path (grids with ny % 16 == 0 and nz % 8 == 0; the
    coarser levels here fall back to mma.sync) against the mma.sync path
    and the oracle: logits, loss and every layer's gradient."""
    vs = _vs()
    n = (16, 32, 16)
    theta, x, y = _problem(n, 7)
    xd = _dev(x.reshape(3, -1).astype(np.float32), torch.float32)
    yd = _dev(y.reshape(-1), torch.uint8)
    out = {}
    for kind in ("mma", "tcgen05"):
        net = vs.Net(3)
        net.set_params(theta)
        net.set_conv_kernel(kind)
        z = torch.empty(int(np.prod(n)), dtype=torch.float32, device="cuda")
        net.forward(xd, n, logits=z)
        loss, g = net.loss_grad(xd, yd, n, grad=True)
        out[kind] = (z.cpu().numpy(), loss, g)
    zm, zt = out["mma"][0], out["tcgen05"][0]
    err, cos = _compare(zt.astype(np.float64), zm.astype(np.float64))
    assert err < 1e-2 and cos > 0.9999, (err, cos)
    zo = N.forward(theta, x).reshape(-1)
    err, cos = _compare(zt.astype(np.float64), zo)
    assert err < 5e-2 and cos > 0.998, (err, cos)
    lo, go = N.loss_and_grad(theta, x, y.astype(np.float64))
    assert out["tcgen05"][1] == pytest.approx(lo, rel=1e-2)
    for name, sl in _layer_slices(3):
        err, cos = _compare(out["tcgen05"][2][sl].astype(np.float64), go[sl])
        assert err < 5e-2 and cos > 0.998, (name, err, cos)


def test_weight_stationary_tcgen05_matches_mma():
    """A 64^3 grid: its full-resolution levels have enough 16 x 8 bricks for
    the weight-stationary tcgen05 kernel (8 bricks per block sharing one
    weight load, accumulators in tensor memory); logits and gradients
    against the mma.sync path."""
    vs = _vs()
    n = (64, 64, 64)
    theta, x, y = _problem(n, 9)
    xd = _dev(x.reshape(3, -1).astype(np.float32), torch.float32)
    yd = _dev(y.reshape(-1), torch.uint8)
    out = {}
    for kind in ("mma", "tcgen05"):
        net = vs.Net(3)
        net.set_params(theta)
        net.set_conv_kernel(kind)
        z = torch.empty(int(np.prod(n)), dtype=torch.float32, device="cuda")
        net.forward(xd, n, logits=z)
        loss, g = net.loss_grad(xd, yd, n, grad=True)
        out[kind] = (z.cpu().numpy().astype(np.float64), loss, g.astype(np.float64))
    err, cos = _compare(out["tcgen05"][0], out["mma"][0])
    assert err < 1e-2 and cos > 0.9999, (err, cos)
    assert out["tcgen05"][1] == pytest.approx(out["mma"][1], rel=1e-3)
    for name, sl in _layer_slices(3):
        err, cos = _compare(out["tcgen05"][2][sl], out["mma"][2][sl])
        assert err < 2e-2 and cos > 0.9998, (name, err, cos)


def test_wide_input_without_folding_matches_oracle():
    """With 3 features the input layer carries each cell's x neighbours as
    channels (9 of its 32); with 12 features that no longer fits and the
    layer keeps its 27 taps.  Logits, loss and every layer's gradient of the
    12-feature network against the oracle, on both convolution paths."""
    vs = _vs()
    n = (16, 32, 16)
    F = 12
    theta, x, y = _problem(n, 11, F=F)
    xd = _dev(x.reshape(F, -1).astype(np.float32), torch.float32)
    yd = _dev(y.reshape(-1), torch.uint8)
    zo = N.forward(theta, x).reshape(-1)
    lo, go = N.loss_and_grad(theta, x, y.astype(np.float64))
    for kind in ("mma", "tcgen05"):
        net = vs.Net(F)
        assert net.P == N.param_count(F)
        net.set_params(theta)
        net.set_conv_kernel(kind)
        z = torch.empty(int(np.prod(n)), dtype=torch.float32, device="cuda")
        net.forward(xd, n, logits=z)
        err, cos = _compare(z.cpu().numpy().astype(np.float64), zo)
        assert err < 5e-2 and cos > 0.998, (kind, err, cos)
        loss, g = net.loss_grad(xd, yd, n, grad=True)
        assert loss == pytest.approx(lo, rel=1e-2)
        for name, sl in _layer_slices(F):
            err, cos = _compare(g[sl].astype(np.float64), go[sl])
            assert err < 5e-2 and cos > 0.998, (kind, name, err, cos)
