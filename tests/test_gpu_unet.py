"""GPU checks of the learned initialiser's kernels against the oracle
(oracle/unet.py), through the C ABI: logits, loss and the gradient of every
layer from the same bfloat16 weights and inputs, element by element.

The oracle keeps the tensors the network stores (activations, pooled
activations, ReLU-masked output gradients) in bfloat16 like the library
(store=bf16_round) and computes everything else in FP64.  Tolerance, for
each compared tensor T (the logits, one layer's weight or bias gradient)
and each element:

  |T_gpu - T_o| <= 2^-4 |T_o| + 2^-6 max|T_o|,

and for the logits also

  |z_gpu - z_o| <= 2^-7 |z_o| + 2^-9 max|z_o|   (one bfloat16 ulp)

for all but 1 % of the cells.  Why no tighter: the GPU accumulates in FP32
and the oracle in FP64, so a stored value next to a bfloat16 rounding
boundary can round to the other neighbour (one ulp, 2^-7 relative); the
next layer sums 27 C_in such values and its own stored values then cross
boundaries too, so the stored tensors differ by about an ulp in most
elements after a few layers.  A tensor reached through n stored roundings
(the logits through the 7 of the forward pass, the input layer's weight
gradient through those and the 7 masked gradients of the backward pass)
carries about sqrt(n) ulps, a few times that in its largest elements: the
bound above is 8 ulps relative plus 2 ulps of the tensor's largest entry,
about twice the largest difference measured.  A wrong tap, a transposed
weight, a dropped term or wrong cells at a grid face change the affected
elements by far more, and a face of any test grid holds more than 1 % of
its cells.  The loss agrees to relative 1e-4."""
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


BOUND = (2.0 ** -4, 2.0 ** -6)
ULP = (2.0 ** -7, 2.0 ** -9)
ULP_SHARE = 1e-2


def _elementwise(g, go, what, ulp_share=None):
    """The element-wise bound above; with ulp_share, also the one-ulp bound
    for all but that share of the elements."""
    g = np.asarray(g, np.float64).ravel()
    go = np.asarray(go, np.float64).ravel()
    d = np.abs(g - go)
    m = np.abs(go).max()
    worst = float((d / np.maximum(BOUND[0] * np.abs(go) + BOUND[1] * m, 1e-300)).max())
    over = int((d > ULP[0] * np.abs(go) + ULP[1] * m).sum())
    ok = worst <= 1.0 and (ulp_share is None or over <= ulp_share * g.size)
    assert ok, (what, worst, over, g.size)


def _compare(z, zo, g, go, loss, lo, F, what):
    _elementwise(z, zo, what + " logits", ULP_SHARE)
    assert loss == pytest.approx(lo, rel=1e-4), what
    for name, sl in _layer_slices(F):
        _elementwise(g[sl], go[sl], what + " " + name)


def _oracle(theta, x, y):
    """Logits (inference) and loss and gradient of the network with its
    stored tensors in bfloat16."""
    zo = N.forward(theta, x, store=N.bf16_round)
    lo, go = N.loss_and_grad(theta, x, y.astype(np.float64), store=N.bf16_round)
    return zo, lo, go


def _gpu(theta, x, y, n, kind="tcgen05", F=3):
    vs = _vs()
    net = vs.Net(F)
    net.set_params(theta)
    net.set_conv_kernel(kind)
    xd = _dev(x.reshape(F, -1).astype(np.float32), torch.float32)
    yd = _dev(y.reshape(-1), torch.uint8)
    z = torch.empty(int(np.prod(n)), dtype=torch.float32, device="cuda")
    chi = torch.empty(int(np.prod(n)), dtype=torch.uint8, device="cuda")
    net.forward(xd, n, logits=z, chi=chi)
    zg = z.cpu().numpy().astype(np.float64)
    assert np.array_equal(chi.cpu().numpy(), (zg > 0).astype(np.uint8))
    loss, g = net.loss_grad(xd, yd, n, grad=True)
    net.close()
    return zg, loss, g.astype(np.float64)


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
    net.close()
    zo, lo, go = _oracle(theta, x, y)
    z, loss, g = _gpu(theta, x, y, n)
    _compare(z, zo.reshape(-1), g, go, loss, lo, 3, "16x16x24")


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
    z = torch.empty(16 * 24 * 16, dtype=torch.float32, device="cuda")
    net.forward(xd, full, crop=crop, logits=z)
    zo, lo, go = _oracle(theta, x[(slice(None),) + sl], y[sl])
    _compare(z.cpu().numpy(), zo.reshape(-1), g, go, loss, lo, 3, "crop")


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


def test_training_is_deterministic():
    """The same training steps twice give bit-identical losses and
    parameters on both convolution paths: every gradient is summed in a
    fixed order (per-block partials added in block order, no atomics)."""
    vs = _vs()
    n = (32, 32, 32)
    theta, x, y = _problem(n, 3)
    xd = _dev(x.reshape(3, -1).astype(np.float32), torch.float32)
    yd = _dev(y.reshape(-1), torch.uint8)
    for kind in ("tcgen05", "mma"):
        runs = []
        for _ in range(2):
            net = vs.Net(3)
            net.set_params(theta)
            net.set_conv_kernel(kind)
            losses = []
            for _ in range(6):
                losses.append(net.loss_grad(xd, yd, n))
                net.adam_step(lr=2e-3)
            runs.append((losses, net.get_params()))
            net.close()
        assert runs[0][0] == runs[1][0], kind
        assert np.array_equal(runs[0][1], runs[1][1]), kind


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


def test_tcgen05_convolutions_match_oracle():
    """The tcgen05 path on a grid with ny % 16 == 0 and nz % 8 == 0 (one
    brick per block, k_conv_tc, at full resolution; the coarser levels fall
    back to mma.sync) and the mma.sync path, each against the oracle."""
    n = (16, 32, 16)
    theta, x, y = _problem(n, 7)
    zo, lo, go = _oracle(theta, x, y)
    for kind in ("mma", "tcgen05"):
        z, loss, g = _gpu(theta, x, y, n, kind)
        _compare(z, zo.reshape(-1), g, go, loss, lo, 3, "16x32x16 " + kind)


def test_tma_convolutions_match_oracle():
    """32 x 64 x 48 cells: the full-resolution level has 768 bricks of
    1 x 16 x 8 cells (at least 608), so its convolutions run on the TMA
    kernel k_conv_tma: e0 with its x taps folded into channels, d0 with the
    1 x 1 head fused into its epilogue for inference, and both layers' input
    gradients; the half-resolution level (96 bricks) runs k_conv_tc.
    Logits of the fused-head inference, loss and every gradient against the
    oracle."""
    n = (32, 64, 48)
    theta, x, y = _problem(n, 21)
    zo, lo, go = _oracle(theta, x, y)
    z, loss, g = _gpu(theta, x, y, n)
    _compare(z, zo.reshape(-1), g, go, loss, lo, 3, "32x64x48")


def test_weight_stationary_tcgen05_matches_oracle_and_mma():
    """A 64^3 grid: the TMA kernel at full resolution, k_conv_tc at half
    resolution (256 bricks).  Against the oracle; and, as an extra, against
    the mma.sync path with the same element-wise tolerance."""
    n = (64, 64, 64)
    theta, x, y = _problem(n, 9)
    zo, lo, go = _oracle(theta, x, y)
    out = {kind: _gpu(theta, x, y, n, kind) for kind in ("tcgen05", "mma")}
    z, loss, g = out["tcgen05"]
    _compare(z, zo.reshape(-1), g, go, loss, lo, 3, "64^3 tcgen05")
    zm, lm, gm = out["mma"]
    _compare(z, zm, g, gm, loss, lm, 3, "64^3 tcgen05 vs mma")


def test_wide_input_without_folding_matches_oracle():
    """With 3 features the input layer carries each cell's x neighbours as
    channels (9 of its 32); with 12 features that no longer fits and the
    layer keeps its 27 taps.  Logits, loss and every layer's gradient of the
    12-feature network against the oracle, on both convolution paths."""
    n = (16, 32, 16)
    F = 12
    theta, x, y = _problem(n, 11, F=F)
    assert _vs().Net(F).P == N.param_count(F)
    zo, lo, go = _oracle(theta, x, y)
    for kind in ("mma", "tcgen05"):
        z, loss, g = _gpu(theta, x, y, n, kind, F=F)
        _compare(z, zo.reshape(-1), g, go, loss, lo, F, "F=12 " + kind)
