"""Plain FP64 oracle of the learned initialiser's network.

TEST INFRASTRUCTURE ONLY (like the rest of `oracle/`): the tests, the smoke
check and the benchmark's CPU legs may use it; the CUDA path never does and
shares no code with it.

The paper relaxes from tight or loose initial surfaces (Sec. 3.1, "Initial
surfaces"); the learned initialiser replaces that start by a guess of the
relaxed labels from two features of the atoms: an atom-density indicator
and the Coulomb-field-approximation term of the energy density.  The flip
sweep always finishes from the guess.

The network (channels per level 32, 64, 128, 128; every grid dimension a
multiple of 8):

  e0 = relu(conv3(x))                 F   -> 32   at R
  e1 = relu(conv3(pool(e0)))          32  -> 64   at R/2
  e2 = relu(conv3(pool(e1)))          64  -> 128  at R/4
  e3 = relu(conv3(pool(e2)))          128 -> 128  at R/8
  d2 = relu(conv3([e2, up(e3)]))      256 -> 64   at R/4
  d1 = relu(conv3([e1, up(d2)]))      128 -> 32   at R/2
  d0 = relu(conv3([e0, up(d1)]))      64  -> 32   at R
  z  = conv1(d0)                      32  -> 1    at R    (logit of chi = 1)
  loss = mean over cells of the binary cross entropy of sigmoid(z) and chi

conv3: 3x3x3 cross-correlation with zero padding and a bias; conv1: 1x1x1;
pool: mean over 2x2x2 blocks; up: nearest-neighbour doubling; [a, b]:
channel concatenation.  Arrays are channels-first (C, nx, ny, nz) here.

Every function is written out from these definitions; the backward pass is
the chain rule of the same definitions, pinned by central finite differences
of the loss.

Storage precision.  The network keeps its weights and the tensors it
passes between layers in bfloat16 (8 significant bits) and accumulates in
FP32.  forward() and loss_and_grad() take `store`, the rounding applied to
every tensor the network keeps: the activations after each ReLU, the pooled
activations and, in the backward pass, each layer's ReLU-masked output
gradient (the tensor its weight and input gradients are built from).
store=None keeps everything in FP64 (the exact function of the bfloat16
weights and inputs); store=bf16_round gives the network at its defined
storage precision, with FP64 arithmetic everywhere else.
"""
from __future__ import annotations

import numpy as np

LAYERS = [  # name, input channels (skip, coarse), output channels, kernel
    ("e0", (None, None), 32, 3),
    ("e1", (32, None), 64, 3),
    ("e2", (64, None), 128, 3),
    ("e3", (128, None), 128, 3),
    ("d2", (128, 128), 64, 3),
    ("d1", (64, 64), 32, 3),
    ("d0", (32, 32), 32, 3),
    ("head", (32, None), 1, 1),
]


def layer_shapes(F):
    """(name, cin, cout, k) of each layer for F input features."""
    out = []
    for name, (a, b), co, k in LAYERS:
        ci = F if name == "e0" else a + (b or 0)
        out.append((name, ci, co, k))
    return out


def param_count(F):
    return sum(co * ci * k ** 3 + co for _, ci, co, k in layer_shapes(F))


def unpack(theta, F):
    """Flat parameter vector -> {name: (W[co, ci, k, k, k], b[co])}, layer by
    layer in the order above, each W then b."""
    out, o = {}, 0
    for name, ci, co, k in layer_shapes(F):
        n = co * ci * k ** 3
        W = np.asarray(theta[o:o + n], np.float64).reshape(co, ci, k, k, k)
        o += n
        b = np.asarray(theta[o:o + co], np.float64)
        o += co
        out[name] = (W, b)
    assert o == len(theta)
    return out


def pack(grads, F):
    parts = []
    for name, _, _, _ in layer_shapes(F):
        W, b = grads[name]
        parts += [W.reshape(-1), b.reshape(-1)]
    return np.concatenate(parts)


def bf16_round(x):
    """Round to the nearest bfloat16 (ties to even), via float32."""
    f = np.ascontiguousarray(np.asarray(x, np.float32))
    u = f.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def init_params(F, seed):
    """He-normal weights (std sqrt(2 / fan_in)), zero biases, rounded to
    bfloat16 so that both sides start from representable weights."""
    rng = np.random.default_rng(seed)
    parts = []
    for _, ci, co, k in layer_shapes(F):
        fan = ci * k ** 3
        parts.append(rng.normal(0.0, np.sqrt(2.0 / fan), co * ci * k ** 3))
        parts.append(np.zeros(co))
    return bf16_round(np.concatenate(parts))


# ---------------------------------------------------------------- layers

def _shift(X, a, b, c):
    """X shifted so that out[..., i, j, k] = X[..., i+a, j+b, k+c] (zero
    outside)."""
    out = np.zeros_like(X)
    n = X.shape[1:]
    src = [slice(max(0, d), min(nn, nn + d)) for d, nn in zip((a, b, c), n)]
    dst = [slice(max(0, -d), min(nn, nn - d)) for d, nn in zip((a, b, c), n)]
    out[(slice(None),) + tuple(dst)] = X[(slice(None),) + tuple(src)]
    return out


def conv(X, W, b):
    """Y[co, p] = b[co] + sum_{ci, t} W[co, ci, t] X[ci, p + t - r]."""
    k = W.shape[2]
    r = k // 2
    Y = np.zeros((W.shape[0],) + X.shape[1:]) + b[:, None, None, None]
    for a in range(k):
        for bb in range(k):
            for c in range(k):
                Xs = _shift(X, a - r, bb - r, c - r)
                Y += np.tensordot(W[:, :, a, bb, c], Xs, axes=(1, 0))
    return Y


def conv_backward(X, W, dY):
    """Gradients of conv with respect to X, W and b."""
    k = W.shape[2]
    r = k // 2
    dX = np.zeros_like(X)
    dW = np.zeros_like(W)
    for a in range(k):
        for bb in range(k):
            for c in range(k):
                Xs = _shift(X, a - r, bb - r, c - r)
                dW[:, :, a, bb, c] = np.tensordot(dY, Xs, axes=([1, 2, 3], [1, 2, 3]))
                # X[ci, q] feeds Y[co, q - t + r]
                dX += _shift(np.tensordot(W[:, :, a, bb, c], dY, axes=(0, 0)),
                             -(a - r), -(bb - r), -(c - r))
    db = dY.sum(axis=(1, 2, 3))
    return dX, dW, db


def pool(X):
    C, nx, ny, nz = X.shape
    return X.reshape(C, nx // 2, 2, ny // 2, 2, nz // 2, 2).mean(axis=(2, 4, 6))


def pool_backward(dY):
    return np.repeat(np.repeat(np.repeat(dY, 2, 1), 2, 2), 2, 3) / 8.0


def up(X):
    return np.repeat(np.repeat(np.repeat(X, 2, 1), 2, 2), 2, 3)


def up_backward(dY):
    C, nx, ny, nz = dY.shape
    return dY.reshape(C, nx // 2, 2, ny // 2, 2, nz // 2, 2).sum(axis=(2, 4, 6))


def bce_with_logits(z, y):
    """Mean binary cross entropy of sigmoid(z) against labels y, and its
    gradient with respect to z."""
    z = np.asarray(z, np.float64)
    y = np.asarray(y, np.float64)
    loss = np.mean(np.maximum(z, 0.0) - z * y + np.log1p(np.exp(-np.abs(z))))
    s = 1.0 / (1.0 + np.exp(-z))
    return loss, (s - y) / z.size


# ---------------------------------------------------------------- network

def _store(store):
    return (lambda v: v) if store is None else store


def forward(theta, x, F=None, keep=False, store=None):
    """Logits z (nx, ny, nz) of features x (F, nx, ny, nz); `store` rounds
    every kept activation (see the module notes)."""
    F = x.shape[0] if F is None else F
    P = unpack(theta, F)
    q = _store(store)
    relu = lambda v: np.maximum(v, 0.0)
    a = {}
    a["e0"] = q(relu(conv(x, *P["e0"])))
    a["p0"] = q(pool(a["e0"]))
    a["e1"] = q(relu(conv(a["p0"], *P["e1"])))
    a["p1"] = q(pool(a["e1"]))
    a["e2"] = q(relu(conv(a["p1"], *P["e2"])))
    a["p2"] = q(pool(a["e2"]))
    a["e3"] = q(relu(conv(a["p2"], *P["e3"])))
    a["c2"] = np.concatenate([a["e2"], up(a["e3"])])
    a["d2"] = q(relu(conv(a["c2"], *P["d2"])))
    a["c1"] = np.concatenate([a["e1"], up(a["d2"])])
    a["d1"] = q(relu(conv(a["c1"], *P["d1"])))
    a["c0"] = np.concatenate([a["e0"], up(a["d1"])])
    a["d0"] = q(relu(conv(a["c0"], *P["d0"])))
    z = conv(a["d0"], *P["head"])[0]
    return (z, a, P) if keep else z


def loss_and_grad(theta, x, y, store=None):
    """Loss and its gradient with respect to the flat parameters; `store`
    rounds the kept activations and the masked output gradients."""
    F = x.shape[0]
    q = _store(store)
    z, a, P = forward(theta, x, F, keep=True, store=store)
    loss, dz = bce_with_logits(z, y)
    g = {}
    _, g_hW, g_hb = conv_backward(a["d0"], P["head"][0], dz[None])
    dd0 = np.einsum("oi,oxyz->ixyz", P["head"][0][:, :, 0, 0, 0], dz[None])
    g["head"] = (g_hW, g_hb)

    def block(name, inp, out, dout):
        dpre = q(dout * (out > 0))
        dinp, dW, db = conv_backward(inp, P[name][0], dpre)
        g[name] = (dW, db)
        return dinp

    dc0 = block("d0", a["c0"], a["d0"], dd0)
    de0 = dc0[:32].copy()
    dd1 = up_backward(dc0[32:])
    dc1 = block("d1", a["c1"], a["d1"], dd1)
    de1 = dc1[:64].copy()
    dd2 = up_backward(dc1[64:])
    dc2 = block("d2", a["c2"], a["d2"], dd2)
    de2 = dc2[:128].copy()
    de3 = up_backward(dc2[128:])
    dp2 = block("e3", a["p2"], a["e3"], de3)
    de2 += pool_backward(dp2)
    dp1 = block("e2", a["p1"], a["e2"], de2)
    de1 += pool_backward(dp1)
    dp0 = block("e1", a["p0"], a["e1"], de1)
    de0 += pool_backward(dp0)
    block("e0", x, a["e0"], de0)
    return loss, pack(g, F)


def features(U, E_sq_term, chi_tight, scale=0.01):
    """Input features (3, nx, ny, nz) of a system: asinh of the vdW part of
    the energy density U - C|E|^2 and of the CFA part C|E|^2, each over
    `scale` kBT/A^3, and the tight-surface labels (1 within sigma_i of an
    atom) as the atom-density indicator."""
    U = np.asarray(U, np.float64)
    cfa = np.asarray(E_sq_term, np.float64)
    return np.stack([np.arcsinh((U - cfa) / scale), np.arcsinh(cfa / scale),
                     np.asarray(chi_tight, np.float64)])
