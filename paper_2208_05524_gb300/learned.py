"""Learned initialiser: training data from the plain method, training, and
the guess the flip sweep finishes from.

Every step runs in the CUDA library (fields, tight labels, flip sweep,
features, the network's forward and backward passes, Adam); this module
only chooses systems and crops and moves handles around.
"""
from __future__ import annotations

import numpy as np

from . import vesis

FEATURE_SCALE = 0.01    # kBT/A^3, the scale inside the features' asinh


def example(sysd, stream=None, keep_system=False):
    """Features and target labels of one system: the fields at its atoms,
    the tight start, and the labels the flip sweep relaxes it to.  Returns a
    dict of device tensors (x: 3 x G features, chi: relaxed labels, chi_t:
    tight start, U, E) with the sweep's rounds and flips from the tight
    start."""
    import torch
    S = vesis.System(sysd, stream=stream)
    G = S.G
    dev = torch.device("cuda", torch.cuda.current_device())
    U = torch.empty(G, dtype=torch.float32, device=dev)
    E = torch.empty(3 * G, dtype=torch.float32, device=dev)
    S.energy_field(U, E)
    chi_t = torch.empty(G, dtype=torch.uint8, device=dev)
    S.init_labels(chi_t, "tight")
    x = torch.empty(3 * G, dtype=torch.float32, device=dev)
    S.features(U, E, chi_t, x, scale=FEATURE_SCALE)
    chi = chi_t.clone()
    r = S.blsm_relax(chi, U, E)
    out = dict(shape=S.shape, x=x, chi=chi, chi_t=chi_t, U=U, E=E, rounds=r["rounds"],
               flips=r["flips"], G_relaxed=r["terms"]["total"])
    if keep_system:
        out["system"] = S
    else:
        S.close()
    return out


def init_params(net, seed):
    """He-normal weights (standard deviation sqrt(2 / fan-in)), rounded to
    bfloat16, and zero biases, in the network's flat parameter order."""
    import torch
    rng = np.random.default_rng(seed)
    shapes = [(net.F, 32, 3), (32, 64, 3), (64, 128, 3), (128, 128, 3), (256, 64, 3),
              (128, 32, 3), (64, 32, 3), (32, 1, 1)]
    parts = []
    for ci, co, k in shapes:
        w = rng.normal(0.0, np.sqrt(2.0 / (ci * k ** 3)), co * ci * k ** 3)
        parts.append(torch.from_numpy(w.astype(np.float32)).to(torch.bfloat16)
                     .to(torch.float32).numpy())
        parts.append(np.zeros(co, np.float32))
    theta = np.concatenate(parts)
    net.set_params(theta)
    return theta


def random_crop(shape, size, rng):
    """Crop origin (multiple of 8) and size (min(size, dim) rounded down to
    8) inside a grid."""
    c = [min(size, (d // 8) * 8) for d in shape]
    o = [int(rng.integers(0, (d - s) // 8 + 1)) * 8 for d, s in zip(shape, c)]
    return tuple(o) + tuple(c)


def train(net, examples, steps, crop=64, lr=1e-3, seed=0, log_every=0):
    """Adam on random crops of random examples; returns the losses."""
    rng = np.random.default_rng(seed)
    losses = []
    for k in range(steps):
        e = examples[int(rng.integers(len(examples)))]
        c = random_crop(e["shape"], crop, rng)
        losses.append(net.loss_grad(e["x"], e["chi"], e["shape"], crop=c))
        net.adam_step(lr=lr)
        if log_every and (k + 1) % log_every == 0:
            print(f"step {k + 1}: loss {np.mean(losses[-log_every:]):.4f}", flush=True)
    return losses


def guess(net, x, shape):
    """The network's labels chi = [logit > 0] of a whole grid (dimensions
    multiples of 8)."""
    import torch
    G = int(np.prod(shape))
    chi = torch.empty(G, dtype=torch.uint8, device=x.device)
    net.forward(x, shape, chi=chi)
    return chi
