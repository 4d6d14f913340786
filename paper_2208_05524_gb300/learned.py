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


def protein_field(index, seed, atoms=(500, 4000), n=256, h=0.4):
    """The `index`-th training solute of a seeded set in the style of the
    protein-like workload: a random-walk globule whose atom count is drawn
    log-uniform in `atoms`, with that workload's parameter distributions,
    on an n^3 grid at spacing h.  Each solute has its own seed, drawn from
    the set's seed, so any one of them can be rebuilt alone."""
    from . import synth
    rng = np.random.default_rng([seed, index])
    na = int(round(np.exp(rng.uniform(np.log(atoms[0]), np.log(atoms[1])))))
    return synth.protein_like(n_atoms=na, n=n, h=h, seed=int(rng.integers(1 << 31)))


def crop_bank(systems, n_fields, seed, crop=64, group=8, log_every=0):
    """Training crops from plain relaxations: for each of the n_fields
    solutes that `systems` yields (protein_field(i, seed) for i = 0, 1, ...,
    built here or by worker processes), the tight start relaxed by the flip
    sweep at fixed atoms (the plain method; `group` solutes at a time in one
    multi-system sweep, vesis_blsm_relax_batch), and one crop^3 window of
    its features and relaxed labels, centred on a randomly chosen atom (so
    that it holds solute, interface and solvent) and kept inside the grid on
    the 8-cell lattice.  Returns the crops as device tensors x
    [n_fields][3][crop^3] and chi [n_fields][crop^3], with the sweeps'
    rounds and flips."""
    import torch
    dev = torch.device("cuda", torch.cuda.current_device())
    V = crop ** 3
    X = torch.empty((n_fields, 3, V), dtype=torch.float32, device=dev)
    Y = torch.empty((n_fields, V), dtype=torch.uint8, device=dev)
    rounds = flips = 0
    it = iter(zip(range(n_fields), systems))
    while True:
        batch = []
        for _ in range(group):
            nxt = next(it, None)
            if nxt is None:
                break
            i, sd = nxt
            S = vesis.System(sd)
            U = torch.empty(S.G, dtype=torch.float32, device=dev)
            E = torch.empty(3 * S.G, dtype=torch.float32, device=dev)
            S.energy_field(U, E)
            chi = torch.empty(S.G, dtype=torch.uint8, device=dev)
            S.init_labels(chi, "tight")
            x = torch.empty(3 * S.G, dtype=torch.float32, device=dev)
            S.features(U, E, chi, x, scale=FEATURE_SCALE)
            batch.append((i, sd, S, U, chi, x))
        if not batch:
            break
        res = vesis.blsm_relax_batch([b[2] for b in batch], [b[4] for b in batch],
                                     [b[3] for b in batch])
        for (i, sd, S, U, chi, x), r in zip(batch, res):
            e = dict(shape=S.shape, x=x, chi=chi, rounds=r["rounds"], flips=r["flips"])
            S.close()
            _crop_into(X, Y, i, e, sd, seed, crop)
            rounds += e["rounds"]
            flips += e["flips"]
        done = batch[-1][0] + 1
        if log_every and (done // log_every) != ((done - len(batch)) // log_every):
            print(f"field {done}/{n_fields}", flush=True)
    return dict(x=X, chi=Y, crop=crop, rounds=rounds, flips=flips)


def _crop_into(X, Y, i, e, sd, seed, crop):
    """Copies the crop^3 window of example e (features x, relaxed labels
    chi) around an atom of sd chosen with the generator of (seed, i) into
    X[i] and Y[i]."""
    V = crop ** 3
    rng = np.random.default_rng([seed, i, 1])
    a = sd["xyz"][int(rng.integers(len(sd["xyz"])))]
    cell = np.floor((a - np.asarray(sd["origin"])) / sd["h"]).astype(int)
    o = [int(np.clip((c - crop // 2) // 8 * 8, 0, d - crop)) for c, d in zip(cell, e["shape"])]
    sl = tuple(slice(oo, oo + crop) for oo in o)
    nx, ny, nz = e["shape"]
    X[i] = e["x"].view(3, nx, ny, nz)[(slice(None),) + sl].reshape(3, V)
    Y[i] = e["chi"].view(nx, ny, nz)[sl].reshape(V)


def train_bank(net, bank, steps, lr=1e-3, seed=0):
    """Adam, one crop of the bank per step, drawn with a seeded generator;
    returns the losses.  Every gradient is summed in a fixed order, so the
    same bank, seed and start give the same parameters."""
    rng = np.random.default_rng(seed)
    c = bank["crop"]
    losses = []
    for _ in range(steps):
        i = int(rng.integers(bank["x"].shape[0]))
        losses.append(net.loss_grad(bank["x"][i], bank["chi"][i], (c, c, c)))
        net.adam_step(lr=lr)
    return losses


def guess(net, x, shape):
    """The network's labels chi = [logit > 0] of a whole grid (dimensions
    multiples of 8)."""
    import torch
    G = int(np.prod(shape))
    chi = torch.empty(G, dtype=torch.uint8, device=x.device)
    net.forward(x, shape, chi=chi)
    return chi
