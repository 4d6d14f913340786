"""What the learned initialiser gains over the plain start: a network
trained (by the library's own kernels) on label fields that the flip sweep
relaxed from tight starts guesses the relaxed labels of a held-out system;
the unchanged sweep finishes from the guess.  The guess must be closer to
the relaxed labels than the tight start is, and the sweep from it must need
fewer rounds and flips."""
import numpy as np
import pytest

from oracle import unet as N
from paper_2208_05524_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def test_trained_guess_beats_the_tight_start():
    from paper_2208_05524_gb300 import learned, vesis
    h = 0.6
    train_set = [learned.example(synth.host_guest(i, seed=3, h=h)) for i in range(6)]
    held = learned.example(synth.host_guest(40, seed=3, h=h), keep_system=True)
    net = vesis.Net(3)
    theta = learned.init_params(net, seed=0)
    assert len(theta) == N.param_count(3)
    losses = learned.train(net, train_set, steps=240, crop=48, lr=2e-3, seed=1)
    assert np.mean(losses[-20:]) < 0.5 * np.mean(losses[:20])
    S = held["system"]
    chi_g = learned.guess(net, held["x"], held["shape"])
    ref = held["chi"]
    miss_tight = int((held["chi_t"] != ref).sum())
    miss_guess = int((chi_g != ref).sum())
    assert miss_guess < miss_tight, (miss_guess, miss_tight)
    r = S.blsm_relax(chi_g, held["U"], held["E"])
    assert r["rounds"] < held["rounds"], (r["rounds"], held["rounds"])
    assert r["flips"] < held["flips"], (r["flips"], held["flips"])
    # the sweep from the guess ends at a local minimum of the same energy
    # landscape: close to the cold start's energy
    assert r["terms"]["total"] == pytest.approx(held["G_relaxed"], rel=1e-2, abs=1.0)
