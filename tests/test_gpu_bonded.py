"""Bending and torsion terms of G_ss (Eq. Gss) on the GPU against the
oracle: energies, and their gradient (the appendix's force formulas)."""
import math

import numpy as np
import pytest

import oracle as O
from paper_2208_05524_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _sys():
    s = synth.protein_like(n_atoms=300, n=64, h=0.5, seed=5)
    return synth.with_bends_torsions(s, theta0_shift=0.2)


def test_bend_torsion_energies_and_gradient_match_oracle():
    from paper_2208_05524_gb300 import vesis
    s = _sys()
    S = vesis.System(s)
    t = S.ss_terms()
    eb, et, gbt = O.bonded_terms(s)
    assert t["bend"] == pytest.approx(eb, rel=1e-10)
    assert t["torsion"] == pytest.approx(et, rel=1e-10)
    chi = torch.from_numpy(O.init_labels(s).reshape(-1)).cuda()
    g_with = S.atom_forces(chi)
    S.set_bonded()                      # remove them
    assert S.ss_terms()["bend"] == 0.0 and S.ss_terms()["torsion"] == 0.0
    g_without = S.atom_forces(chi)
    d = g_with - g_without
    assert np.allclose(d, gbt, rtol=1e-8, atol=1e-8 * np.abs(gbt).max())
    # and the whole gradient against the oracle's
    S.set_bonded(s["angles"], s["angle_B"], s["angle_theta0"], s["torsions"],
                 s["torsion_C"], s["torsion_psi"])
    go = O.gradient(s, O.params(), O.init_labels(s))
    g = S.atom_forces(chi)
    assert np.all(np.abs(g - go) <= 1e-4 * np.abs(go) + 1e-4 * np.abs(go).max())


def test_relax_with_bends_and_torsions_lowers_the_energy():
    from paper_2208_05524_gb300 import vesis
    s = _sys()
    S = vesis.System(s)
    chi = torch.empty(S.G, dtype=torch.uint8, device="cuda")
    S.init_labels(chi, "tight")
    U = torch.empty(S.G, dtype=torch.float32, device="cuda")
    E = torch.empty(3 * S.G, dtype=torch.float32, device="cuda")
    t0 = S.energy_field(U, E, chi=chi, terms=True)
    r = S.relax(chi, s["xyz"], max_outer=5)
    assert r["status"] >= 0 and r["iterations"] >= 1
    assert r["G"] < t0["total"]


def test_set_bonded_arguments():
    from paper_2208_05524_gb300 import vesis
    s = _sys()
    S = vesis.System(s)
    bad = s["torsion_psi"].copy()
    bad[0, 2] = 1.0
    with pytest.raises(vesis.VesisError, match="phases"):
        S.set_bonded(s["angles"], s["angle_B"], s["angle_theta0"], s["torsions"],
                     s["torsion_C"], bad)
    ang = s["angles"].copy()
    ang[0, 0] = 10 ** 6
    with pytest.raises(vesis.VesisError, match="range"):
        S.set_bonded(ang, s["angle_B"], s["angle_theta0"])
    with pytest.raises(vesis.VesisError):
        S.set_bonded(s["angles"], s["angle_B"], np.full(len(s["angles"]), 4.0))
    assert math.isfinite(S.ss_terms()["bend"])
