"""Potential of mean force (the paper's appendix): one point of the two-atom
curve against the oracle, and the definition's bookkeeping."""
import numpy as np
import pytest

import oracle as O
from paper_2208_05524_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _pair(d, charges, n=48, h=0.4):
    s = synth.two_atom(d, charges=charges, n=n, h=h)
    s["bonds"] = np.zeros((0, 2), np.int32)
    s["bond_k"] = np.zeros(0)
    s["bond_r0"] = np.zeros(0)
    return s


@pytest.mark.parametrize("charges", [(1.0, -1.0), (1.0, 1.0)])
def test_pmf_point_matches_oracle(charges):
    from paper_2208_05524_gb300 import pmf, vesis
    d = 6.0
    s = _pair(d, charges)
    p = O.params()
    S = vesis.System(s)
    G = S.G
    U = torch.empty(G, dtype=torch.float32, device="cuda")
    E = torch.empty(3 * G, dtype=torch.float32, device="cuda")
    chi = torch.empty(G, dtype=torch.uint8, device="cuda")
    got = pmf.relaxed_parts(S, chi, U, E, s["xyz"], "tight")
    # the oracle relaxes the same start with the same FP32 U (identical labels)
    n = tuple(int(v) for v in s["n"])
    chi0 = O.init_labels(s)
    ref = chi0.copy()
    O.blsm_parallel(ref, U.cpu().numpy().astype(np.float64).reshape(n),
                    O.surface_constants(s, p))
    assert np.array_equal(chi.cpu().numpy(), ref.reshape(-1))
    T = O.energy_terms(s, p, ref)
    assert got["geom"] == pytest.approx(T["surf"], rel=1e-9)
    assert got["vdw"] == pytest.approx(T["vdw"], rel=1e-5)
    assert got["elec"] == pytest.approx(T["cfa"], rel=1e-5)
    e_ss, _ = O.ss_terms(s, p)
    assert got["lj"] == pytest.approx(e_ss[1], rel=1e-12)
    assert got["coulomb"] == pytest.approx(e_ss[2], rel=1e-12)
    # Coulomb between the atoms alone: l_B q1 q2 / (eps_ss d)
    lb = O.bjerrum(p["temperature"])
    assert got["coulomb"] == pytest.approx(lb * charges[0] * charges[1] / (p["eps_ss"] * d),
                                           rel=1e-12)


def test_pmf_definition_bookkeeping():
    from paper_2208_05524_gb300 import pmf, vesis
    s = _pair(8.0, (1.0, -1.0))
    S, S1, S2 = (vesis.System(x) for x in (s, synth.subset(s, [0]), synth.subset(s, [1])))
    G = S.G
    bufs = []
    for _ in range(3):
        bufs += [torch.empty(G, dtype=torch.float32, device="cuda"),
                 torch.empty(3 * G, dtype=torch.float32, device="cuda")]
    chis = [torch.empty(G, dtype=torch.uint8, device="cuda") for _ in range(3)]
    rows = pmf.two_atom_curve(S, S1, S2, *chis, bufs, [5.0, 8.0], "tight")
    for r in rows:
        assert r["total"] == pytest.approx(r["geom"] + r["vdw"] + r["elec"] + r["far"])
    # the atoms alone carry no pair terms, so the cross Coulomb is the pair's
    assert S1.ss_terms()["coulomb"] == 0.0 and S2.ss_terms()["lj"] == 0.0
