"""GPU parity of the literal serial flipping (Sec. 3.1, Steps 2.1-2.2).

vesis_blsm_heap against the oracle's min-heap (or_blsm_heap) from the same
labels and FP32 U: the same number of flips, the same FP64 sum of their dE
(summed in flip order on both sides, so bit for bit) and the same labels.
"""
import numpy as np
import pytest

import oracle as O
from paper_2208_05524_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _vs():
    from paper_2208_05524_gb300 import vesis
    return vesis


def _dev(a, dtype):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda").to(dtype).contiguous()


def _blob(n, seed):
    rng = np.random.default_rng(seed)
    idx = np.indices(n).reshape(3, -1).T.astype(np.float64)
    chi = np.zeros(int(np.prod(n)), np.uint8)
    for _ in range(6):
        c = rng.uniform(0.25, 0.75, 3) * np.array(n)
        r = rng.uniform(0.1, 0.3) * min(n)
        chi |= (np.linalg.norm(idx - c, axis=1) < r).astype(np.uint8)
    return chi.reshape(n)


def _case(case):
    h = 0.3
    n = {"tiny": (3, 2, 5), "blob": (30, 28, 26), "ragged": (45, 17, 50)}.get(case, (20, 18, 24))
    s = synth.single_ion(n=8, h=h)
    s["n"] = np.array(n)
    s["origin"] = -0.5 * np.array(n) * h
    kw = {}
    if case == "r2":
        kw = dict(trunc_r=2, gauss_sigma=h)
    elif case == "r8":
        kw = dict(trunc_r=8, gauss_sigma=2.0 * h)
    elif case == "sin2":
        kw = dict(kernel="sin2", sin2_lambda=2.0)
    if case == "all_solvent":
        chi0 = np.zeros(n, np.uint8)
    elif case == "all_solute":
        chi0 = np.ones(n, np.uint8)
    elif case in ("tiny", "random"):
        chi0 = synth.random_labels(n, seed=31)
    else:
        chi0 = _blob(n, 9 if case != "ragged" else 2)
    U32 = (synth.random_field(n, seed=23, scale=0.05) - 0.02).astype(np.float32)
    return s, kw, chi0, U32


@pytest.mark.parametrize("case", ["blob", "ragged", "r2", "r8", "sin2", "tiny", "random",
                                  "all_solvent", "all_solute"])
def test_heap_bit_exact(case):
    vs = _vs()
    s, kw, chi0, U32 = _case(case)
    p = O.params(**kw)
    sc = O.surface_constants(s, p)
    ref = chi0.copy()
    ro = O.blsm_heap(ref, U32.astype(np.float64), sc)
    S = vs.System(s, **kw)
    chi = _dev(chi0.reshape(-1), torch.uint8)
    r = S.blsm_heap(chi, _dev(U32.reshape(-1), torch.float32), terms=False)
    if case == "all_solvent":
        assert ro["flips"] == 0
    elif case not in ("all_solute",):
        assert ro["flips"] > 0
    assert r["status"] == 0
    assert r["flips"] == ro["flips"]
    assert r["dE_sum"] == ro["dE_sum"]
    assert np.array_equal(chi.cpu().numpy(), ref.reshape(-1))


def test_heap_cap_and_energy_drop():
    vs = _vs()
    s, kw, chi0, U32 = _case("blob")
    p = O.params()
    sc = O.surface_constants(s, p)
    full = O.blsm_heap(chi0.copy(), U32.astype(np.float64), sc)
    cap = max(1, full["flips"] // 3)
    ref = chi0.copy()
    ro = O.blsm_heap(ref, U32.astype(np.float64), sc, max_flips=cap)
    S = vs.System(s)
    chi = _dev(chi0.reshape(-1), torch.uint8)
    U = _dev(U32.reshape(-1), torch.float32)
    T0 = S.energy_terms(chi, U)
    r = S.blsm_heap(chi, U, max_flips=cap)
    assert r["status"] == 1 and r["flips"] == cap == ro["flips"]
    assert r["dE_sum"] == ro["dE_sum"]
    assert np.array_equal(chi.cpu().numpy(), ref.reshape(-1))
    # the energy falls by exactly the flipped cells' dE (up to the rounding
    # of the two totals)
    assert r["terms"]["total"] - T0["total"] == pytest.approx(r["dE_sum"], rel=1e-9, abs=1e-9)
    # continuing from the capped state ends where the uncapped run ends
    r2 = S.blsm_heap(chi, U, terms=False)
    assert r2["flips"] == full["flips"] - cap
    chi_full = _dev(chi0.reshape(-1), torch.uint8)
    S.blsm_heap(chi_full, U, terms=False)
    assert torch.equal(chi, chi_full)


def test_heap_single_ion_full_size():
    """64^3 single ion from the 7 A sphere: the heap's flips and labels
    equal the oracle's, and on this problem the heap and the parallel rule
    reach the same state."""
    vs = _vs()
    s = synth.single_ion()
    p = O.params()
    Uo, _, _ = O.fields(s, p)
    U32 = Uo.astype(np.float32)
    sc = O.surface_constants(s, p)
    chi0 = O.init_labels(s)
    ref = chi0.copy()
    ro = O.blsm_heap(ref, U32.astype(np.float64), sc)
    S = vs.System(s)
    chi = _dev(chi0.reshape(-1), torch.uint8)
    U = _dev(U32.reshape(-1), torch.float32)
    r = S.blsm_heap(chi, U, terms=False)
    assert r["flips"] == ro["flips"] > 1000
    assert r["dE_sum"] == ro["dE_sum"]
    assert np.array_equal(chi.cpu().numpy(), ref.reshape(-1))
    chi_p = _dev(chi0.reshape(-1), torch.uint8)
    S.blsm_relax(chi_p, U, terms=False)
    assert torch.equal(chi_p, chi)
