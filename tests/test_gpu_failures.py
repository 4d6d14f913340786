"""Failure paths of the C ABI on the GPU, made without any GPU fault.

* The flip sweep's grid barrier is bounded (vesis_set_wait_limit): with a
  limit of 0 polls every block that finds the barrier still open gives up,
  the sweep returns VESIS_E_CUDA, and the same system then relaxes the same
  labels to exactly the state of an undisturbed run.
* Non-finite positions are refused with VESIS_E_NAN before anything is
  launched; an atom outside the box is refused with VESIS_E_OUT_OF_BOX
  (at set-up and when positions are replaced).
* The cap on consecutive shrinks of M (Step 3.4 loops back to Step 3.3;
  the cap is this library's reading) ends vesis_relax with
  VESIS_W_NOT_CONVERGED, stop reason 3, the positions of the last accepted
  iterate, and the same trial count and M as the oracle's relaxation.
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


def _cluster():
    return synth.random_cluster(24, 40, 0.5, seed=1, net_charge=1.0)


def _start(S):
    U = torch.empty(S.G, dtype=torch.float32, device="cuda")
    E = torch.empty(3 * S.G, dtype=torch.float32, device="cuda")
    S.energy_field(U, E)
    chi0 = torch.empty(S.G, dtype=torch.uint8, device="cuda")
    S.init_labels(chi0, "tight")
    return U, E, chi0


def _dev(a, dtype):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda").to(dtype).contiguous()


def test_sweep_barrier_timeout_returns_error_and_the_system_recovers():
    vs = _vs()
    s = _cluster()
    S = vs.System(s)
    # the oracle's tight labels and its energy density rounded to FP32 feed
    # both sides, so that the sweep alone is compared
    p = O.params()
    sc = O.surface_constants(s, p)
    chi_o = O.init_labels(s)
    Uo = O.fields(s, p)[0].astype(np.float32)
    chi0 = _dev(chi_o.reshape(-1), torch.uint8)
    U = _dev(Uo.reshape(-1), torch.float32)
    chi_ok = chi0.clone()
    ok = S.blsm_relax(chi_ok, U)
    assert ok["flips"] > 0
    for attempt in range(3):
        S.set_wait_limit(0)
        chi = chi0.clone()
        try:
            S.blsm_relax(chi, U)
        except vs.VesisError as e:
            assert e.code == -2 and "timed out" in str(e)
            break
    else:
        pytest.fail("a sweep with a wait limit of 0 polls never timed out")
    # the same system, the default limit, fresh labels: the undisturbed result
    S.set_wait_limit()
    chi = chi0.clone()
    again = S.blsm_relax(chi, U)
    assert torch.equal(chi, chi_ok)
    assert (again["rounds"], again["flips"]) == (ok["rounds"], ok["flips"])
    assert again["dE_sum"] == ok["dE_sum"]
    # and against the oracle's parallel rule from the same FP32 U
    ref = chi_o.copy()
    ro = O.blsm_parallel(ref, Uo.astype(np.float64), sc)
    assert np.array_equal(chi.cpu().numpy(), ref.reshape(-1))
    assert again["rounds"] == ro["rounds"]
    # the same failure inside a full relaxation, then a normal one
    xyz = np.ascontiguousarray(s["xyz"])
    S.set_wait_limit(0)
    with pytest.raises(vs.VesisError) as e:
        S.relax(chi0.clone(), xyz, max_outer=2)
    assert e.value.code == -2
    S.set_wait_limit()
    chi_a = chi0.clone()
    ra = S.relax(chi_a, xyz, max_outer=2)
    T = vs.System(s)
    chi_b = chi0.clone()
    rb = T.relax(chi_b, xyz, max_outer=2)
    assert torch.equal(chi_a, chi_b) and np.array_equal(ra["xyz"], rb["xyz"])
    assert ra["G"] == rb["G"] and ra["gd_trials"] == rb["gd_trials"]
    with pytest.raises(vs.VesisError):
        S.set_wait_limit(-1)
    S.close()
    T.close()


def test_nonfinite_positions_are_refused():
    vs = _vs()
    s = _cluster()
    S = vs.System(s)
    U, E, chi0 = _start(S)
    g0 = S.atom_forces(chi0)
    bad = np.array(s["xyz"], np.float64)
    for v in (np.nan, np.inf, -np.inf):
        bad[3, 1] = v
        for call in (lambda: S.set_positions(bad),
                     lambda: S.relax(chi0.clone(), bad, max_outer=1),
                     lambda: S.atom_forces(chi0, xyz=bad),
                     lambda: S.energy_field(U, E, xyz=bad)):
            with pytest.raises(vs.VesisError) as e:
                call()
            assert e.value.code == -3 and "non-finite" in str(e.value)
    # nothing was replaced: the gradient at the stored positions is unchanged
    assert np.array_equal(S.atom_forces(chi0), g0)
    sd = dict(s)
    sd["xyz"] = bad
    with pytest.raises(vs.VesisError) as e:
        vs.System(sd)
    assert e.value.code == -3
    S.close()


def test_atoms_outside_the_box_are_refused():
    vs = _vs()
    s = _cluster()
    S = vs.System(s)
    U, E, chi0 = _start(S)
    g0 = S.atom_forces(chi0)
    hi = np.asarray(s["origin"], np.float64) + np.asarray(s["n"]) * s["h"]
    bad = np.array(s["xyz"], np.float64)
    bad[5, 2] = hi[2] + 0.3
    with pytest.raises(vs.VesisError) as e:
        S.set_positions(bad)
    assert e.value.code == -4 and "outside the box" in str(e.value)
    with pytest.raises(vs.VesisError) as e:
        S.relax(chi0.clone(), bad, max_outer=1)
    assert e.value.code == -4
    # valid positions again: the system answers as before
    S.set_positions(s["xyz"])
    assert np.array_equal(S.atom_forces(chi0), g0)
    sd = dict(s)
    sd["xyz"] = bad
    with pytest.raises(vs.VesisError) as e:
        vs.System(sd)
    assert e.value.code == -4
    S.close()


@pytest.mark.parametrize("retries", [0, 3])
def test_shrink_cap_ends_the_relaxation_as_not_converged(retries):
    """M0 = 1e6 sends the first trial atoms far outside the box: every trial
    is rejected (reading: a trial leaving the box counts as an energy
    increase) and M shrinks by alpha each time, until the cap."""
    vs = _vs()
    s = _cluster()
    S = vs.System(s)
    _, _, chi0 = _start(S)
    xyz = np.ascontiguousarray(s["xyz"])
    chi = chi0.clone()
    r = S.relax(chi, xyz, max_outer=5, M0=1e6, max_gd_retries=retries)
    assert r["status"] == 2 and r["stop_reason"] == 3
    assert r["iterations"] == 0 and r["gd_trials"] == retries + 1
    assert np.array_equal(r["xyz"], xyz)
    assert r["M"] == pytest.approx(1e6 * (1 / np.sqrt(2)) ** (retries + 1), rel=1e-12)
    p = O.params()
    ro = O.relax(s, p, O.relax_opts(max_outer=5, M0=1e6, max_gd_retries=retries))
    assert ro["status"] == 2 and ro["iters"] == 0
    assert np.array_equal(ro["xyz"], xyz)
    S.close()
