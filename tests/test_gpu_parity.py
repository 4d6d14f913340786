"""CUDA path vs the FP64 CPU oracle, through the C ABI (needs a GPU).

Tolerances (stated once, used below):
  * fields U, E: FP32 pair sums vs FP64: |gpu - oracle| <= 1e-4 |oracle|
    + 1e-4 max|oracle| (relative 1e-4 per cell with a floor).
  * W (kernel convolution), flip energies, candidate masks, labels after a
    sweep from the same FP32 U: bit-exact.
  * energy totals: relative 1e-6 (FP64 sums of FP32 cell values).
  * gradients: |gpu - oracle| <= 1e-4 |oracle| + 1e-4 max|oracle|.
  * converged positions: 1e-3 A.
"""
import math

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


def _fields_gpu(S, n):
    G = int(np.prod(n))
    U = torch.empty(G, dtype=torch.float32, device="cuda")
    E = torch.empty(3 * G, dtype=torch.float32, device="cuda")
    return U, E


def _close(gpu, ref, rel=1e-4):
    ref = np.asarray(ref, np.float64)
    gpu = np.asarray(gpu, np.float64)
    tol = rel * np.abs(ref) + rel * np.abs(ref).max()
    bad = np.abs(gpu - ref) > tol
    return int(bad.sum()), float(np.max(np.abs(gpu - ref) / (tol + 1e-300)))


# ------------------------------------------------------------------ fields

@pytest.mark.parametrize("n,h,natoms,seed", [((40, 36, 28), 0.5, 30, 1),
                                             ((27, 33, 29), 1.0, 300, 2)])
def test_energy_field_matches_oracle(n, h, natoms, seed):
    vs = _vs()
    s = synth.random_cluster(natoms, 8, h, seed=seed, net_charge=-1.0)
    s["n"] = np.array(n)
    s["origin"] = -0.5 * np.array(n) * h
    p = O.params()
    S = vs.System(s)
    U, E = _fields_gpu(S, n)
    S.energy_field(U, E)
    Uo, _, Eo = O.fields(s, p)
    nb, worst = _close(U.cpu().numpy(), Uo.reshape(-1))
    assert nb == 0, worst
    Eg = E.cpu().numpy().reshape(3, -1).T
    nb, worst = _close(Eg, Eo.reshape(-1, 3))
    assert nb == 0, worst


def test_energy_field_single_ion_and_terms():
    vs = _vs()
    s = synth.single_ion()
    p = O.params()
    S = vs.System(s)
    n = tuple(int(v) for v in s["n"])
    U, E = _fields_gpu(S, n)
    chi0 = O.init_labels(s)
    chi = _dev(chi0.reshape(-1), torch.uint8)
    T = S.energy_field(U, E, chi=chi, terms=True)
    Uo, _, Eo = O.fields(s, p)
    nb, worst = _close(U.cpu().numpy(), Uo.reshape(-1))
    assert nb == 0, worst
    To = O.energy_terms(s, p, chi0, U=Uo, E=Eo)
    for k in ("surf", "far", "ss"):
        assert T[k] == pytest.approx(To[k], rel=1e-6, abs=1e-9)
    assert T["vdw"] + T["cfa"] == pytest.approx(To["vol"], rel=1e-6)
    assert T["total"] == pytest.approx(To["total"], rel=1e-6)


def test_init_labels_match_oracle():
    vs = _vs()
    s = synth.random_cluster(60, 8, 0.45, seed=3)
    s["n"] = np.array([48, 44, 40])
    s["origin"] = -0.5 * s["n"] * 0.45
    S = vs.System(s)
    G = int(np.prod(s["n"]))
    chi = torch.empty(G, dtype=torch.uint8, device="cuda")
    S.init_labels(chi, "tight")
    ref = O.init_labels(s).reshape(-1)
    got = chi.cpu().numpy()
    diff = np.nonzero(got != ref)[0]
    if len(diff):
        _, phi = O.init_labels_at(s, diff)
        assert np.all(np.abs(phi) < 1e-4)
    s2 = synth.single_ion(n=40, h=0.4, r_init=5.3)
    S2 = vs.System(s2)
    c2 = torch.empty(40 ** 3, dtype=torch.uint8, device="cuda")
    S2.init_labels(c2, "sphere", radius=5.3)
    assert np.array_equal(c2.cpu().numpy(), O.init_labels(s2).reshape(-1))


# --------------------------------------------------------------- surface

@pytest.mark.parametrize("n", [(37, 29, 41), (8, 9, 10), (1, 5, 64)])
def test_surface_weights_exact(n):
    vs = _vs()
    s = synth.single_ion(n=8, h=0.3)
    s["n"] = np.array(n)
    s["origin"] = -0.5 * np.array(n) * 0.3
    S = vs.System(s)
    chi0 = synth.random_labels(n, seed=sum(n), p=0.4)
    chi = _dev(chi0.reshape(-1), torch.uint8)
    W = torch.empty(int(np.prod(n)), dtype=torch.int32, device="cuda")
    S.surface_weights(chi, W)
    sc = O.surface_constants(s, O.params())
    assert np.array_equal(W.cpu().numpy().astype(np.int64), O.conv(chi0, sc["q"]).reshape(-1))


def test_flip_energies_bit_exact():
    vs = _vs()
    n = (33, 30, 27)
    s = synth.single_ion(n=8, h=0.35)
    s["n"] = np.array(n)
    s["origin"] = -0.5 * np.array(n) * 0.35
    S = vs.System(s)
    chi0 = synth.random_labels(n, seed=4, p=0.5)
    U32 = synth.random_field(n, seed=5, scale=0.3)
    chi = _dev(chi0.reshape(-1), torch.uint8)
    U = _dev(U32.reshape(-1), torch.float32)
    G = int(np.prod(n))
    dE = torch.empty(G, dtype=torch.float64, device="cuda")
    cand = torch.empty(G, dtype=torch.uint8, device="cuda")
    S.flip_energies(chi, U, dE, cand)
    sc = O.surface_constants(s, O.params())
    dEo, co = O.delta_e(chi0, U32.astype(np.float64), sc)
    assert np.array_equal(cand.cpu().numpy(), co.reshape(-1))
    assert np.array_equal(dE.cpu().numpy(), dEo.reshape(-1))


def _check_stamp_modes(S, chi0, U, ref, ro, **kw):
    """The sweep decides only stamped tiles (mode 1), every leader tile
    (mode 0) or chooses by the leader count (-1): the rounds, flips and
    labels of every mode are the oracle's."""
    for mode in (1, 0, -1):
        S.set_sweep_stamps(mode)
        chi = _dev(chi0.reshape(-1), torch.uint8)
        r = S.blsm_relax(chi, U, terms=False, **kw)
        assert (r["rounds"], r["flips"]) == (ro["rounds"], ro["flips"]), mode
        assert np.array_equal(chi.cpu().numpy(), ref.reshape(-1)), mode
    S.set_sweep_stamps(-1)


def _blob(n, seed):
    """Seeded label field with structure: a union of random balls."""
    rng = np.random.default_rng(seed)
    idx = np.indices(n).reshape(3, -1).T.astype(np.float64)
    chi = np.zeros(int(np.prod(n)), np.uint8)
    for _ in range(6):
        c = rng.uniform(0.25, 0.75, 3) * np.array(n)
        r = rng.uniform(0.1, 0.3) * min(n)
        chi |= (np.linalg.norm(idx - c, axis=1) < r).astype(np.uint8)
    return chi.reshape(n)


@pytest.mark.parametrize("n,seed", [((30, 28, 26), 1), ((45, 17, 50), 2)])
def test_blsm_rounds_bit_exact(n, seed):
    vs = _vs()
    s = synth.single_ion(n=8, h=0.3)
    s["n"] = np.array(n)
    s["origin"] = -0.5 * np.array(n) * 0.3
    S = vs.System(s)
    chi0 = _blob(n, seed)
    U32 = (synth.random_field(n, seed=seed + 10, scale=0.05) - 0.02).astype(np.float32)
    sc = O.surface_constants(s, O.params())
    ref = chi0.copy()
    ro = O.blsm_parallel(ref, U32.astype(np.float64), sc, record_rounds=True)
    chi = _dev(chi0.reshape(-1), torch.uint8)
    U = _dev(U32.reshape(-1), torch.float32)
    r = S.blsm_relax(chi, U, terms=False)
    assert r["rounds"] == ro["rounds"]
    assert r["flips"] == ro["flips"]
    assert r["dE_sum"] == pytest.approx(ro["dE_sum"], rel=1e-12, abs=1e-12)
    assert np.array_equal(chi.cpu().numpy(), ref.reshape(-1))
    _check_stamp_modes(S, chi0, U, ref, ro)
    # the same after a capped number of rounds
    chi = _dev(chi0.reshape(-1), torch.uint8)
    k = max(1, ro["rounds"] // 3)
    r = S.blsm_relax(chi, U, max_rounds=k, terms=False)
    ref2 = chi0.copy()
    O.blsm_parallel(ref2, U32.astype(np.float64), sc, max_rounds=k)
    assert r["rounds"] == k
    assert np.array_equal(chi.cpu().numpy(), ref2.reshape(-1))
    for mode in (1, 0):      # the cap with the decide stamps forced on and off
        S.set_sweep_stamps(mode)
        chi = _dev(chi0.reshape(-1), torch.uint8)
        r = S.blsm_relax(chi, U, max_rounds=k, terms=False)
        assert r["rounds"] == k and np.array_equal(chi.cpu().numpy(), ref2.reshape(-1)), mode
    S.set_sweep_stamps(-1)


def test_blsm_single_ion_full_size():
    """64^3 single ion: identical labels and rounds from the same FP32 U;
    the relaxed radius and energy meet the closed-form sphere minimum."""
    vs = _vs()
    s = synth.single_ion()
    p = O.params()
    n = tuple(int(v) for v in s["n"])
    Uo, _, Eo = O.fields(s, p)
    U32 = Uo.astype(np.float32)
    sc = O.surface_constants(s, p)
    chi0 = O.init_labels(s)
    ref = chi0.copy()
    ro = O.blsm_parallel(ref, U32.astype(np.float64), sc)
    S = vs.System(s)
    chi = _dev(chi0.reshape(-1), torch.uint8)
    r = S.blsm_relax(chi, _dev(U32.reshape(-1), torch.float32), terms=False)
    assert r["rounds"] == ro["rounds"] and r["flips"] == ro["flips"]
    assert np.array_equal(chi.cpu().numpy(), ref.reshape(-1))
    _check_stamp_modes(S, chi0, _dev(U32.reshape(-1), torch.float32), ref, ro)
    # GPU's own FP32 fields: labels may differ only where the oracle's
    # |dE| is below 1e-9 kBT; energy at the closed-form minimum
    U, E = _fields_gpu(S, n)
    chi = _dev(chi0.reshape(-1), torch.uint8)
    S.energy_field(U, E)
    r = S.blsm_relax(chi, U, E)
    got = chi.cpu().numpy().reshape(n)
    mism = np.argwhere(got != ref)
    if len(mism):
        dEo, _ = O.delta_e(ref, Uo, sc)
        assert np.all(np.abs(dEo[tuple(mism.T)]) < 1e-9), len(mism)
    Rs, Gs = O.sphere_minimum(3.5, s["eps_sw"][0], 1.0, p)
    R_eq = (3 * got.sum() * sc["h3"] / (4 * math.pi)) ** (1 / 3)
    assert abs(R_eq - Rs) < s["h"]
    assert r["terms"]["total"] == pytest.approx(Gs, rel=0.01)
    To = O.energy_terms(s, p, ref, U=Uo, E=Eo)
    assert r["terms"]["total"] == pytest.approx(To["total"], rel=1e-6)


# ---------------------------------------------------------------- forces

@pytest.mark.parametrize("natoms,n,h", [(7, (30, 26, 34), 0.5), (250, (40, 40, 40), 0.7)])
def test_atom_forces_match_oracle(natoms, n, h):
    vs = _vs()
    s = synth.random_cluster(natoms, 8, h, seed=natoms, net_charge=1.0)
    s["n"] = np.array(n)
    s["origin"] = -0.5 * np.array(n) * h
    p = O.params()
    chi0 = O.init_labels(s)
    S = vs.System(s)
    chi = _dev(chi0.reshape(-1), torch.uint8)
    g, e = S.atom_forces(chi, energy=True)
    go = O.gradient(s, p, chi0)
    nb, worst = _close(g, go)
    assert nb == 0, worst
    To = O.energy_terms(s, p, chi0)
    assert e == pytest.approx(To["total"], rel=1e-6)


def _pencil_case(n, natoms, seed, h=0.5):
    """Atoms on a jittered lattice of about 5 A that fills the box (no bonds,
    so the solute-solute terms stay moderate) and labels with half of the
    cells farther than 2.5 A from every atom solvent, at random, so that
    solvent runs are broken inside every z-pencil."""
    rng = np.random.default_rng(seed)
    L = np.asarray(n, np.float64) * h
    s = synth.random_cluster(natoms, 8, h, seed=seed, net_charge=1.0)
    m = np.maximum(np.floor(L / 5.0), 1).astype(int)
    cells = np.stack(np.meshgrid(*[np.arange(k) for k in m], indexing="ij"), -1).reshape(-1, 3)
    assert len(cells) >= natoms
    pick = cells[rng.permutation(len(cells))[:natoms]]
    step = L / m
    jitter = (rng.random((natoms, 3)) - 0.5) * 0.3 * step
    s["xyz"] = -0.5 * L + (pick + 0.5) * step + jitter
    s["bonds"] = np.zeros((0, 2), np.int32)
    s["bond_k"] = np.zeros(0)
    s["bond_r0"] = np.zeros(0)
    s["n"] = np.array(n)
    s["origin"] = -0.5 * L
    axes = [-0.5 * L[c] + (np.arange(n[c]) + 0.5) * h for c in range(3)]
    X = np.stack(np.meshgrid(*axes, indexing="ij"), -1).reshape(-1, 3)
    from scipy.spatial import cKDTree
    near = cKDTree(s["xyz"]).query(X, distance_upper_bound=2.5)[0] < 2.5
    solvent = ~near & (rng.random(len(X)) < 0.5)
    return s, (~solvent).astype(np.uint8).reshape(tuple(n))


@pytest.mark.parametrize("n,natoms", [((40, 34, 1), 12),      # one cell per pencil, 4 groups
                                      ((340, 320, 3), 1000),  # short pencils, 1 group, 2 tiles
                                      ((240, 230, 3), 520),   # short pencils, 4 groups
                                      ((4, 5, 300), 28)])     # pencils cut by the stages
def test_atom_forces_by_pencil_match_oracle(n, natoms):
    """The gradient kernel takes the solvent cells of each 256-cell stage by
    z-pencil (dx, dy once per pencil and atom, the pencil's x/y terms from
    its summed pair factor).  Gradient (Eq. GradientG) against the oracle's
    on grids that stress that split: nz = 1, nz = 3 with two atom tiles, and
    nz = 300 (a pencil spans two stages), with one and with four groups of
    threads sharing the staged cells; random labels, so the solvent
    cells of a pencil are not contiguous.  The far field is off on both
    sides: these boxes are thinner than an atom, and the solvent it places
    just outside them would dwarf the grid's terms being tested."""
    vs = _vs()
    s, chi0 = _pencil_case(n, natoms, seed=natoms)
    p = O.params(far_field=False)
    S = vs.System(s, far_field=0)
    chi = _dev(chi0.reshape(-1), torch.uint8)
    g = S.atom_forces(chi)
    go = O.gradient(s, p, chi0)
    nb, worst = _close(g, go)
    assert nb == 0, worst
    S.set_tiles(8, 2)     # the other atom tile: bit-identical
    assert np.array_equal(S.atom_forces(chi), g)


# ------------------------------------------------------------ relaxation

def test_solute_solute_pair_terms_match_oracle():
    """G_ss's bonds, LJ and Coulomb (Eq. Gss) on a charged, bonded 300-atom
    solute: the GPU evaluates the pair terms in double-float arithmetic and
    must agree with the FP64 oracle to near FP64 accuracy.  With rho_w = 0
    and eps_w = eps_m the solvation forces vanish, so the gradient the
    library returns is G_ss's alone."""
    vs = _vs()
    s = synth.protein_like(n_atoms=300, n=64, h=0.5, seed=5)
    kw = dict(rho_w=0.0, eps_w=1.0)
    S = vs.System(s, **kw)
    t = S.ss_terms()
    e, g = O.ss_terms(s, O.params(**kw))
    assert t["bonds"] == pytest.approx(e[0], rel=1e-12)
    assert t["lj"] == pytest.approx(e[1], rel=1e-12)
    assert t["coulomb"] == pytest.approx(e[2], rel=1e-12)
    chi = _dev(O.init_labels(s).reshape(-1), torch.uint8)
    got = S.atom_forces(chi)
    assert np.allclose(got, g, rtol=1e-10, atol=1e-12 * np.abs(g).max())


def test_relax_two_atom_molecule_matches_oracle():
    vs = _vs()
    s = synth.two_atom_molecule(8.0, 7.0, n=32, h=0.5)
    p = O.params()
    ro = O.relax(s, p, O.relax_opts())
    S = vs.System(s)
    chi0 = O.init_labels(s)
    chi = _dev(chi0.reshape(-1), torch.uint8)
    r = S.relax(chi, s["xyz"])
    assert r["status"] == 0 and r["stop_reason"] == 1
    assert np.abs(r["xyz"] - ro["xyz"]).max() < 1e-3
    assert r["G"] == pytest.approx(ro["G"], rel=1e-4)
    x = np.sort(r["xyz"][:, 0])
    assert x[1] - x[0] == pytest.approx(8.0, abs=0.01)


def test_relax_charged_multi_atom_lock_step_matches_oracle():
    """A charged 48-atom protein-like solute (net -3 e) on 48^3 at h = 0.5 A,
    five outer iterations of Sec. 3.3 (Step 2 sweep, Step 3.1 gradient,
    Eq. moveatoms with Eq. adjustmml, the accept/shrink rule of Step 3.4)
    on the GPU and in the oracle, the oracle's fields stored in FP32 like
    the GPU's.  The two take the same accepted and rejected trials, flip
    rounds and flips, and end with the same M, the same labels, positions
    within 1e-3 A and G within 1e-6."""
    vs = _vs()
    s = synth.protein_like(n_atoms=48, n=48, h=0.5, seed=5)
    p = O.params()
    ro = O.relax(s, p, O.relax_opts(max_outer=5), fields_fp32=True)
    assert ro["iters"] == 5
    hist = ro["history"]
    assert any(h["retries"] > 0 for h in hist)        # rejected trials occur
    S = vs.System(s)
    S.set_history(8)
    chi0 = O.init_labels(s)
    chi = _dev(chi0.reshape(-1), torch.uint8)
    r = S.relax(chi, s["xyz"], max_outer=5)
    assert r["iterations"] == 5 and r["records"] == 5
    # iteration by iteration: the sweep, the step that set the mobility, the
    # trials, N_cnt, M and the energies before and after the step
    for a, b in zip(r["history"], hist):
        assert (a["k"], a["rounds"], a["flips"], a["trials"], a["ncnt"]) == \
            (b["k"], b["rounds"], b["flips"], b["retries"] + 1, b["ncnt"])
        assert a["M"] == b["M"]
        assert a["G"] == pytest.approx(b["G"], rel=1e-6)
        assert a["G_old"] == pytest.approx(b["G_old"], rel=1e-6)
        assert a["max_grad"] == pytest.approx(b["gmax"], rel=1e-4)
    assert r["gd_trials"] == sum(h["retries"] + 1 for h in hist)
    assert r["flip_rounds"] == sum(h["rounds"] for h in hist)
    assert r["flips"] == sum(h["flips"] for h in hist)
    assert r["M"] == hist[-1]["M"]
    mism = int((chi.cpu().numpy() != ro["chi"].reshape(-1)).sum())
    assert mism == 0, mism
    assert np.abs(r["xyz"] - ro["xyz"]).max() < 1e-3
    assert r["G"] == pytest.approx(ro["G"], rel=1e-6)


def test_relax_resumes_bit_identically_from_a_saved_state():
    """Checkpoint and resume: ten outer iterations of a charged solute in one
    call, against four iterations, the state saved (labels, positions,
    vesis_get_state), a new system loaded with it (vesis_set_state) and
    the relaxation continued to k = 10 (opts.resume): identical labels,
    positions, energy, M and counts."""
    vs = _vs()
    s = synth.protein_like(n_atoms=48, n=48, h=0.5, seed=5)
    chi0 = O.init_labels(s)
    A = vs.System(s)
    chi_a = _dev(chi0.reshape(-1), torch.uint8)
    ra = A.relax(chi_a, s["xyz"], max_outer=10)
    st_a = A.get_state()
    assert st_a["valid"] == 1 and st_a["k"] == ra["iterations"] == 10
    B = vs.System(s)
    chi_b = _dev(chi0.reshape(-1), torch.uint8)
    rb1 = B.relax(chi_b, s["xyz"], max_outer=4)
    saved = (chi_b.cpu().numpy().copy(), rb1["xyz"].copy(), B.get_state())
    assert saved[2]["k"] == 4
    B.close()
    C_ = vs.System(s)
    with pytest.raises(vs.VesisError):      # nothing to resume yet
        C_.relax(_dev(saved[0], torch.uint8), saved[1], max_outer=10, resume=1)
    C_.set_state(saved[2])
    chi_c = _dev(saved[0], torch.uint8)
    rb2 = C_.relax(chi_c, saved[1], max_outer=10, resume=1)
    assert rb2["iterations"] == 10
    assert torch.equal(chi_c, chi_a)
    assert np.array_equal(rb2["xyz"], ra["xyz"])
    assert rb2["G"] == ra["G"] and rb2["M"] == ra["M"]
    for key in ("gd_trials", "flip_rounds", "flips"):
        assert rb1[key] + rb2[key] == ra[key], key
    assert C_.get_state() == st_a
    with pytest.raises(vs.VesisError):
        C_.set_state(dict(st_a, M=-1.0))
    A.close()
    C_.close()


# --------------------------------------------------- full-size, sampled

def test_protein_like_full_size_sampled():
    """2,000-atom protein-like solute on the 256^3 grid (h = 0.4 A) in the
    launch configuration of the benchmark: fields at sampled cells against
    the oracle, exact W, tight labels at sampled cells, and the flip sweep's
    reported energy change against a from-scratch recomputation."""
    vs = _vs()
    s = synth.protein_like()
    p = O.params()
    n = tuple(int(v) for v in s["n"])
    G = int(np.prod(n))
    S = vs.System(s)
    U, E = _fields_gpu(S, n)
    chi = torch.empty(G, dtype=torch.uint8, device="cuda")
    S.init_labels(chi, "tight")
    T0 = S.energy_field(U, E, chi=chi, terms=True)
    rng = np.random.default_rng(0)
    cells = np.concatenate([rng.integers(0, G, 3000),
                            np.nonzero(chi.cpu().numpy())[0][::997]])
    pts = O.cell_positions(s, cells)
    Uo, _, Eo = O.point_fields(s, p, pts)
    Ug = U.cpu().numpy()[cells]
    # floor from the solvent cells of the sample
    chis = chi.cpu().numpy()[cells]
    floor = 1e-4 * np.abs(Uo[chis == 0]).max()
    assert np.all(np.abs(Ug - Uo) <= 1e-4 * np.abs(Uo) + floor)
    Eg = E.cpu().numpy().reshape(3, -1)[:, cells].T
    fl = 1e-4 * np.abs(Eo).max()
    assert np.all(np.abs(Eg - Eo) <= 1e-4 * np.abs(Eo) + fl)
    lab, phi = O.init_labels_at(s, cells)
    bad = lab != chis
    assert np.all(np.abs(phi[bad]) < 1e-4)
    W = torch.empty(G, dtype=torch.int32, device="cuda")
    S.surface_weights(chi, W)
    sc = O.surface_constants(s, p)
    assert np.array_equal(W.cpu().numpy().astype(np.int64),
                          O.conv(chi.cpu().numpy().reshape(n), sc["q"]).reshape(-1))
    r = S.blsm_relax(chi, U, E)
    assert r["status"] == 0 and r["rounds"] > 0
    assert r["terms"]["total"] - T0["total"] == pytest.approx(r["dE_sum"], rel=1e-6, abs=1e-6)


def test_blsm_small_kernel_radius_bit_exact():
    """r = 2 (bricks of edge 2 in the selection): identical rounds and labels."""
    vs = _vs()
    n = (26, 21, 23)
    h = 0.3
    s = synth.single_ion(n=8, h=h)
    s["n"] = np.array(n)
    s["origin"] = -0.5 * np.array(n) * h
    p = O.params(trunc_r=2, gauss_sigma=h)
    S = vs.System(s, trunc_r=2, gauss_sigma=h)
    chi0 = _blob(n, 7)
    U32 = (synth.random_field(n, seed=17, scale=0.05) - 0.02).astype(np.float32)
    sc = O.surface_constants(s, p)
    ref = chi0.copy()
    ro = O.blsm_parallel(ref, U32.astype(np.float64), sc)
    chi = _dev(chi0.reshape(-1), torch.uint8)
    r = S.blsm_relax(chi, _dev(U32.reshape(-1), torch.float32), terms=False)
    assert ro["rounds"] > 0
    assert r["rounds"] == ro["rounds"] and r["flips"] == ro["flips"]
    assert np.array_equal(chi.cpu().numpy(), ref.reshape(-1))
    _check_stamp_modes(S, chi0, _dev(U32.reshape(-1), torch.float32), ref, ro)


@pytest.mark.parametrize("case", ["all_solvent", "all_solute", "tiny", "random", "r1", "r8"])
def test_blsm_edge_cases_bit_exact(case):
    """Degenerate label fields, a grid smaller than one tile, a checkerboard-
    like random start (many candidates per tile), and the smallest and
    largest kernel radii (bricks of edge 2; the widest 6^3 brick
    neighbourhood): identical rounds, flips and labels."""
    vs = _vs()
    h = 0.3
    n = (3, 2, 5) if case == "tiny" else (20, 18, 24)
    s = synth.single_ion(n=8, h=h)
    s["n"] = np.array(n)
    s["origin"] = -0.5 * np.array(n) * h
    kw = {}
    if case == "r1":
        kw = dict(trunc_r=1, gauss_sigma=0.5 * h)
    elif case == "r8":
        kw = dict(trunc_r=8, gauss_sigma=2.0 * h)
    p = O.params(**kw)
    S = vs.System(s, **kw)
    if case == "all_solvent":
        chi0 = np.zeros(n, np.uint8)
    elif case == "all_solute":
        chi0 = np.ones(n, np.uint8)
    elif case in ("tiny", "random"):
        chi0 = synth.random_labels(n, seed=31)
    else:
        chi0 = _blob(n, 9)
    U32 = (synth.random_field(n, seed=23, scale=0.05) - 0.02).astype(np.float32)
    sc = O.surface_constants(s, p)
    ref = chi0.copy()
    ro = O.blsm_parallel(ref, U32.astype(np.float64), sc)
    chi = _dev(chi0.reshape(-1), torch.uint8)
    r = S.blsm_relax(chi, _dev(U32.reshape(-1), torch.float32), terms=False)
    if case == "all_solvent":
        assert ro["rounds"] == 0
    assert r["rounds"] == ro["rounds"] and r["flips"] == ro["flips"]
    assert r["dE_sum"] == pytest.approx(ro["dE_sum"], rel=1e-12, abs=1e-12)
    assert np.array_equal(chi.cpu().numpy(), ref.reshape(-1))
    _check_stamp_modes(S, chi0, _dev(U32.reshape(-1), torch.float32), ref, ro)


def test_two_domain_complex_full_size_sampled():
    """20,000-atom two-domain complex on the 384^3 grid (h = 0.4 A): fields
    at sampled cells against the oracle, exact W of the tight labels, the
    sweep's energy change against a from-scratch recomputation, and no flip
    left that lowers the energy (every candidate's dE >= 0 afterwards)."""
    vs = _vs()
    s = synth.two_domain_complex()
    p = O.params()
    n = tuple(int(v) for v in s["n"])
    G = int(np.prod(n))
    S = vs.System(s)
    U, E = _fields_gpu(S, n)
    chi = torch.empty(G, dtype=torch.uint8, device="cuda")
    S.init_labels(chi, "tight")
    T0 = S.energy_field(U, E, chi=chi, terms=True)
    rng = np.random.default_rng(5)
    chin = chi.cpu().numpy()
    cells = np.concatenate([rng.integers(0, G, 2000), np.nonzero(chin)[0][::4999]])
    pts = O.cell_positions(s, cells)
    Uo, ljo, Eo = O.point_fields(s, p, pts)
    chis = chin[cells]
    floor = 1e-4 * np.abs(Uo[chis == 0]).max()
    # U = rho_w sum U_LJ + C |E|^2: where the two parts nearly cancel, the
    # FP32 result is good to 1e-4 of the parts, not of their small sum
    parts = np.abs(p["rho_w"] * ljo) + np.abs(O.cfa_prefactor(p) * (Eo * Eo).sum(1))
    assert np.all(np.abs(U.cpu().numpy()[cells] - Uo) <= 1e-4 * parts + floor)
    Eg = E.cpu().numpy().reshape(3, -1)[:, cells].T
    assert np.all(np.abs(Eg - Eo) <= 1e-4 * np.abs(Eo) + 1e-4 * np.abs(Eo).max())
    W = torch.empty(G, dtype=torch.int32, device="cuda")
    S.surface_weights(chi, W)
    sc = O.surface_constants(s, p)
    assert np.array_equal(W.cpu().numpy().astype(np.int64),
                          O.conv(chin.reshape(n), sc["q"]).reshape(-1))
    del W
    chi0 = chi.clone()
    r = S.blsm_relax(chi, U, E)
    assert r["status"] == 0 and r["rounds"] > 0
    assert r["terms"]["total"] - T0["total"] == pytest.approx(r["dE_sum"], rel=1e-6, abs=1e-6)
    dE = torch.empty(G, dtype=torch.float64, device="cuda")
    cand = torch.empty(G, dtype=torch.uint8, device="cuda")
    S.flip_energies(chi, U, dE, cand)
    m = cand.bool()
    assert int(m.sum()) > 0
    assert float(dE[m].min()) >= 0.0
    del dE, cand
    # the same rounds and labels with every leader tile decided every round
    # (these blocks own 728 tiles each: the multi-pass tile lists), and
    # through the multi-system kernel's global tile numbering
    S.set_sweep_stamps(0)
    c2 = chi0.clone()
    r2 = S.blsm_relax(c2, U, E, terms=False)
    S.set_sweep_stamps(-1)
    assert (r2["rounds"], r2["flips"]) == (r["rounds"], r["flips"]) and torch.equal(c2, chi)
    c3 = chi0.clone()
    r3 = vs.blsm_relax_batch([S], [c3], [U])[0]
    assert (r3["rounds"], r3["flips"]) == (r["rounds"], r["flips"]) and torch.equal(c3, chi)
    del c2, c3
    # one outer iteration with the sweep on 19 blocks (more than 2,048 tiles
    # per block: several listing passes per phase) against the default grid
    xyz = np.ascontiguousarray(s["xyz"])
    a = chi0.clone()
    ra = S.relax(a, xyz, max_outer=1)
    b = chi0.clone()
    rb = vs.relax_batch([S], [b], [xyz], threads=1, sweep_slots=8, max_outer=1)[0]
    assert (rb["flip_rounds"], rb["flips"]) == (ra["flip_rounds"], ra["flips"])
    assert torch.equal(a, b) and rb["G"] == ra["G"]
    S.close()


@pytest.mark.parametrize("n", [(20, 18, 24), (21, 17, 13)])
def test_sin2_kernel_bit_exact(n):
    """The paper's sin^2 kernel (lambda = 2, h = 0.25 A: a ball of radius 4
    cells): W, flip energies, candidates, sweep rounds, flips and labels, and
    the surface energy agree bit for bit with the oracle (nz = 24 takes the
    8-cell stencil kernel, nz = 13 the per-cell one)."""
    vs = _vs()
    h = 0.25
    s = synth.single_ion(n=8, h=h)
    s["n"] = np.array(n)
    s["origin"] = -0.5 * np.array(n) * h
    p = O.params(kernel="sin2", sin2_lambda=2.0)
    sc = O.surface_constants(s, p)
    S = vs.System(s, kernel="sin2", sin2_lambda=2.0)
    G = int(np.prod(n))
    chi0 = _blob(n, 13)
    chi = _dev(chi0.reshape(-1), torch.uint8)
    W = torch.empty(G, dtype=torch.int32, device="cuda")
    S.surface_weights(chi, W)
    assert np.array_equal(W.cpu().numpy().astype(np.int64),
                          O.conv3(chi0, sc["k3"]).reshape(-1))
    U32 = (synth.random_field(n, seed=29, scale=0.05) - 0.02).astype(np.float32)
    U = _dev(U32.reshape(-1), torch.float32)
    dE = torch.empty(G, dtype=torch.float64, device="cuda")
    cand = torch.empty(G, dtype=torch.uint8, device="cuda")
    S.flip_energies(chi, U, dE, cand)
    dEo, co = O.delta_e(chi0, U32.astype(np.float64), sc)
    assert np.array_equal(cand.cpu().numpy(), co.reshape(-1))
    assert np.array_equal(dE.cpu().numpy(), dEo.reshape(-1))
    ref = chi0.copy()
    ro = O.blsm_parallel(ref, U32.astype(np.float64), sc)
    r = S.blsm_relax(chi, U, terms=False)
    assert ro["rounds"] > 0
    assert r["rounds"] == ro["rounds"] and r["flips"] == ro["flips"]
    assert np.array_equal(chi.cpu().numpy(), ref.reshape(-1))
    _check_stamp_modes(S, chi0, U, ref, ro)
    E = torch.zeros(3 * G, dtype=torch.float32, device="cuda")
    t = S.energy_terms(chi, U, E)
    es, _ = O.surface_energy(ref, sc)
    assert t["surf"] == es


def test_energy_clamp_with_atom_near_cell_in_second_half_of_tile():
    """A tile of 130 atoms where atom 0 sits 0.1 A from a cell centre and
    the other 129 are far from it: the clamp r >= r_min must still apply at
    that cell (every atom of a tile enters the clamp test, including the
    first of the two a thread stages)."""
    vs = _vs()
    n, h = 24, 0.5
    s = synth.random_cluster(130, n, h, seed=41)
    xyz = np.array(s["xyz"], np.float64)
    # atom 0 next to a cell centre near one corner, the rest near the other
    cell = np.array([3, 4, 5])
    c0 = np.asarray(s["origin"]) + (cell + 0.5) * h
    xyz[0] = c0 + np.array([0.1, 0.0, 0.0])
    rest = xyz[1:] - xyz[1:].mean(0)
    rest *= min(1.0, 2.0 / np.abs(rest).max())
    xyz[1:] = rest + (np.asarray(s["origin"]) + 0.75 * n * h)
    s["xyz"] = xyz
    s["bonds"] = np.zeros((0, 2), np.int64)
    s["bond_k"] = np.zeros(0)
    s["bond_r0"] = np.zeros(0)
    p = O.params()
    S = vs.System(s)
    G = n ** 3
    U, E = _fields_gpu(S, (n, n, n))
    S.energy_field(U, E)
    Uo, _, Eo = O.fields(s, p)
    k = (cell[0] * n + cell[1]) * n + cell[2]
    assert U.cpu().numpy()[k] == pytest.approx(Uo.reshape(-1)[k], rel=1e-4)
    nb, worst = _close(U.cpu().numpy(), Uo.reshape(-1))
    assert nb == 0, worst
