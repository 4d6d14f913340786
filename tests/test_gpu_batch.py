"""GPU checks of the tile shapes, the autotuner and the batched relaxation.

The tile shapes of the two pair kernels change only which thread handles
which cells or atoms, never the order of any sum, so the fields and
gradients of every shape are compared byte for byte, and one shape against
the FP64 oracle.  The batched relaxation must give each system exactly what
vesis_relax gives it alone.
"""
import numpy as np
import pytest

import oracle as O
from paper_2208_05524_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

SHAPES = [(4, 2), (4, 4), (8, 2), (8, 4), (16, 2), (16, 4)]


def _vs():
    from paper_2208_05524_gb300 import vesis
    return vesis


def _dev(a, dtype):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda").to(dtype).contiguous()


def _cluster():
    # 700 atoms: ragged atom tiles for 256 and 512 atoms per block; nz = 53
    # leaves a ragged pencil for both 4 and 8 cells per thread
    s = synth.random_cluster(700, 8, 0.7, seed=11, net_charge=-2.0)
    n = (54, 52, 53)
    s["n"] = np.array(n)
    s["origin"] = -0.5 * np.array(n) * 0.7
    return s


def test_tile_shapes_bit_identical_and_match_oracle():
    vs = _vs()
    s = _cluster()
    S = vs.System(s)
    G = S.G
    chi0 = O.init_labels(s)
    chi = _dev(chi0.reshape(-1), torch.uint8)
    out = {}
    for pe, fa in SHAPES:
        S.set_tiles(pe, fa)
        assert S.get_tiles() == (pe, fa)
        U = torch.empty(G, dtype=torch.float32, device="cuda")
        E = torch.empty(3 * G, dtype=torch.float32, device="cuda")
        S.energy_field(U, E)
        g = S.atom_forces(chi)
        out[(pe, fa)] = (U.cpu().numpy(), E.cpu().numpy(), g)
    ref = out[(8, 4)]
    for k, v in out.items():
        assert np.array_equal(v[0].view(np.uint32), ref[0].view(np.uint32)), k
        assert np.array_equal(v[1].view(np.uint32), ref[1].view(np.uint32)), k
        assert np.array_equal(v[2].view(np.uint64), ref[2].view(np.uint64)), k
    # the smallest shapes against the oracle
    p = O.params()
    Uo, _, Eo = O.fields(s, p)
    U4 = out[(4, 2)][0]
    tol = 1e-4 * np.abs(Uo.reshape(-1)) + 1e-4 * np.abs(Uo).max()
    assert np.all(np.abs(U4 - Uo.reshape(-1)) <= tol)
    go = O.gradient(s, p, chi0)
    g2 = out[(4, 2)][2]
    assert np.all(np.abs(g2 - go) <= 1e-4 * np.abs(go) + 1e-4 * np.abs(go).max())


def test_tile_shape_arguments():
    vs = _vs()
    S = vs.System(synth.single_ion(n=32, h=0.5))
    with pytest.raises(vs.VesisError):
        S.set_tiles(6, 4)
    with pytest.raises(vs.VesisError):
        S.set_tiles(8, 3)
    assert S.get_tiles() == (8, 4)


def test_autotune_keeps_a_valid_shape_and_results():
    vs = _vs()
    s = _cluster()
    S = vs.System(s)
    chi = _dev(O.init_labels(s).reshape(-1), torch.uint8)
    g0 = S.atom_forces(chi)
    S.set_timing(True)
    r = S.autotune(chi, reps=2)
    assert (r["energy_pencil"], r["force_atoms"]) in SHAPES
    assert all(v > 0.0 for v in r["ms"].values())
    pe = {4: r["ms"]["energy_pencil4"], 8: r["ms"]["energy_pencil8"], 16: r["ms"]["energy_pencil16"]}
    assert pe[r["energy_pencil"]] == min(pe.values())
    assert r["force_atoms"] == (2 if r["ms"]["force_atoms2"] < r["ms"]["force_atoms4"] else 4)
    # the autotuner's launches are not counted as gradient work
    assert S.get_timing()["pair_force_pairs"] == 0
    g1 = S.atom_forces(chi)
    assert np.array_equal(g0.view(np.uint64), g1.view(np.uint64))


def _batch_systems():
    # four host-guest systems of the batched set at twice its spacing (grids
    # of 80-160 cells), one of them with the paper's sin^2 surface kernel
    vs = _vs()
    out = []
    for i, idx in enumerate((0, 3, 7, 12)):
        s = synth.host_guest(idx, h=0.6)
        kw = {"kernel": "sin2"} if i == 2 else {}
        out.append((s, vs.System(s, **kw)))
    return out


def test_relax_batch_equals_sequential_relaxations():
    vs = _vs()
    systems = _batch_systems()
    opts = dict(max_outer=3)
    chis0 = []
    for s, S in systems:
        c = torch.empty(S.G, dtype=torch.uint8, device="cuda")
        S.init_labels(c, "tight")
        chis0.append(c)
    seq = []
    for (s, S), c0 in zip(systems, chis0):
        c = c0.clone()
        r = S.relax(c, s["xyz"], **opts)
        seq.append((r, c.cpu().numpy()))
    chis = [c0.clone() for c0 in chis0]
    res = vs.relax_batch([S for _, S in systems], chis, [s["xyz"] for s, _ in systems],
                         threads=3, sweep_slots=2, **opts)
    for i, ((r0, c0), r1, c1) in enumerate(zip(seq, res, chis)):
        assert r1["status"] == r0["status"] and r1["status"] >= 0, i
        assert np.array_equal(c1.cpu().numpy(), c0), i
        assert np.array_equal(r1["xyz"], r0["xyz"]), i
        for k in ("iterations", "stop_reason", "flip_rounds", "flips", "gd_trials",
                  "pair_evals", "G", "M", "max_grad"):
            assert r1[k] == r0[k], (i, k)
        assert r1["terms"] == r0["terms"], i
        assert r0["flips"] > 0 and r0["iterations"] >= 1, i
    # one thread and one slot: the same again
    chis = [c0.clone() for c0 in chis0]
    res1 = vs.relax_batch([S for _, S in systems], chis, [s["xyz"] for s, _ in systems],
                          threads=1, sweep_slots=1, **opts)
    for (r0, c0), r1, c1 in zip(seq, res1, chis):
        assert np.array_equal(c1.cpu().numpy(), c0)
        assert r1["G"] == r0["G"]
    # the systems keep working on their own streams afterwards
    s, S = systems[0]
    c = chis0[0].clone()
    r = S.relax(c, s["xyz"], **opts)
    assert r["G"] == seq[0][0]["G"]


def test_relax_batch_rejects_a_repeated_system():
    vs = _vs()
    s = synth.single_ion(n=32, h=0.5)
    S = vs.System(s)
    c = torch.empty(S.G, dtype=torch.uint8, device="cuda")
    S.init_labels(c, "tight")
    with pytest.raises(vs.VesisError, match="twice"):
        vs.relax_batch([S, S], [c, c.clone()], [s["xyz"], s["xyz"]], max_outer=1)
    assert vs.relax_batch([], [], []) == []


def _sweep_inputs(s):
    """The oracle's tight labels and its energy density rounded to FP32."""
    p = O.params()
    Uo = O.fields(s, p)[0].astype(np.float32)
    return O.init_labels(s), Uo


@pytest.mark.parametrize("kernel", ["gauss", "sin2"])
def test_multi_system_sweep_matches_single_sweeps_and_oracle(kernel):
    """vesis_blsm_relax_batch: the flip rounds of six systems of different
    grids (ragged, one already relaxed, one all solvent) in one cooperative
    launch give every system the labels, rounds and flips of
    vesis_blsm_relax alone, and the oracle's parallel rule on two of them."""
    vs = _vs()
    # the sin^2 stencil depends on h, so that batch keeps h = 0.5 A; the
    # Gaussian's weights do not, and its batch takes the h = 0.7 A cluster
    sds = [synth.random_cluster(30, 40, 0.5, seed=1, net_charge=1.0),
           synth.random_cluster(60, 44, 0.5, seed=2, net_charge=-1.0),
           synth.protein_like(n_atoms=48, n=48, h=0.5, seed=5),
           _cluster() if kernel == "gauss" else synth.random_cluster(90, 37, 0.5, seed=6),
           synth.random_cluster(20, 40, 0.5, seed=3),
           synth.random_cluster(20, 40, 0.5, seed=4)]
    kw = {} if kernel == "gauss" else {"kernel": "sin2"}
    systems = [vs.System(sd, **kw) for sd in sds]
    starts, Us = [], []
    for k, sd in enumerate(sds):
        chi0, Uo = _sweep_inputs(sd)
        if k == 5:
            chi0 = np.zeros_like(chi0)            # all solvent: nothing to flip
        starts.append(chi0)
        Us.append(_dev(Uo.reshape(-1), torch.float32))
    single = []
    for S, chi0, U in zip(systems, starts, Us):
        c = _dev(chi0.reshape(-1), torch.uint8)
        r = S.blsm_relax(c, U, terms=False)
        single.append((c.cpu().numpy(), r))
    # system 4 starts from its relaxed labels: no rounds at all
    starts[4] = single[4][0].reshape(starts[4].shape)
    single[4] = (single[4][0], dict(rounds=0, flips=0, dE_sum=0.0))
    chis = [_dev(c.reshape(-1), torch.uint8) for c in starts]
    res = vs.blsm_relax_batch(systems, chis, Us)
    for k, (c, r, (cs, rs)) in enumerate(zip(chis, res, single)):
        assert np.array_equal(c.cpu().numpy(), cs), k
        assert (r["rounds"], r["flips"]) == (rs["rounds"], rs["flips"]), k
        assert r["dE_sum"] == pytest.approx(rs["dE_sum"], rel=1e-12, abs=1e-12), k
    assert single[5][1]["flips"] == 0 and res[5]["flips"] == 0
    p = O.params(kernel=kernel)
    for k in (0, 2):
        sc = O.surface_constants(sds[k], p)
        ref = _sweep_inputs(sds[k])[0].copy()
        ro = O.blsm_parallel(ref, Us[k].cpu().numpy().astype(np.float64).reshape(ref.shape), sc)
        assert np.array_equal(chis[k].cpu().numpy(), ref.reshape(-1)), k
        assert res[k]["rounds"] == ro["rounds"], k
    # the same with the decide stamps always on (the first system's mode
    # applies to the batch)
    systems[0].set_sweep_stamps(1)
    chis = [_dev(c.reshape(-1), torch.uint8) for c in starts]
    res1 = vs.blsm_relax_batch(systems, chis, Us)
    for k, (c, r, (cs, rs)) in enumerate(zip(chis, res1, single)):
        assert np.array_equal(c.cpu().numpy(), cs), k
        assert (r["rounds"], r["flips"]) == (rs["rounds"], rs["flips"]), k
    systems[0].set_sweep_stamps(-1)
    # a cap on the rounds stops the batch with the warning
    chis = [_dev(c.reshape(-1), torch.uint8) for c in starts]
    res = vs.blsm_relax_batch(systems, chis, Us, max_rounds=2)
    assert res[0]["status"] == 1
    for S in systems:
        S.close()
