"""Host-side checks of the C ABI library (no GPU needed).

The library loads without a device, exports every function include/vesis.h
declares, and the ctypes mirrors of its structs have the C layout.  No
compute call is made here.
"""
import ctypes as C
import os
import re
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "vesis.h")


@pytest.fixture(scope="module")
def built():
    from paper_2208_05524_gb300 import build
    return build.build()


def _declared():
    with open(HEADER) as f:
        src = f.read()
    return sorted(set(re.findall(r"^\s*(?:int|void|const char \*)\s*(vesis_\w+)\s*\(",
                                 src, flags=re.M)))


def test_library_exports_every_declared_symbol(built):
    names = _declared()
    assert len(names) >= 16
    L = C.CDLL(built)
    for n in names:
        assert hasattr(L, n), n
    out = subprocess.run(["nm", "-D", "--defined-only", built], capture_output=True,
                         text=True, check=True).stdout
    exported = set(re.findall(r" T (vesis_\w+)", out))
    assert set(names) <= exported
    # nothing else of the library's own namespace leaks as a C symbol
    assert exported <= set(names)


def test_binding_declares_every_symbol(built):
    from paper_2208_05524_gb300 import vesis
    with open(vesis.__file__) as f:
        src = f.read()
    for n in _declared():
        assert n in src, n


def _c_layout(struct, fields):
    prog = ["#include <stdio.h>", "#include <stddef.h>", '#include "vesis.h"',
            "int main(void){", f'printf("%zu\\n", sizeof({struct}));']
    for f in fields:
        prog.append(f'printf("%zu\\n", offsetof({struct}, {f}));')
    prog.append("return 0;}")
    return "\n".join(prog)


@pytest.mark.parametrize("cname,pyname", [("vesis_params", "Params"),
                                          ("vesis_relax_opts", "RelaxOpts"),
                                          ("vesis_relax_stats", "RelaxStats"),
                                          ("vesis_timing", "Timing"),
                                          ("vesis_relax_state", "RelaxState"),
                                          ("vesis_iter_record", "IterRecord")])
def test_struct_layouts_match_header(tmp_path, built, cname, pyname):
    from paper_2208_05524_gb300 import vesis
    cls = getattr(vesis, pyname)
    fields = [f for f, _ in cls._fields_]
    src = tmp_path / "layout.c"
    src.write_text(_c_layout(cname, fields))
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                   check=True)
    vals = [int(x) for x in subprocess.run([str(exe)], capture_output=True, text=True,
                                           check=True).stdout.split()]
    assert vals[0] == C.sizeof(cls)
    for f, off in zip(fields, vals[1:]):
        assert getattr(cls, f).offset == off, f


def test_defaults_follow_table1_and_step1(built):
    from paper_2208_05524_gb300 import vesis
    p = vesis.default_params()
    assert (p.temperature, p.rho_w, p.gamma0, p.eps_m, p.eps_w) == (298.0, 0.0333, 0.174, 1.0, 80.0)
    o = vesis.default_relax_opts()
    assert (o.max_outer, o.ncnt_star, o.window, o.M0) == (3000, 5, 100, 1.0)
    assert o.alpha == pytest.approx(1 / np.sqrt(2))
    assert (o.dgstar_frac, o.tol_grad, o.tol_energy) == (0.05, 1e-4, 1e-5)


def test_argument_errors_without_device(built):
    # validation happens before any CUDA call
    from paper_2208_05524_gb300 import vesis
    L = vesis.lib()
    p = vesis.default_params()
    h = C.c_void_p()
    x = np.zeros(3)
    rc = L.vesis_init_system(C.byref(p), 0, x.ctypes.data_as(C.c_void_p), *([x.ctypes.data_as(C.c_void_p)] * 5),
                             0, None, None, None, None, C.byref(h))
    assert rc == -1 and b"n_atoms" in L.vesis_last_error()
    p.trunc_r = 9
    rc = L.vesis_init_system(C.byref(p), 1, *([x.ctypes.data_as(C.c_void_p)] * 6),
                             0, None, None, None, None, C.byref(h))
    assert rc == -1 and b"trunc_r" in L.vesis_last_error()
    assert L.vesis_destroy(None) == 0


def test_synthetic_inputs_are_seeded():
    from paper_2208_05524_gb300 import synth
    a = synth.protein_like(n_atoms=300, n=32, seed=7)
    b = synth.protein_like(n_atoms=300, n=32, seed=7)
    for k in ("xyz", "sigma_sw", "eps_sw", "q", "bonds", "bond_r0"):
        assert np.array_equal(a[k], b[k])
    assert a["q"].sum() == pytest.approx(-3.0)
    assert np.all((a["sigma_sw"] >= 3.0) & (a["sigma_sw"] <= 4.0))
    c = synth.protein_like(n_atoms=300, n=32, seed=8)
    assert not np.array_equal(a["xyz"], c["xyz"])


def test_batch_and_tile_argument_errors_without_device(built):
    # checked before any CUDA call
    from paper_2208_05524_gb300 import vesis
    L = vesis.lib()
    o = vesis.default_relax_opts()
    assert L.vesis_relax_batch(0, None, None, None, C.byref(o), 4, 2, None, None) == 0
    one = (C.c_void_p * 1)(None)
    rc = L.vesis_relax_batch(1, C.cast(one, C.c_void_p), C.cast(one, C.c_void_p),
                             C.cast(one, C.c_void_p), C.byref(o), 4, 2, None, None)
    assert rc == -1 and b"NULL system" in L.vesis_last_error()
    rc = L.vesis_relax_batch(1, C.cast(one, C.c_void_p), C.cast(one, C.c_void_p),
                             C.cast(one, C.c_void_p), C.byref(o), 0, 2, None, None)
    assert rc == -1 and b"threads" in L.vesis_last_error()
    rc = L.vesis_relax_batch(1, C.cast(one, C.c_void_p), C.cast(one, C.c_void_p),
                             C.cast(one, C.c_void_p), C.byref(o), 4, 0, None, None)
    assert rc == -1 and b"sweep_slots" in L.vesis_last_error()
    assert L.vesis_relax_batch(-1, None, None, None, None, 1, 1, None, None) == -1
    assert L.vesis_set_tiles(None, 8, 4) == -1
    assert L.vesis_set_sweep_stamps(None, 1) == -1
    assert L.vesis_get_tiles(None, None, None) == -1
    assert L.vesis_autotune(None, None, 3, None) == -1


def test_host_guest_set_follows_its_recipe():
    from paper_2208_05524_gb300 import synth
    a = synth.host_guest(5)
    b = synth.host_guest(5)
    for k in ("xyz", "sigma_sw", "q", "bonds"):
        assert np.array_equal(a[k], b[k])
    c = synth.host_guest(6)
    assert not np.array_equal(a["xyz"][:20], c["xyz"][:20])
    for s in (a, c):
        assert 150 <= s["n_host"] <= 4000 and 20 <= s["n_guest"] <= 80
        assert len(s["xyz"]) == s["n_host"] + s["n_guest"]
        assert s["q"].sum() == pytest.approx(0.0, abs=1e-9)
        n = int(s["n"][0])
        assert np.all(s["n"] == n) and n % 16 == 0 and n >= 64
        # every atom is at least 8 A inside the box
        half = 0.5 * n * float(s["h"])
        assert np.abs(s["xyz"]).max() + 8.0 <= half + 1e-9
        # host and guest do not overlap: the closest pair is a bond apart or more
        hx, gx = s["xyz"][:s["n_host"]], s["xyz"][s["n_host"]:]
        d = np.sqrt(((hx[:, None, :] - gx[None, :, :]) ** 2).sum(-1)).min()
        assert d > 3.0


def test_pmf_combination_follows_the_appendix_definition():
    from paper_2208_05524_gb300 import pmf
    pair = dict(geom=10.0, vdw=-4.0, elec=-30.0, far=-2.0, lj=0.5, coulomb=-46.0)
    a1 = dict(geom=6.0, vdw=-2.5, elec=-20.0, far=-1.0, lj=0.0, coulomb=0.0)
    a2 = dict(geom=5.0, vdw=-2.0, elec=-15.0, far=-1.5, lj=0.0, coulomb=0.0)
    r = pmf.combine(pair, [a1, a2])
    assert r["geom"] == pytest.approx(10.0 - 11.0)
    assert r["vdw"] == pytest.approx(-4.0 + 4.5 + 0.5)        # plus the cross LJ
    assert r["elec"] == pytest.approx(-30.0 + 35.0 - 46.0)    # plus the cross Coulomb
    assert r["far"] == pytest.approx(-2.0 + 2.5)
    assert r["total"] == pytest.approx(r["geom"] + r["vdw"] + r["elec"] + r["far"])


def test_random_crops_stay_inside_and_on_the_8_cell_lattice():
    from paper_2208_05524_gb300 import learned
    rng = np.random.default_rng(0)
    for shape in [(64, 64, 64), (80, 96, 112), (40, 200, 16)]:
        for _ in range(50):
            c = learned.random_crop(shape, 64, rng)
            for d in range(3):
                assert c[d] % 8 == 0 and c[3 + d] % 8 == 0 and c[3 + d] >= 8
                assert c[d] + c[3 + d] <= shape[d]


def test_bend_torsion_lists_from_a_bond_graph():
    from paper_2208_05524_gb300 import synth
    # a 5-atom chain 0-1-2-3-4 with a branch 2-5: angles at 1 (0-1-2), at 2
    # (1-2-3, 1-2-5, 3-2-5), at 3 (2-3-4); torsions along 3-bond paths
    s = synth.single_ion(n=16, h=0.5)
    s["xyz"] = np.array([[0, 0, 0], [1.5, 0, 0], [2, 1.4, 0], [3.5, 1.5, 0.3],
                         [4, 2.9, 0.2], [1.6, 2.2, 1.2]], float)
    for k in ("sigma_sw", "eps_sw", "q", "sigma_ss", "eps_ss"):
        s[k] = np.full(6, float(np.asarray(s[k])[0]))
    s["bonds"] = np.array([[0, 1], [1, 2], [2, 3], [3, 4], [2, 5]], np.int32)
    s["bond_k"] = np.full(5, 800.0)
    s["bond_r0"] = np.full(5, 1.5)
    t = synth.with_bends_torsions(s)
    ang = {tuple(a) for a in t["angles"]}
    assert ang == {(0, 1, 2), (1, 2, 3), (1, 2, 5), (3, 2, 5), (2, 3, 4)}
    tor = {tuple(x) for x in t["torsions"]}
    # every path i-j-k-l over three bonds, listed once per middle bond direction
    assert {(0, 1, 2, 3), (0, 1, 2, 5), (1, 2, 3, 4), (5, 2, 3, 4)} <= tor | {tuple(x[::-1]) for x in tor}
    assert np.allclose(t["torsion_psi"][0], [np.pi, 0, np.pi, 0, np.pi, 0, np.pi])
    sub = synth.subset(t, [1, 2, 3])
    assert sub["bonds"].tolist() == [[0, 1], [1, 2]]


def test_network_and_extension_argument_errors_without_device(built):
    # the learned initialiser's and the f-rows' entry points check their
    # arguments before any CUDA call
    from paper_2208_05524_gb300 import vesis
    L = vesis.lib()
    h = C.c_void_p()
    assert L.vesis_net_create(3, None, None) == -1
    assert L.vesis_net_create(0, None, C.byref(h)) == -1
    assert b"n_features" in L.vesis_last_error()
    assert L.vesis_net_create(33, None, C.byref(h)) == -1
    n = C.c_longlong()
    assert L.vesis_net_param_count(None, C.byref(n)) == -1
    assert L.vesis_net_set_params(None, None) == -1
    assert L.vesis_net_forward(None, None, 8, 8, 8, None, None, None) == -1
    assert L.vesis_net_loss_grad(None, None, None, 8, 8, 8, None, None, None) == -1
    assert L.vesis_net_adam_step(None, 1e-3, 0.9, 0.999, 1e-8) == -1
    assert L.vesis_net_set_conv_kernel(None, 1) == -1
    assert L.vesis_net_destroy(None) == 0
    out = (C.c_double * 5)()
    assert L.vesis_ss_terms(None, out) == -1
    assert L.vesis_blsm_heap(None, None, None, None, 10, None, None, None) == -1
    assert L.vesis_features(None, None, None, None, 0.01, None) == -1
