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
    src = open(HEADER).read()
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
    src = open(vesis.__file__).read()
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
                                          ("vesis_timing", "Timing")])
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
