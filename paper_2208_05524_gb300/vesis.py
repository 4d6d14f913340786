"""ctypes binding of libvesis.so (C ABI in include/vesis.h).

Argument marshalling only: every step of the hot path runs in the CUDA
library.  Device arrays are torch CUDA tensors (contiguous, on the device
the system was created on); host arrays are numpy float64.  If the library
is missing the import of `lib()` raises: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libvesis.so")

_d, _i, _p, _ll = C.c_double, C.c_int, C.c_void_p, C.c_longlong


class Params(C.Structure):
    _fields_ = [("gamma0", _d), ("rho_w", _d), ("eps_m", _d), ("eps_w", _d),
                ("temperature", _d), ("eps_ss", _d), ("nx", _i), ("ny", _i),
                ("nz", _i), ("h", _d), ("origin", _d * 3),
                ("gauss_sigma", _d), ("trunc_r", _i), ("r_min", _d),
                ("far_field", _i), ("far_nuv", _i), ("far_nt", _i),
                ("kernel", _i), ("sin2_lambda", _d)]


class RelaxOpts(C.Structure):
    _fields_ = [("max_outer", _i), ("ncnt_star", _i), ("window", _i),
                ("M0", _d), ("alpha", _d), ("dgstar_frac", _d),
                ("tol_grad", _d), ("tol_energy", _d), ("max_flip_rounds", _i),
                ("max_gd_retries", _i), ("resume", _i)]


class RelaxState(C.Structure):
    _fields_ = [("k", _i), ("ncnt", _i), ("stable", _i), ("valid", _i), ("M", _d),
                ("G_prev", _d)]


class RelaxStats(C.Structure):
    _fields_ = [("status", _i), ("iterations", _i), ("stop_reason", _i),
                ("flip_rounds", _ll), ("flips", _ll), ("gd_trials", _ll),
                ("pair_evals", _ll), ("G", _d), ("terms", _d * 6), ("M", _d),
                ("max_grad", _d), ("records", _i)]


class IterRecord(C.Structure):
    _fields_ = [("k", _i), ("rounds", _i), ("flips", _ll), ("trials", _i), ("ncnt", _i),
                ("G", _d), ("G_old", _d), ("M", _d), ("max_grad", _d)]


class Timing(C.Structure):
    _fields_ = [("pair_energy_ms", _d), ("pair_energy_launches", _ll),
                ("pair_energy_pairs", _ll), ("pair_force_ms", _d),
                ("pair_force_launches", _ll), ("pair_force_pairs", _ll),
                ("sweep_ms", _d), ("sweep_rounds", _ll), ("sweep_cells", _ll),
                ("kernel_launches", _ll), ("conv_ms", _d), ("conv_launches", _ll),
                ("conv_cells", _ll), ("sweep_tiles_decide", _ll),
                ("sweep_tiles_update", _ll)]


STATUS = {0: "OK", -1: "E_ARG", -2: "E_CUDA", -3: "E_NAN", -4: "E_OUT_OF_BOX",
          -5: "E_ALLOC", 1: "W_MAX_ROUNDS", 2: "W_NOT_CONVERGED"}
TERMS = ("surf", "vdw", "cfa", "far", "ss", "total")


class VesisError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"vesis {STATUS.get(code, code)}: {msg}")
        self.code = code


_lib = None


def lib():
    """Load libvesis.so (built by paper_2208_05524_gb300.build)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(
                "libvesis.so is not built; run paper_2208_05524_gb300.build.build()")
        L = C.CDLL(LIB_PATH)
        L.vesis_default_params.argtypes = [C.POINTER(Params)]
        L.vesis_default_params.restype = None
        L.vesis_default_relax_opts.argtypes = [C.POINTER(RelaxOpts)]
        L.vesis_default_relax_opts.restype = None
        L.vesis_init_system.argtypes = [C.POINTER(Params), _i, _p, _p, _p, _p,
                                        _p, _p, _i, _p, _p, _p, _p,
                                        C.POINTER(_p)]
        L.vesis_set_positions.argtypes = [_p, _p]
        L.vesis_get_positions.argtypes = [_p, _p]
        L.vesis_init_labels.argtypes = [_p, _i, _p, _d, _p, _p]
        L.vesis_energy_field.argtypes = [_p, _p, _p, _p, _p, _p]
        L.vesis_energy_terms.argtypes = [_p, _p, _p, _p, _p]
        L.vesis_surface_weights.argtypes = [_p, _p, _p]
        L.vesis_flip_energies.argtypes = [_p, _p, _p, _p, _p]
        L.vesis_blsm_relax.argtypes = [_p, _p, _p, _p, _i, C.POINTER(_i),
                                       C.POINTER(_ll), C.POINTER(_d), _p]
        L.vesis_atom_forces.argtypes = [_p, _p, _p, _p, _p, _p]
        L.vesis_blsm_heap.argtypes = [_p, _p, _p, _p, _ll, C.POINTER(_ll), C.POINTER(_d),
                                      _p]
        L.vesis_relax.argtypes = [_p, _p, _p, C.POINTER(RelaxOpts),
                                  C.POINTER(RelaxStats)]
        L.vesis_set_timing.argtypes = [_p, _i]
        L.vesis_get_timing.argtypes = [_p, C.POINTER(Timing)]
        L.vesis_surface_weights_noalloc.argtypes = [C.POINTER(Params), _p, _p, _p]
        L.vesis_set_tiles.argtypes = [_p, _i, _i]
        L.vesis_set_wait_limit.argtypes = [_p, _ll]
        L.vesis_set_sweep_stamps.argtypes = [_p, _i]
        L.vesis_get_state.argtypes = [_p, C.POINTER(RelaxState)]
        L.vesis_blsm_relax_batch.argtypes = [_i, _p, _p, _p, _i, _p, _p, _p]
        L.vesis_set_history.argtypes = [_p, _p, _i]
        L.vesis_set_state.argtypes = [_p, C.POINTER(RelaxState)]
        L.vesis_features.argtypes = [_p, _p, _p, _p, _d, _p]
        L.vesis_ss_terms.argtypes = [_p, _p]
        L.vesis_set_bonded.argtypes = [_p, _i, _p, _p, _p, _i, _p, _p, _p]
        L.vesis_net_create.argtypes = [_i, _p, _p]
        L.vesis_net_param_count.argtypes = [_p, C.POINTER(_ll)]
        L.vesis_net_set_params.argtypes = [_p, _p]
        L.vesis_net_get_params.argtypes = [_p, _p]
        L.vesis_net_forward.argtypes = [_p, _p, _i, _i, _i, _p, _p, _p]
        L.vesis_net_loss_grad.argtypes = [_p, _p, _p, _i, _i, _i, _p, C.POINTER(_d), _p]
        L.vesis_net_adam_step.argtypes = [_p, _d, _d, _d, _d]
        L.vesis_net_set_conv_kernel.argtypes = [_p, _i]
        L.vesis_net_destroy.argtypes = [_p]
        L.vesis_get_tiles.argtypes = [_p, C.POINTER(_i), C.POINTER(_i)]
        L.vesis_autotune.argtypes = [_p, _p, _i, _p]
        L.vesis_relax_batch.argtypes = [_i, _p, _p, _p, C.POINTER(RelaxOpts), _i, _i,
                                        _p, _p]
        L.vesis_destroy.argtypes = [_p]
        L.vesis_last_error.restype = C.c_char_p
        _lib = L
    return _lib


def _check(rc, allow_warn=True):
    if rc < 0 or (rc > 0 and not allow_warn):
        raise VesisError(rc, lib().vesis_last_error().decode())
    return rc


def _np(a, dtype=np.float64):
    return np.ascontiguousarray(a, dtype=dtype)


def _hp(a):
    return a.ctypes.data_as(_p) if a is not None else None


def _dp(t, dtype=None, numel=None):
    """Raw device pointer of a contiguous CUDA tensor (checked)."""
    if t is None:
        return None
    if not t.is_cuda or not t.is_contiguous():
        raise ValueError("device arrays must be contiguous CUDA tensors")
    if dtype is not None and t.dtype != dtype:
        raise ValueError(f"expected {dtype}, got {t.dtype}")
    if numel is not None and t.numel() < numel:
        raise ValueError(f"tensor too small: {t.numel()} < {numel}")
    return _p(t.data_ptr())


def default_params(**kw):
    p = Params()
    lib().vesis_default_params(C.byref(p))
    for k, v in kw.items():
        if k == "origin":
            p.origin[:] = [float(x) for x in v]
        else:
            setattr(p, k, v)
    return p


def default_relax_opts(**kw):
    o = RelaxOpts()
    lib().vesis_default_relax_opts(C.byref(o))
    for k, v in kw.items():
        setattr(o, k, v)
    return o


NOALLOC_MAX_CELLS = 1 << 20


def surface_weights_noalloc(params, chi, W, stream=None):
    """vesis_surface_weights_noalloc: the kernel convolution of the labels
    without any device allocation (for callers that cannot allocate, e.g.
    inside a stream capture).  params: a Params (grid, h, kernel); chi and W
    contiguous CUDA tensors of G uint8 / int32.  Calls share one scratch
    array: do not overlap them on the GPU."""
    import torch
    G = params.nx * params.ny * params.nz
    st = stream if stream is not None else torch.cuda.current_stream()
    _check(lib().vesis_surface_weights_noalloc(
        C.byref(params), _dp(chi, torch.uint8, G), _dp(W, torch.int32, G),
        _p(st.cuda_stream)))


class System:
    """One solute system on the current CUDA device.

    sysd: dict from paper_2208_05524_gb300.synth (atoms, grid, bonds).
    params: overrides of vesis_params fields (gauss_sigma <= 0 means 2 h).
    stream: torch.cuda.Stream (default: the current stream)."""

    def __init__(self, sysd, stream=None, **params):
        import torch
        n = [int(v) for v in sysd["n"]]
        p = default_params(nx=n[0], ny=n[1], nz=n[2], h=float(sysd["h"]),
                           origin=sysd["origin"])
        for k, v in params.items():
            if k == "origin":
                p.origin[:] = [float(x) for x in v]
            elif k == "kernel":     # "gauss" / "sin2" (or 0 / 1)
                p.kernel = {"gauss": 0, "sin2": 1}.get(v, v)
            else:
                setattr(p, k, v)
        self.params = p
        self.n_atoms = len(sysd["xyz"])
        self.sigma = np.asarray(sysd["sigma_sw"], np.float64).copy()
        self.G = n[0] * n[1] * n[2]
        self.shape = tuple(n)
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self._keep = [_np(sysd[k]) for k in ("xyz", "sigma_sw", "eps_sw", "q",
                                            "sigma_ss", "eps_ss")]
        bonds = _np(sysd["bonds"], np.int32).reshape(-1, 2)
        bk, br = _np(sysd["bond_k"]), _np(sysd["bond_r0"])
        self._keep += [bonds, bk, br]
        h = _p()
        _check(lib().vesis_init_system(
            C.byref(p), self.n_atoms, *[_hp(a) for a in self._keep[:6]],
            len(bonds), _hp(bonds), _hp(bk), _hp(br),
            _p(self.stream.cuda_stream), C.byref(h)), allow_warn=False)
        self.h = h
        if len(sysd.get("angles", ())) or len(sysd.get("torsions", ())):
            self.set_bonded(sysd.get("angles"), sysd.get("angle_B"), sysd.get("angle_theta0"),
                            sysd.get("torsions"), sysd.get("torsion_C"),
                            sysd.get("torsion_psi"))

    # ------------------------------------------------------------- calls
    def close(self):
        if getattr(self, "h", None):
            lib().vesis_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_positions(self, xyz):
        a = _np(xyz).reshape(-1, 3)
        _check(lib().vesis_set_positions(self.h, _hp(a)), allow_warn=False)

    def get_positions(self):
        out = np.zeros((self.n_atoms, 3))
        _check(lib().vesis_get_positions(self.h, _hp(out)), allow_warn=False)
        return out

    def init_labels(self, chi, kind="tight", d=None, radius=0.0, center=None):
        import torch
        k = {"sphere": 0, "tight": 1}[kind]
        dd = None if d is None else _np(d)
        cc = None if center is None else _np(center)
        _check(lib().vesis_init_labels(self.h, k, _hp(dd), float(radius),
                                       _hp(cc), _dp(chi, torch.uint8, self.G)))

    def energy_field(self, U, E=None, chi=None, xyz=None, terms=False):
        import torch
        out = (_d * 6)() if terms else None
        x = None if xyz is None else _np(xyz).reshape(-1, 3)
        _check(lib().vesis_energy_field(
            self.h, _hp(x), _dp(U, torch.float32, self.G),
            _dp(E, torch.float32, 3 * self.G) if E is not None else None,
            _dp(chi, torch.uint8, self.G) if chi is not None else None,
            C.cast(out, _p) if out is not None else None))
        return dict(zip(TERMS, list(out))) if out is not None else None

    def energy_terms(self, chi, U, E=None):
        import torch
        out = (_d * 6)()
        _check(lib().vesis_energy_terms(
            self.h, _dp(chi, torch.uint8, self.G), _dp(U, torch.float32, self.G),
            _dp(E, torch.float32, 3 * self.G) if E is not None else None,
            C.cast(out, _p)))
        return dict(zip(TERMS, list(out)))

    def surface_weights(self, chi, W):
        import torch
        _check(lib().vesis_surface_weights(
            self.h, _dp(chi, torch.uint8, self.G), _dp(W, torch.int32, self.G)))

    def flip_energies(self, chi, U, dE, cand):
        import torch
        _check(lib().vesis_flip_energies(
            self.h, _dp(chi, torch.uint8, self.G), _dp(U, torch.float32, self.G),
            _dp(dE, torch.float64, self.G), _dp(cand, torch.uint8, self.G)))

    def blsm_relax(self, chi, U, E=None, max_rounds=100000, terms=True):
        import torch
        rounds, flips, dsum = _i(0), _ll(0), _d(0.0)
        out = (_d * 6)() if terms else None
        rc = _check(lib().vesis_blsm_relax(
            self.h, _dp(chi, torch.uint8, self.G), _dp(U, torch.float32, self.G),
            _dp(E, torch.float32, 3 * self.G) if E is not None else None,
            int(max_rounds), C.byref(rounds), C.byref(flips), C.byref(dsum),
            C.cast(out, _p) if out is not None else None))
        r = dict(status=rc, rounds=rounds.value, flips=flips.value,
                 dE_sum=dsum.value)
        if out is not None:
            r["terms"] = dict(zip(TERMS, list(out)))
        return r

    def blsm_heap(self, chi, U, E=None, max_flips=1 << 62, terms=True):
        """The literal serial flipping (vesis_blsm_heap)."""
        import torch
        flips, dsum = _ll(0), _d(0.0)
        out = (_d * 6)() if terms else None
        rc = _check(lib().vesis_blsm_heap(
            self.h, _dp(chi, torch.uint8, self.G), _dp(U, torch.float32, self.G),
            _dp(E, torch.float32, 3 * self.G) if E is not None else None,
            int(max_flips), C.byref(flips), C.byref(dsum),
            C.cast(out, _p) if out is not None else None))
        r = dict(status=rc, flips=flips.value, dE_sum=dsum.value)
        if out is not None:
            r["terms"] = dict(zip(TERMS, list(out)))
        return r

    def atom_forces(self, chi, xyz=None, E=None, energy=False):
        import torch
        g = np.zeros((self.n_atoms, 3))
        e = _d(0.0)
        x = None if xyz is None else _np(xyz).reshape(-1, 3)
        _check(lib().vesis_atom_forces(
            self.h, _dp(chi, torch.uint8, self.G), _hp(x),
            _dp(E, torch.float32, 3 * self.G) if E is not None else None,
            _hp(g), C.byref(e) if energy else None))
        return (g, e.value) if energy else g

    def set_timing(self, enable=True):
        _check(lib().vesis_set_timing(self.h, int(bool(enable))))

    def get_timing(self):
        t = Timing()
        _check(lib().vesis_get_timing(self.h, C.byref(t)))
        return {f: getattr(t, f) for f, _ in Timing._fields_}

    def set_history(self, capacity):
        """Per-iteration log of later relax calls (vesis_set_history): up to
        `capacity` records, returned by relax() as res["history"]; 0 turns
        it off."""
        self._hist = (IterRecord * capacity)() if capacity > 0 else None
        _check(lib().vesis_set_history(self.h, C.cast(self._hist, _p) if capacity else None,
                                       int(capacity)))

    def get_state(self):
        """Where the last relaxation stopped (vesis_get_state), as a dict."""
        st = RelaxState()
        _check(lib().vesis_get_state(self.h, C.byref(st)))
        return {f: getattr(st, f) for f, _ in RelaxState._fields_}

    def set_state(self, state):
        """Loads a saved relaxation state (vesis_set_state); relax(...,
        resume=1) then continues from it."""
        st = RelaxState(**{f: state[f] for f, _ in RelaxState._fields_})
        _check(lib().vesis_set_state(self.h, C.byref(st)))

    def set_wait_limit(self, polls=1 << 24):
        """Polls a flip-sweep block makes at a grid barrier before the sweep
        gives up with VESIS_E_CUDA (vesis_set_wait_limit)."""
        _check(lib().vesis_set_wait_limit(self.h, int(polls)))

    def set_sweep_stamps(self, mode=-1):
        """Which tiles a flip-sweep round decides (vesis_set_sweep_stamps):
        -1 by the leader count, 0 every leader tile, 1 only the stamped ones.
        Results are identical in every mode."""
        _check(lib().vesis_set_sweep_stamps(self.h, int(mode)))

    def set_tiles(self, energy_pencil=8, force_atoms=4):
        _check(lib().vesis_set_tiles(self.h, int(energy_pencil), int(force_atoms)))

    def get_tiles(self):
        pe, fa = _i(0), _i(0)
        _check(lib().vesis_get_tiles(self.h, C.byref(pe), C.byref(fa)))
        return pe.value, fa.value

    def autotune(self, chi, reps=3):
        """Times the pair kernels' tile shapes on this system and keeps the
        fastest; returns the chosen shapes and the four mean times (ms)."""
        import torch
        t = (_d * 5)()
        _check(lib().vesis_autotune(self.h, _dp(chi, torch.uint8, self.G), int(reps),
                                    C.cast(t, _p)))
        pe, fa = self.get_tiles()
        return dict(energy_pencil=pe, force_atoms=fa,
                    ms={"energy_pencil4": t[0], "energy_pencil8": t[1], "energy_pencil16": t[2],
                        "force_atoms2": t[3], "force_atoms4": t[4]})

    def ss_terms(self):
        """Solute-solute bonds, LJ, Coulomb, bends and torsions at the
        current positions."""
        out = (_d * 5)()
        _check(lib().vesis_ss_terms(self.h, C.cast(out, _p)))
        return dict(bonds=out[0], lj=out[1], coulomb=out[2], bend=out[3], torsion=out[4])

    def set_bonded(self, angles=None, angle_B=None, angle_theta0=None, torsions=None,
                   torsion_C=None, torsion_psi=None):
        """Bend and torsion terms (vesis_set_bonded); None clears a kind."""
        a = np.zeros((0, 3), np.int32) if angles is None else _np(angles, np.int32).reshape(-1, 3)
        t = np.zeros((0, 4), np.int32) if torsions is None else _np(torsions, np.int32).reshape(-1, 4)
        B = _np(angle_B if angles is not None else np.zeros(0))
        T0 = _np(angle_theta0 if angles is not None else np.zeros(0))
        Cc = _np(torsion_C if torsions is not None else np.zeros((0, 7))).reshape(-1, 7)
        P = _np(torsion_psi if torsions is not None else np.zeros((0, 7))).reshape(-1, 7)
        self._bonded = (a, B, T0, t, Cc, P)
        _check(lib().vesis_set_bonded(self.h, len(a), _hp(a), _hp(B), _hp(T0), len(t), _hp(t),
                                      _hp(Cc), _hp(P)), allow_warn=False)

    def features(self, U, E, chi_tight, x, scale=0.01):
        """Learned-initialiser input planes (3 x G floats) into x."""
        import torch
        _check(lib().vesis_features(self.h, _dp(U, torch.float32, self.G),
                                    _dp(E, torch.float32, 3 * self.G),
                                    _dp(chi_tight, torch.uint8, self.G), float(scale),
                                    _dp(x, torch.float32, 3 * self.G)))

    def relax(self, chi, xyz, **opts):
        import torch
        o = default_relax_opts(**opts)
        x = _np(xyz).reshape(-1, 3).copy()
        st = RelaxStats()
        rc = _check(lib().vesis_relax(self.h, _dp(chi, torch.uint8, self.G),
                                      _hp(x), C.byref(o), C.byref(st)))
        res = {f: getattr(st, f) for f, _ in RelaxStats._fields_ if f != "terms"}
        res["terms"] = dict(zip(TERMS, list(st.terms)))
        res["status"] = rc
        res["xyz"] = x
        if getattr(self, "_hist", None) is not None:
            res["history"] = [{f: getattr(r, f) for f, _ in IterRecord._fields_}
                              for r in self._hist[:st.records]]
        return res


def blsm_relax_batch(systems, chis, Us, max_rounds=100000):
    """vesis_blsm_relax_batch: the flip rounds of every (system, chi, U) in
    one persistent launch; chi tensors are relaxed in place.  Returns one
    dict per system (status of the call, rounds, flips, dE_sum)."""
    import torch
    n = len(systems)
    if not (len(chis) == n and len(Us) == n):
        raise ValueError("systems, chis and Us differ in length")
    hs = (_p * n)(*[s.h for s in systems])
    cs = (_p * n)(*[_dp(c, torch.uint8, s.G) for s, c in zip(systems, chis)])
    us = (_p * n)(*[_dp(u, torch.float32, s.G) for s, u in zip(systems, Us)])
    rounds = (_i * n)()
    flips = (_ll * n)()
    dsum = (_d * n)()
    rc = _check(lib().vesis_blsm_relax_batch(n, C.cast(hs, _p), C.cast(cs, _p), C.cast(us, _p),
                                             int(max_rounds), C.cast(rounds, _p),
                                             C.cast(flips, _p), C.cast(dsum, _p)))
    return [dict(status=rc, rounds=rounds[i], flips=flips[i], dE_sum=dsum[i]) for i in range(n)]


def relax_batch(systems, chis, xyzs, threads=8, sweep_slots=2, **opts):
    """vesis_relax_batch: relaxes every (system, chi, xyz) with the same
    options on `threads` host threads; chi tensors are updated in place.
    Returns one result dict per system, as System.relax does."""
    import torch
    n = len(systems)
    if not (len(chis) == n and len(xyzs) == n):
        raise ValueError("systems, chis and xyzs differ in length")
    o = default_relax_opts(**opts)
    hs = (_p * n)(*[s.h for s in systems])
    cs = (_p * n)(*[_dp(c, torch.uint8, s.G) for s, c in zip(systems, chis)])
    xs = [_np(x).reshape(-1, 3).copy() for x in xyzs]
    xp = (_p * n)(*[_hp(x) for x in xs])
    st = (RelaxStats * n)()
    status = (_i * n)()
    _check(lib().vesis_relax_batch(n, C.cast(hs, _p), C.cast(cs, _p), C.cast(xp, _p),
                                   C.byref(o), int(threads), int(sweep_slots),
                                   C.cast(st, _p), C.cast(status, _p)))
    out = []
    for i in range(n):
        res = {f: getattr(st[i], f) for f, _ in RelaxStats._fields_ if f != "terms"}
        res["terms"] = dict(zip(TERMS, list(st[i].terms)))
        res["status"] = status[i]
        res["xyz"] = xs[i]
        out.append(res)
    return out


class Net:
    """The learned initialiser's network (vesis_net_*): a 3-D U-Net on
    n_features input planes; parameters in the flat order of the header."""

    def __init__(self, n_features=3, stream=None):
        import torch
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        h = _p()
        _check(lib().vesis_net_create(int(n_features), _p(self.stream.cuda_stream),
                                      C.byref(h)), allow_warn=False)
        self.h = h
        self.F = int(n_features)
        n = _ll(0)
        _check(lib().vesis_net_param_count(self.h, C.byref(n)))
        self.P = n.value

    def close(self):
        if getattr(self, "h", None):
            lib().vesis_net_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_params(self, theta):
        a = np.ascontiguousarray(theta, np.float32)
        if a.size != self.P:
            raise ValueError(f"expected {self.P} parameters, got {a.size}")
        _check(lib().vesis_net_set_params(self.h, _hp(a)))

    def get_params(self):
        out = np.zeros(self.P, np.float32)
        _check(lib().vesis_net_get_params(self.h, _hp(out)))
        return out

    @staticmethod
    def _crop(crop):
        return None if crop is None else (_i * 6)(*[int(v) for v in crop])

    def forward(self, x, shape, crop=None, logits=None, chi=None):
        import torch
        n = [int(v) for v in shape]
        c = self._crop(crop)
        V = int(np.prod(crop[3:])) if crop is not None else int(np.prod(n))
        _check(lib().vesis_net_forward(
            self.h, _dp(x, torch.float32, self.F * int(np.prod(n))), n[0], n[1], n[2],
            C.cast(c, _p) if c is not None else None,
            _dp(logits, torch.float32, V) if logits is not None else None,
            _dp(chi, torch.uint8, V) if chi is not None else None))

    def loss_grad(self, x, chi, shape, crop=None, grad=False):
        import torch
        n = [int(v) for v in shape]
        G = int(np.prod(n))
        c = self._crop(crop)
        loss = _d(0.0)
        g = np.zeros(self.P, np.float32) if grad else None
        _check(lib().vesis_net_loss_grad(
            self.h, _dp(x, torch.float32, self.F * G), _dp(chi, torch.uint8, G), n[0], n[1],
            n[2], C.cast(c, _p) if c is not None else None, C.byref(loss), _hp(g)))
        return (loss.value, g) if grad else loss.value

    def set_conv_kernel(self, kind):
        """0: mma.sync convolutions; 1: tcgen05 where the grid allows."""
        _check(lib().vesis_net_set_conv_kernel(self.h, {"mma": 0, "tcgen05": 1}.get(kind, kind)))

    def adam_step(self, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8):
        _check(lib().vesis_net_adam_step(self.h, float(lr), float(beta1), float(beta2),
                                         float(eps)))
