"""Plain FP64 CPU oracle for the VESIS hot path (arXiv 2208.05524).

TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the CPU
baseline leg of the benchmark may import this package; the product path
(the CUDA library and its binding) never does, and the two share no code.
Its inputs come from the seeded generators alone; its arithmetic is
written here and in vesis_oracle.c from the paper:

  * Eq. (Ur), Eq. (LJpotential): energy density U and Coulomb field E.
  * Eq. (Area), Eq. (4flip): discrete surface energy, with a separable
    truncated Gaussian in place of the sin^2 kernel (see `surface_kernel`).
  * Eq. (dGj1), Eq. (dGj2): flip energies; Sec. 3.1 Step 2: flipping.
  * Eq. (moveatoms), Eq. (adjustmml), Sec. 3.2 and Steps 3-5: adaptive-
    mobility gradient descent.
  * Eq. (GradientG): gradient, taken as the exact derivative of the discrete
    energy.
  * Eq. (GGR2) last term: the integral outside the box (`far_field_nodes`).

Parity status of each function is listed in `PARITY`.
"""
from __future__ import annotations

import ctypes as C
import math
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "vesis_oracle.c")
_LIB_DIR = os.path.join(_HERE, "_build")
_LIB = os.path.join(_LIB_DIR, "liboracle.so")
_lock = threading.Lock()
_lib = None

PARITY = {
    "fields": "pinned: Gauss law, LJ zero/minimum, superposition, sphere closed form",
    "conv": "pinned: direct 3-D sum, flat-interface calibration",
    "delta_e": "pinned: from-scratch energy differences of single flips",
    "blsm_parallel": "pinned: exact energy decrease per round, local minimality, "
                     "separation of flips, contains the cube rule",
    "blsm_heap": "pinned: exact energy decrease per flip, exhaustive minimum",
    "gradient": "pinned: central finite differences of the discrete energy",
    "ss": "pinned: finite differences, two-atom closed form",
    "far_field": "pinned: adaptive scipy quadrature, ray quadrature",
    "relax": "pinned: two-atom molecule state printed in Sec. 5.2 and its closed form",
}


def build(force: bool = False) -> str:
    """Compile vesis_oracle.c with gcc (OpenMP, no FP contraction)."""
    os.makedirs(_LIB_DIR, exist_ok=True)
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    tmp = _LIB + f".{os.getpid()}.tmp"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp",
           "-ffp-contract=off", "-fno-fast-math", _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = C.CDLL(build())
            d, i, i64, p = C.c_double, C.c_int, C.c_int64, C.c_void_p
            L.or_grid_terms.argtypes = [i, i, i, d, p, i, p, p, p, p, d, p, p]
            L.or_point_terms.argtypes = [i64, p, i, p, p, p, p, d, p, p]
            L.or_grid_grad.argtypes = [i, i, i, d, p, p, p, i, p, p, p, p, d, d, d, p]
            L.or_point_grad.argtypes = [i64, p, p, p, i, p, p, p, p, d, d, d, p]
            L.or_ss.argtypes = [i, p, p, p, p, i, p, p, p, d, p, p]
            L.or_conv.argtypes = [i, i, i, p, i, p, p]
            L.or_conv3.argtypes = [i, i, i, p, i, p, p]
            L.or_surface_sum.argtypes = [i64, p, p, i64]
            L.or_surface_sum.restype = i64
            L.or_delta_e.argtypes = [i, i, i, p, p, p, d, i64, i64, d, p, p]
            L.or_select.argtypes = [i, i, i, p, p, i, p, p]
            L.or_select.restype = i64
            L.or_select_cells.argtypes = [i, i, i, p, p, i, p, p]
            L.or_select_cells.restype = i64
            L.or_energy.argtypes = [i, i, i, p, p, i, p, p, d, i64, d]
            L.or_energy.restype = d
            L.or_blsm_parallel.argtypes = [i, i, i, p, p, i, p, p, d, i64, i64, d,
                                           i, p, p, p, i, p]
            L.or_blsm_parallel.restype = i
            L.or_blsm_heap.argtypes = [i, i, i, p, p, i, p, p, d, i64, i64, d,
                                       i64, p, i, p]
            L.or_blsm_heap.restype = i64
            L.or_init_tight.argtypes = [i, i, i, d, p, i, p, p, p]
            L.or_init_tight_at.argtypes = [i64, p, i, i, i, d, p, i, p, p, p, p]
            _lib = L
    return _lib


def _p(a):
    return a.ctypes.data_as(C.c_void_p)


def _c64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


# ------------------------------------------------------------ parameters

def params(**kw):
    """Model parameters: Table 1 (T, rho_w, gamma0, eps_m, eps_w) plus the
    discretisation choices of this implementation.  `gauss_sigma` None means
    2 h; `kernel` is "gauss" (separable truncated Gaussian) or "sin2" (the
    paper's sin^2 kernel with radius sin2_lambda sqrt(h), Sec. 3.1); `eps_ss`
    is the dielectric constant of the solute-solute Coulomb
    term (the paper writes eps_w in Eq. Gss and eps_m in the appendix; eps_m
    is the default here)."""
    p = dict(gamma0=0.174, rho_w=0.0333, eps_m=1.0, eps_w=80.0,
             temperature=298.0, eps_ss=None, gauss_sigma=None, trunc_r=6,
             rmin=0.2, far_field=True, far_nuv=16, far_nt=8,
             kernel="gauss", sin2_lambda=2.0)
    p.update(kw)
    if p["eps_ss"] is None:
        p["eps_ss"] = p["eps_m"]
    return p


def relax_opts(**kw):
    """Algorithm constants of Step 1: N*_cnt = 5, M = 1, alpha = 1/sqrt(2),
    delta G* = 5% of |G_old|, Tol1 = 1e-4 (gradient), Tol2 = 1e-5 (energy)
    held for 100 consecutive steps, k_max = 3000."""
    o = dict(max_outer=3000, ncnt_star=5, window=100, M0=1.0,
             alpha=1.0 / math.sqrt(2.0), dgstar_frac=0.05, tol_grad=1e-4,
             tol_energy=1e-5, max_flip_rounds=100000, max_gd_retries=60)
    o.update(kw)
    return o


def bjerrum(temperature):
    """l_B = e^2 / (4 pi eps0 k_B T) in Angstrom (CODATA 2018 constants)."""
    e = 1.602176634e-19
    eps0 = 8.8541878128e-12
    kB = 1.380649e-23
    return e * e / (4.0 * math.pi * eps0 * kB * temperature) * 1e10


def cfa_prefactor(p):
    """C of Eq. (Ur) in kBT*Angstrom: 1/(32 pi^2 eps0) (1/eps_w - 1/eps_m)
    times e^2/(k_B T) = (l_B / 8 pi)(1/eps_w - 1/eps_m)."""
    lb = bjerrum(p["temperature"])
    return lb / (8.0 * math.pi) * (1.0 / p["eps_w"] - 1.0 / p["eps_m"])


def surface_kernel(sigma_over_h: float, r: int):
    """Integer 1-D weights q_a, a = -r..r, of the product kernel
    g(a,b,c) = q_a q_b q_c / 256^3: Gaussian exp(-a^2 h^2 / 2 sigma^2)
    normalised over the window, q_a = round(256 g_a) for a != 0 and
    q_0 = 256 - sum_{a != 0} q_a, so the weights sum to 256 exactly."""
    a = np.arange(-r, r + 1)
    g = np.exp(-(a.astype(np.float64) ** 2) / (2.0 * sigma_over_h ** 2))
    g /= g.sum()
    q = np.rint(256.0 * g).astype(np.int64)
    q[r] = 0
    q[r] = 256 - q.sum()
    assert q[r] >= 0
    return q.astype(np.int32)


SIN2_BITS = 16   # integer sin^2 weights: round(2^16 K)


def sin2_c0():
    """C0 of Sec. 3.1 for K(y) = sin^2(pi |y|) on the unit ball:
    1 / int_0^1 int_{B(0,1), y3 > s} K(y) dy ds.  The inner double integral
    is int_{y3 > 0} K(|y|) y3 dy = pi int_0^1 sin^2(pi t) t^3 dt
    = pi (pi^2 - 3) / (8 pi^2), so C0 = 8 pi / (pi^2 - 3)."""
    return 8.0 * math.pi / (math.pi * math.pi - 3.0)


def sin2_kernel(h: float, lam: float, bits: int = SIN2_BITS):
    """Integer stencil of the sin^2 kernel (Sec. 3.1): offsets d = (a,b,c)
    with rho = h |d| <= delta = lam sqrt(h) get round(2^bits sin^2(pi rho /
    delta)), the others 0.  Returns (k3 of shape (2R+1)^3, R), R = the largest
    integer with R h <= delta."""
    delta = lam * math.sqrt(h)
    R = int(math.floor(delta / h))
    w = 2 * R + 1
    k3 = np.zeros((w, w, w), np.int64)
    for a in range(-R, R + 1):
        for b in range(-R, R + 1):
            for c in range(-R, R + 1):
                rho = h * math.sqrt(float(a * a + b * b + c * c))
                if rho <= delta:
                    v = math.sin(math.pi * rho / delta)
                    k3[a + R, b + R, c + R] = int(round(float(1 << bits) * (v * v)))
    return k3, R


def surface_constants(sysd, p):
    """Constants of the surface term E_s = c_N sum_j chi_j (S - W_j), W = the
    integer kernel convolution of chi, S = sum of all kernel weights:

    * "gauss": g(a,b,c) = q_a q_b q_c / 256^3, S = D^3 = 256^3, c = c_N S.
      c follows from asking a grid-aligned flat interface to cost exactly
      gamma0 per unit area: per column of cross-section h^2 the plane gives
      sum_{a>0} a q_a / 256 of kernel mass, so c = gamma0 h^2 256 / S1 with
      S1 = sum_{a>0} a q_a (the role of C0 h^4 / lambda^4 in Eq. 4flip).
      Evaluated as ((gamma0 * h) * h * 256) / S1.
    * "sin2": the paper's double sum gamma0 C0 h^4 / lambda^4 sum_{j in m}
      sum_{k in w} K_jk (Sec. 3.1) with K_jk = k3 / 2^16, so
      c_N = gamma0 C0 h^4 / (lambda^4 2^16), evaluated as
      ((gamma0 * C0) * h^4) / (lambda^4 * 2^16).

    g0 = k0 / S is the kernel's centre weight (0 for sin^2)."""
    h = sysd["h"]
    h3 = h * h * h
    if p.get("kernel", "gauss") == "sin2":
        lam = float(p["sin2_lambda"])
        k3, R = sin2_kernel(h, lam)
        S = int(k3.sum())
        k0 = int(k3[R, R, R])
        h4 = h * h * h * h
        cN = ((p["gamma0"] * sin2_c0()) * h4) / (lam * lam * lam * lam * float(1 << SIN2_BITS))
        return dict(kind="sin2", cN=cN, S=S, k0=k0, k3=k3, q=None, r=R, h3=h3,
                    c=cN * S, g0=k0 / S, D3=S, lam=lam)
    sig = p["gauss_sigma"] if p["gauss_sigma"] is not None else 2.0 * h
    r = int(p["trunc_r"])
    q = surface_kernel(sig / h, r)
    S1 = int(sum(a * int(q[r + a]) for a in range(1, r + 1)))
    c = p["gamma0"] * h * h * 256.0 / float(S1)
    D3 = 256 ** 3
    k0 = int(q[r]) ** 3
    g0 = float(k0) / float(D3)
    return dict(kind="gauss", c=c, g0=g0, D3=D3, q=q, r=r, h3=h3, S1=S1,
                cN=c / D3, S=D3, k0=k0, k3=None)


# ----------------------------------------------------------------- fields

def grid_shape(sysd):
    return tuple(int(v) for v in sysd["n"])


def grid_positions(sysd):
    n, h, o = grid_shape(sysd), sysd["h"], sysd["origin"]
    ax = [o[d] + (np.arange(n[d]) + 0.5) * h for d in range(3)]
    X, Y, Z = np.meshgrid(*ax, indexing="ij")
    return np.stack([X, Y, Z], axis=-1)


def fields(sysd, p, xyz=None):
    """U (Eq. Ur), the LJ sum and E on every cell; shapes n, n, n+(3,)."""
    L = lib()
    xyz = _c64(sysd["xyz"] if xyz is None else xyz)
    n = grid_shape(sysd)
    G = n[0] * n[1] * n[2]
    lj = np.zeros(G)
    E = np.zeros((G, 3))
    L.or_grid_terms(n[0], n[1], n[2], sysd["h"], _p(_c64(sysd["origin"])),
                    len(xyz), _p(xyz), _p(_c64(sysd["sigma_sw"])),
                    _p(_c64(sysd["eps_sw"])), _p(_c64(sysd["q"])), p["rmin"],
                    _p(lj), _p(E))
    Cc = cfa_prefactor(p)
    U = p["rho_w"] * lj + Cc * np.einsum("gi,gi->g", E, E)
    return U.reshape(n), lj.reshape(n), E.reshape(n + (3,))


def point_fields(sysd, p, pts, xyz=None):
    """U, LJ sum and E at explicit points (N,3)."""
    L = lib()
    xyz = _c64(sysd["xyz"] if xyz is None else xyz)
    pts = _c64(pts).reshape(-1, 3)
    lj = np.zeros(len(pts))
    E = np.zeros((len(pts), 3))
    L.or_point_terms(len(pts), _p(pts), len(xyz), _p(xyz),
                     _p(_c64(sysd["sigma_sw"])), _p(_c64(sysd["eps_sw"])),
                     _p(_c64(sysd["q"])), p["rmin"], _p(lj), _p(E))
    U = p["rho_w"] * lj + cfa_prefactor(p) * np.einsum("gi,gi->g", E, E)
    return U, lj, E


def cell_positions(sysd, cells):
    n, h, o = grid_shape(sysd), sysd["h"], sysd["origin"]
    cells = np.asarray(cells, np.int64)
    i = cells // (n[1] * n[2])
    j = (cells // n[2]) % n[1]
    k = cells % n[2]
    return np.stack([o[0] + (i + 0.5) * h, o[1] + (j + 0.5) * h,
                     o[2] + (k + 0.5) * h], axis=-1)


# -------------------------------------------------------------- far field

def far_field_nodes(sysd, nuv=16, nt=8):
    """Quadrature for the integral over R^3 minus the box (Eq. GGR2, last
    term).  The exterior is the union of six face pyramids
    {c + s p : p on a face, s >= 1} about the box centre c.  For the face
    x = +Lx, y = c + s (Lx, Ly u, Lz v) with u, v in (-1, 1) has volume
    element Lx Ly Lz s^2 ds du dv (the same on every face); with t = 1/s in
    (0, 1] this is Lx Ly Lz t^-4 dt du dv.  Gauss-Legendre in u, v (nuv)
    and t (nt).  Returns points (M,3) and weights (M,)."""
    n, h, o = np.asarray(sysd["n"], np.float64), sysd["h"], sysd["origin"]
    Lh = 0.5 * n * h
    c0 = np.asarray(o, np.float64) + Lh
    xu, wu = np.polynomial.legendre.leggauss(nuv)
    xt, wt = np.polynomial.legendre.leggauss(nt)
    t = 0.5 * (xt + 1.0)
    wt = 0.5 * wt
    vol = Lh[0] * Lh[1] * Lh[2]
    pts, wts = [], []
    for axis in range(3):
        oth = [a for a in range(3) if a != axis]
        for sgn in (-1.0, 1.0):
            U, V, T = np.meshgrid(xu, xu, t, indexing="ij")
            WU, WV, WT = np.meshgrid(wu, wu, wt, indexing="ij")
            face = np.zeros(U.shape + (3,))
            face[..., axis] = sgn * Lh[axis]
            face[..., oth[0]] = U * Lh[oth[0]]
            face[..., oth[1]] = V * Lh[oth[1]]
            y = c0 + face / T[..., None]
            w = WU * WV * WT * vol / T ** 4
            pts.append(y.reshape(-1, 3))
            wts.append(w.reshape(-1))
    return np.concatenate(pts), np.concatenate(wts)


def far_field(sysd, p, xyz=None, nodes=None):
    """(E_far, nodes, weights, E at nodes)."""
    if nodes is None:
        nodes = far_field_nodes(sysd, p["far_nuv"], p["far_nt"])
    pts, w = nodes
    U, _, E = point_fields(sysd, p, pts, xyz)
    return float(np.dot(w, U)), pts, w, E


# ---------------------------------------------------------------- energy

def init_labels(sysd):
    """Initial binary level set (Sec. 3.1, Initial surfaces) as 0/1 solute
    labels chi = (1 - phi)/2: a loose sphere |x - c| < R, or the tight
    union of balls min_i(|x - r_i| - d_i) < 0."""
    n = grid_shape(sysd)
    init = sysd["init"]
    if init["kind"] == "sphere":
        P = grid_positions(sysd)
        c = np.asarray(init.get("center", (0.0, 0.0, 0.0)))
        r = np.sqrt(((P - c) ** 2).sum(-1))
        return (r < init["radius"]).astype(np.uint8)
    chi = np.zeros(n, np.uint8)
    xyz = _c64(sysd["xyz"])
    lib().or_init_tight(n[0], n[1], n[2], sysd["h"], _p(_c64(sysd["origin"])),
                        len(xyz), _p(xyz), _p(_c64(init["d"])), _p(chi))
    return chi


def init_labels_at(sysd, cells):
    """Tight-surface labels and phi at a list of cells."""
    n = grid_shape(sysd)
    cells = np.ascontiguousarray(cells, np.int64)
    chi = np.zeros(len(cells), np.uint8)
    phi = np.zeros(len(cells))
    xyz = _c64(sysd["xyz"])
    lib().or_init_tight_at(len(cells), _p(cells), n[0], n[1], n[2], sysd["h"],
                           _p(_c64(sysd["origin"])), len(xyz), _p(xyz),
                           _p(_c64(sysd["init"]["d"])), _p(chi), _p(phi))
    return chi, phi


def conv(chi, q):
    """W = 256^3 (g * chi), exact int64 (three 1-D passes, zero padding)."""
    chi = np.ascontiguousarray(chi, np.uint8)
    n = chi.shape
    W = np.zeros(n, np.int64)
    q = np.ascontiguousarray(q, np.int32)
    r = (len(q) - 1) // 2
    lib().or_conv(n[0], n[1], n[2], _p(chi), r, _p(q), _p(W))
    return W


def conv3(chi, k3):
    """W = sum over the full integer stencil k3 ((2R+1)^3), exact int64,
    zero padding."""
    chi = np.ascontiguousarray(chi, np.uint8)
    n = chi.shape
    W = np.zeros(n, np.int64)
    k3 = np.ascontiguousarray(k3, np.int64)
    R = (k3.shape[0] - 1) // 2
    lib().or_conv3(n[0], n[1], n[2], _p(chi), R, _p(k3), _p(W))
    return W


def conv_kernel(chi, sc):
    """W of the kernel that sc describes (separable Gaussian or stencil)."""
    return conv(chi, sc["q"]) if sc["k3"] is None else conv3(chi, sc["k3"])


def _karrays(sc):
    """(qw, k3) arrays for the C routines: exactly one is not None.  The
    caller keeps them alive across the call."""
    if sc["k3"] is None:
        return np.ascontiguousarray(sc["q"], np.int32), None
    return None, np.ascontiguousarray(sc["k3"], np.int64)


def _pp(a):
    return None if a is None else _p(a)


def surface_energy(chi, sc):
    W = conv_kernel(chi, sc)
    s = lib().or_surface_sum(chi.size, _p(np.ascontiguousarray(chi)), _p(W),
                             sc["S"])
    return sc["cN"] * s, W


def delta_e(chi, U, sc, W=None):
    """dE (Eq. dGj1/dGj2) and the candidate mask."""
    chi = np.ascontiguousarray(chi, np.uint8)
    if W is None:
        W = conv_kernel(chi, sc)
    U = _c64(U)
    n = chi.shape
    dE = np.zeros(n)
    cand = np.zeros(n, np.uint8)
    lib().or_delta_e(n[0], n[1], n[2], _p(chi), _p(W), _p(U), sc["cN"],
                     sc["S"], sc["k0"], sc["h3"], _p(dE), _p(cand))
    return dE, cand


def select(chi, U, sc, rule="bricks"):
    """One round's selection of the parallel rule: (sel mask, keys).
    rule "bricks" is the rule the relaxation uses; "cells" the finer cube
    rule it contains."""
    dE, cand = delta_e(chi, U, sc)
    n = chi.shape
    sel = np.zeros(n, np.uint8)
    keys = np.zeros(n, np.uint64)
    fn = lib().or_select if rule == "bricks" else lib().or_select_cells
    fn(n[0], n[1], n[2], _p(cand), _p(dE), sc["r"], _p(sel), _p(keys))
    return sel, keys, dE, cand


def flip_energy_total(chi, U, sc):
    """c sum chi (1 - w) + h^3 sum_{solvent} U (Eq. 4flip, first two terms)."""
    chi = np.ascontiguousarray(chi, np.uint8)
    n = chi.shape
    qw, k3 = _karrays(sc)
    return lib().or_energy(n[0], n[1], n[2], _p(chi), _p(_c64(U)), sc["r"],
                           _pp(qw), _pp(k3), sc["cN"], sc["S"], sc["h3"])


def blsm_parallel(chi, U, sc, max_rounds=100000, verify=False,
                  record_rounds=False):
    """Rounds of the parallel brick-leader rule to a local minimum, in place.
    Returns dict(rounds, flips, dE_sum, verify_err, round_flips)."""
    chi_c = np.ascontiguousarray(chi, np.uint8)
    n = chi_c.shape
    flips = C.c_int64(0)
    dsum = C.c_double(0.0)
    verr = C.c_double(0.0)
    rf = np.zeros(max_rounds if record_rounds else 1, np.int64)
    qw, k3 = _karrays(sc)
    U64 = _c64(U)
    rounds = lib().or_blsm_parallel(
        n[0], n[1], n[2], _p(chi_c), _p(U64), sc["r"], _pp(qw), _pp(k3),
        sc["cN"], sc["S"], sc["k0"], sc["h3"], max_rounds, C.byref(flips),
        C.byref(dsum), _p(rf) if record_rounds else None, int(verify),
        C.byref(verr))
    if chi_c is not chi:
        chi[...] = chi_c
    out = dict(rounds=rounds, flips=flips.value, dE_sum=dsum.value,
               verify_err=verr.value)
    if record_rounds:
        out["round_flips"] = rf[:rounds].copy()
    return out


def blsm_heap(chi, U, sc, max_flips=1 << 40, verify=False):
    """Literal serial min-heap flipping (Steps 2.1-2.2), in place."""
    chi_c = np.ascontiguousarray(chi, np.uint8)
    n = chi_c.shape
    dsum = C.c_double(0.0)
    verr = C.c_double(0.0)
    qw, k3 = _karrays(sc)
    U64 = _c64(U)
    flips = lib().or_blsm_heap(n[0], n[1], n[2], _p(chi_c), _p(U64),
                               sc["r"], _pp(qw), _pp(k3), sc["cN"], sc["S"], sc["k0"],
                               sc["h3"], max_flips, C.byref(dsum),
                               int(verify), C.byref(verr))
    if chi_c is not chi:
        chi[...] = chi_c
    return dict(flips=flips, dE_sum=dsum.value, verify_err=verr.value)


def ss_terms(sysd, p, xyz=None):
    """G_ss (bonds, LJ, Coulomb) and its gradient (Eq. Gss)."""
    xyz = _c64(sysd["xyz"] if xyz is None else xyz)
    N = len(xyz)
    e = np.zeros(3)
    g = np.zeros((N, 3))
    coul = bjerrum(p["temperature"]) / p["eps_ss"]
    b = np.ascontiguousarray(sysd["bonds"], np.int32)
    lib().or_ss(N, _p(xyz), _p(_c64(sysd["sigma_ss"])), _p(_c64(sysd["eps_ss"])),
                _p(_c64(sysd["q"])), len(b), _p(b), _p(_c64(sysd["bond_k"])),
                _p(_c64(sysd["bond_r0"])), coul, _p(e), _p(g))
    return e, g


def bonded_terms(sysd, xyz=None):
    """Bending and torsion energies of G_ss (Eq. Gss) and their gradient.

    Bend (i, j, k): 1/2 B (theta - theta0)^2, theta the angle between
    r_i - r_j and r_k - r_j.  Torsion (i, j, k, l): sum over n = 0..6 of
    C_n [1 + cos(n tau - psi_n)], tau the angle between u = q1 x q2 and
    v = q2 x q3 with q1 = r_j - r_i, q2 = r_k - r_j, q3 = r_l - r_k.  The
    gradients follow the appendix ("Force calculations of molecular
    mechanical interactions"): B (theta - theta0) grad theta, and
    dW/dLambda grad Lambda with Lambda = cos tau = u.v / (|u| |v|), which
    holds for phases psi_n of 0 or pi.  A bend with sin theta = 0 adds no
    gradient; a torsion with u or v of zero length adds nothing."""
    xyz = _c64(sysd["xyz"] if xyz is None else xyz).reshape(-1, 3)
    g = np.zeros_like(xyz)
    eb = 0.0
    angles = np.asarray(sysd.get("angles", np.zeros((0, 3), int))).reshape(-1, 3)
    for m, (i, j, k) in enumerate(angles):
        a = xyz[i] - xyz[j]
        b = xyz[k] - xyz[j]
        la, lb = np.linalg.norm(a), np.linalg.norm(b)
        c = float(np.dot(a, b) / (la * lb))
        c = min(1.0, max(-1.0, c))
        th = math.acos(c)
        d = th - float(sysd["angle_theta0"][m])
        B = float(sysd["angle_B"][m])
        eb += 0.5 * B * d * d
        sn = math.sin(th)
        if sn < 1e-12:
            continue
        dth_da = -(b / (la * lb) - c * a / (la * la)) / sn
        dth_db = -(a / (la * lb) - c * b / (lb * lb)) / sn
        g[i] += B * d * dth_da
        g[k] += B * d * dth_db
        g[j] -= B * d * (dth_da + dth_db)
    et = 0.0
    tors = np.asarray(sysd.get("torsions", np.zeros((0, 4), int))).reshape(-1, 4)
    for m, (i, j, k, l) in enumerate(tors):
        q1, q2, q3 = xyz[j] - xyz[i], xyz[k] - xyz[j], xyz[l] - xyz[k]
        u, v = np.cross(q1, q2), np.cross(q2, q3)
        lu, lv = np.linalg.norm(u), np.linalg.norm(v)
        if lu * lv < 1e-24:
            continue
        lam = float(np.dot(u, v) / (lu * lv))
        lam = min(1.0, max(-1.0, lam))
        tau = math.acos(lam)
        C = np.asarray(sysd["torsion_C"][m], np.float64)
        psi = np.asarray(sysd["torsion_psi"][m], np.float64)
        et += float(np.sum(C * (1.0 + np.cos(np.arange(7) * tau - psi))))
        cps = np.cos(psi)
        # dW/dLambda = sum_n C_n cos(psi_n) T_n'(Lambda), written out
        dW = ((C[1] * cps[1] - 3 * C[3] * cps[3] + 5 * C[5] * cps[5])
              + lam * (4 * C[2] * cps[2] - 16 * C[4] * cps[4] + 36 * C[6] * cps[6])
              + lam ** 2 * (12 * C[3] * cps[3] - 60 * C[5] * cps[5])
              + lam ** 3 * (32 * C[4] * cps[4] - 192 * C[6] * cps[6])
              + lam ** 4 * (80 * C[5] * cps[5])
              + lam ** 5 * (192 * C[6] * cps[6]))
        dL_du = (v * lu * lu - np.dot(u, v) * u) / (lu ** 3 * lv)
        dL_dv = (u * lv * lv - np.dot(u, v) * v) / (lu * lv ** 3)
        dL_dq1 = np.cross(q2, dL_du)
        dL_dq2 = np.cross(dL_du, q1) + np.cross(q3, dL_dv)
        dL_dq3 = np.cross(dL_dv, q2)
        g[i] += dW * (-dL_dq1)
        g[j] += dW * (dL_dq1 - dL_dq2)
        g[k] += dW * (dL_dq2 - dL_dq3)
        g[l] += dW * dL_dq3
    return eb, et, g


def energy_terms(sysd, p, chi, xyz=None, U=None, E=None):
    """All terms of G = G_VISM + G_ss (Eq. freeenergyfn, Eq. 4flip):
    surface, vdW, CFA (solvent cells), far field, solute-solute, total."""
    sc = surface_constants(sysd, p)
    if U is None:
        U, lj, E = fields(sysd, p, xyz)
    else:
        lj = None
    chi = np.asarray(chi, np.uint8)
    es, _ = surface_energy(chi, sc)
    solv = chi == 0
    Cc = cfa_prefactor(p)
    cfa_pt = Cc * np.einsum("...i,...i->...", E, E)
    vol = sc["h3"] * float(U[solv].sum())
    cfa = sc["h3"] * float(cfa_pt[solv].sum())
    far = far_field(sysd, p, xyz)[0] if p["far_field"] else 0.0
    ess, _ = ss_terms(sysd, p, xyz)
    e_bend, e_tors, _ = bonded_terms(sysd, xyz)
    ss = float(ess.sum()) + e_bend + e_tors
    return dict(surf=es, vdw=vol - cfa, cfa=cfa, far=far, ss=ss,
                total=es + vol + far + ss, vol=vol)


def gradient(sysd, p, chi, xyz=None, E=None):
    """dG/dr_n for every atom with the interface fixed: grid volume term,
    far field and G_ss (Eq. GradientG, as the exact derivative)."""
    L = lib()
    xyz = _c64(sysd["xyz"] if xyz is None else xyz)
    N = len(xyz)
    n = grid_shape(sysd)
    if E is None:
        _, _, E = fields(sysd, p, xyz)
    Cc = cfa_prefactor(p)
    sig, eps, q = (_c64(sysd["sigma_sw"]), _c64(sysd["eps_sw"]),
                   _c64(sysd["q"]))
    g = np.zeros((N, 3))
    L.or_grid_grad(n[0], n[1], n[2], sysd["h"], _p(_c64(sysd["origin"])),
                   _p(np.ascontiguousarray(chi, np.uint8)),
                   _p(_c64(E).reshape(-1, 3)), N, _p(xyz), _p(sig), _p(eps),
                   _p(q), p["rho_w"], Cc, p["rmin"], _p(g))
    if p["far_field"]:
        _, pts, w, Ef = far_field(sysd, p, xyz)
        gf = np.zeros((N, 3))
        L.or_point_grad(len(pts), _p(_c64(pts)), _p(_c64(w)), _p(_c64(Ef)), N,
                        _p(xyz), _p(sig), _p(eps), _p(q), p["rho_w"], Cc,
                        p["rmin"], _p(gf))
        g += gf
    _, gss = ss_terms(sysd, p, xyz)
    _, _, gbt = bonded_terms(sysd, xyz)
    return g + gss + gbt


# ------------------------------------------------------------ relaxation

def _inside(sysd, xyz):
    lo = np.asarray(sysd["origin"], np.float64)
    hi = lo + np.asarray(sysd["n"], np.float64) * sysd["h"]
    return bool(np.all((xyz > lo) & (xyz < hi)))


def relax(sysd, p, opts, chi=None, xyz=None, log=None, fields_fp32=False):
    """Full VESIS iteration (Steps 1-5): flips to a local minimum of the
    interface at fixed atoms (Step 2), then adaptive-mobility gradient
    steps of the atoms at fixed interface (Step 3, Eq. moveatoms with
    M_nl = omega M, omega from Eq. adjustmml), with the accept/shrink rule
    of Step 3.4, until the gradient test (Step 3.2), the energy test held
    for `window` steps (Steps 4-5) or k_max.

    Readings where the paper is silent: delta G* = frac * |G_old|; the
    energy change of Steps 4-5 is between consecutive accepted iterates;
    a trial that moves an atom out of the box, or whose energy is not
    finite, is rejected like an energy increase;
    at most max_gd_retries shrinks per step (then status 2, not
    converged).  Status: 0 gradient converged, 1 energy converged,
    2 not converged (k_max or retry cap).

    fields_fp32: the energy density U and the field E on the grid are
    rounded to FP32 where they are stored (computed in FP64, then kept as
    FP32 values, "FP32 fields, FP64 totals"); every sum, flip energy,
    gradient and the accept test stay FP64."""
    xyz = _c64(sysd["xyz"] if xyz is None else xyz).copy()
    chi = init_labels(sysd) if chi is None else np.array(chi, np.uint8)
    sc = surface_constants(sysd, p)

    def fields_stored(x):
        U, _, E = fields(sysd, p, x)
        if fields_fp32:
            U = U.astype(np.float32).astype(np.float64)
            E = E.astype(np.float32).astype(np.float64)
        return U, E

    U, E = fields_stored(xyz)
    G_prev = energy_terms(sysd, p, chi, xyz, U, E)["total"]
    M, ncnt, stable, k = opts["M0"], 0, 0, 0
    status = 2
    hist = []
    while k < opts["max_outer"]:
        br = blsm_parallel(chi, U, sc, opts["max_flip_rounds"])
        grad = gradient(sysd, p, chi, xyz, E)
        gmax = float(np.abs(grad).max()) if grad.size else 0.0
        if gmax < opts["tol_grad"]:
            status = 0
            break
        G_old = energy_terms(sysd, p, chi, xyz, U, E)["total"]
        omega = 1.0 / gmax
        retries = 0
        while True:
            x_new = xyz - omega * M * grad
            U_n, E_n = fields_stored(x_new)
            G_new = energy_terms(sysd, p, chi, x_new, U_n, E_n)["total"]
            dG = G_new - G_old
            dGs = opts["dgstar_frac"] * abs(G_old)
            if (dG > dGs or (ncnt >= opts["ncnt_star"] and 0.0 < dG <= dGs)
                    or not math.isfinite(G_new) or not _inside(sysd, x_new)):
                M *= opts["alpha"]
                ncnt = 0
                retries += 1
                if retries > opts["max_gd_retries"]:
                    break
                continue
            ncnt += 1
            break
        if retries > opts["max_gd_retries"]:
            status = 2
            break
        xyz, U, E = x_new, U_n, E_n
        d_abs = abs(G_new - G_prev)
        d_rel = d_abs / abs(G_new) if G_new != 0.0 else math.inf
        G_prev = G_new
        k += 1
        hist.append(dict(k=k, G=G_new, G_old=G_old, M=M, ncnt=ncnt,
                         rounds=br["rounds"], flips=br["flips"],
                         retries=retries, gmax=gmax))
        if log:
            log(hist[-1])
        if d_abs < opts["tol_energy"] or d_rel < opts["tol_energy"]:
            stable += 1
            if stable >= opts["window"]:
                status = 1
                break
        else:
            stable = 0
    return dict(status=status, xyz=xyz, chi=chi, iters=k, history=hist,
                G=G_prev)


# ------------------------------------------------------------ closed form

def sphere_energy(R, sigma, eps, q, p):
    """G(R) of one atom inside a spherical cavity of radius R (closed form
    of Eq. G_VISM over R^3 minus the ball): 4 pi gamma0 R^2
    + 16 pi rho_w eps [sigma^12 / (9 R^9) - sigma^6 / (3 R^3)]
    + (l_B / 2) q^2 (1/eps_w - 1/eps_m) / R."""
    lb = bjerrum(p["temperature"])
    surf = 4.0 * math.pi * p["gamma0"] * R * R
    lj = 16.0 * math.pi * p["rho_w"] * eps * (sigma ** 12 / (9.0 * R ** 9)
                                              - sigma ** 6 / (3.0 * R ** 3))
    cfa = 0.5 * lb * q * q * (1.0 / p["eps_w"] - 1.0 / p["eps_m"]) / R
    return surf + lj + cfa, (surf, lj, cfa)


def sphere_minimum(sigma, eps, q, p, lo=1.0, hi=10.0):
    from scipy.optimize import minimize_scalar
    r = minimize_scalar(lambda R: sphere_energy(R, sigma, eps, q, p)[0],
                        bounds=(lo, hi), method="bounded",
                        options=dict(xatol=1e-10))
    return float(r.x), float(r.fun)
