"""Seeded synthetic inputs for the VESIS hot path.

This module only draws random solute geometries and parameters and states
grid specifications. It holds none of the method's arithmetic (no energies,
no kernels, no labels): both the CUDA path and the CPU oracle take their
inputs from here, and nothing else is shared between them.

Units follow the paper's statement of the problem (Sec. 2, Table 1):
lengths in Angstrom, energies in k_B T, charges in units of e.  Parameters
quoted in kJ/mol are converted with k_B T = R T at the system temperature.

A system is a plain dict:
    xyz        (N,3) float64   atom positions
    sigma_sw   (N,)  float64   solute-solvent LJ sigma
    eps_sw     (N,)  float64   solute-solvent LJ epsilon (kBT)
    q          (N,)  float64   partial charges (e)
    sigma_ss   (N,)  float64   solute-solute LJ sigma (mixed pairwise)
    eps_ss     (N,)  float64   solute-solute LJ epsilon (kBT)
    bonds      (B,2) int32     bonded pairs (harmonic, also 1-2 exclusions)
    bond_k     (B,)  float64   spring constants A (kBT/A^2)
    bond_r0    (B,)  float64   equilibrium lengths (A)
    n          (3,)  int       grid cells per axis (z fastest in memory)
    h          float           grid spacing (A)
    origin     (3,)  float64   lower box corner; cell centres at origin+(i+1/2)h
    init       dict            initial surface: {"kind": "sphere", "radius": R}
                               or {"kind": "tight", "d": (N,) radii}
"""
from __future__ import annotations

import math

import numpy as np

# CODATA 2018 gas constant (kJ mol^-1 K^-1): converts the kJ/mol epsilons
# quoted for the synthetic workloads into kBT.
_R_KJ = 8.314462618e-3


def kbt_kj_per_mol(temperature: float = 298.0) -> float:
    return _R_KJ * temperature


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def _empty_bonds():
    return (np.zeros((0, 2), np.int32), np.zeros(0), np.zeros(0))


def _system(xyz, sigma, eps, q, n, h, origin, init, bonds=None,
            sigma_ss=None, eps_ss=None):
    xyz = np.ascontiguousarray(xyz, dtype=np.float64).reshape(-1, 3)
    N = xyz.shape[0]
    b, bk, br0 = _empty_bonds() if bonds is None else bonds
    return dict(
        xyz=xyz,
        sigma_sw=np.ascontiguousarray(np.broadcast_to(sigma, (N,)), np.float64),
        eps_sw=np.ascontiguousarray(np.broadcast_to(eps, (N,)), np.float64),
        q=np.ascontiguousarray(np.broadcast_to(q, (N,)), np.float64),
        sigma_ss=np.ascontiguousarray(np.broadcast_to(
            sigma if sigma_ss is None else sigma_ss, (N,)), np.float64),
        eps_ss=np.ascontiguousarray(np.broadcast_to(
            eps if eps_ss is None else eps_ss, (N,)), np.float64),
        bonds=np.ascontiguousarray(b, np.int32).reshape(-1, 2),
        bond_k=np.ascontiguousarray(bk, np.float64),
        bond_r0=np.ascontiguousarray(br0, np.float64),
        n=np.array(n, dtype=np.int64).reshape(3),
        h=float(h),
        origin=np.array(origin, dtype=np.float64).reshape(3),
        init=init,
    )


def cubic_grid(n: int, h: float):
    """Box (-L, L)^3 with L = n h / 2, cell-centred (Sec. 3.1)."""
    L = 0.5 * n * h
    return (n, n, n), h, (-L, -L, -L)


# ---------------------------------------------------------------- workloads

def single_ion(n: int = 64, h: float = 0.25, sigma: float = 3.5,
               eps_kj: float = 0.65, q: float = 1.0, r_init: float = 7.0,
               temperature: float = 298.0, center=(0.0, 0.0, 0.0)):
    """One charged LJ atom at the box centre, initial sphere of radius r_init.

    Default: 64^3 grid, h = 0.25 A, box [-8, 8]^3, sigma 3.5 A,
    eps 0.65 kJ/mol, Q = +1 e, chi_0 = 7 A sphere.
    """
    nn, hh, o = cubic_grid(n, h)
    eps = eps_kj / kbt_kj_per_mol(temperature)
    return _system([center], sigma, eps, q, nn, hh, o,
                   {"kind": "sphere", "radius": float(r_init)})


def two_atom(d: float, charges=(1.0, -1.0), n: int = 128, h: float = 0.2,
             sigma: float = 3.5, eps_kj: float = 0.65, bond_k: float = 800.0,
             temperature: float = 298.0):
    """Two bonded atoms on the x axis at +-d/2 (separation sweep 4-12 A).

    Default 128^3 grid at h = 0.2 A (box [-12.8, 12.8]^3).  The harmonic
    bond (A = 800 kBT/A^2, r0 = d) holds the separation, as in the paper's
    two-atom molecule.  Initial surface: tight, d_i = sigma_i.
    """
    nn, hh, o = cubic_grid(n, h)
    eps = eps_kj / kbt_kj_per_mol(temperature)
    xyz = [[-0.5 * d, 0.0, 0.0], [0.5 * d, 0.0, 0.0]]
    bonds = (np.array([[0, 1]], np.int32), np.array([bond_k]),
             np.array([float(d)]))
    return _system(xyz, sigma, eps, np.asarray(charges, np.float64), nn, hh,
                   o, {"kind": "tight", "d": np.full(2, sigma)}, bonds)


def two_atom_molecule(r0: float, start: float, n: int = 64, h: float = 0.25):
    """The paper's uncharged two-atom molecule (Sec. 5.2): sigma 3.57 A,
    eps 0.431 kBT, A = 800 kBT/A^2, box (-8, 8)^3, atoms at (+-start, 0, 0).
    The grid spacing is not given in the paper; 64^3 at h = 0.25 A here."""
    nn, hh, o = cubic_grid(n, h)
    xyz = [[start, 0.0, 0.0], [-start, 0.0, 0.0]]
    bonds = (np.array([[0, 1]], np.int32), np.array([800.0]),
             np.array([float(r0)]))
    return _system(xyz, 3.57, 0.431, 0.0, nn, hh, o,
                   {"kind": "tight", "d": np.full(2, 3.57)}, bonds)


def _confined_walk(rng, n, step, radius, min_dist, center, tries=100):
    """Self-avoiding chain with fixed bond length `step`, kept inside the
    ball |x - center| <= radius; a new bead must stay min_dist away from
    every earlier bead except its predecessor.  After `tries` failures the
    walk backs up and regrows."""
    pts = np.zeros((n, 3))
    pts[0] = center
    i = 1
    fails = 0
    budget = 2000 * n + 100000        # regrowths before giving up
    while i < n:
        budget -= 1
        if budget < 0:
            raise RuntimeError("confined walk found no room: the ball is too dense")
        prev = pts[i - 1]
        placed = False
        for _ in range(tries):
            d = rng.normal(size=3)
            d *= step / np.linalg.norm(d)
            p = prev + d
            if np.linalg.norm(p - center) > radius:
                continue
            if i >= 2:
                dd = np.linalg.norm(pts[:i - 1] - p, axis=1)
                if dd.min() < min_dist:
                    continue
            pts[i] = p
            placed = True
            break
        if placed:
            i += 1
            fails = 0
        else:
            fails += 1
            i = max(1, i - min(i - 1, 2 + fails))
    return pts


def _side_atoms(rng, backbone, others_min, jitter, tries=200):
    """One side atom per backbone bead at bead + jitter*N(0,I)/sqrt(3),
    at least `others_min` from every atom but its parent and 1 A from it
    (the jitter scale grows by 20% every 50 failed draws)."""
    nb = len(backbone)
    allp = np.zeros((2 * nb, 3))
    allp[:nb] = backbone
    out = np.zeros_like(backbone)
    for i, b in enumerate(backbone):
        scale = jitter
        cnt = nb + i
        for t in range(tries):
            p = b + scale * rng.normal(size=3) / math.sqrt(3.0)
            if np.linalg.norm(p - b) < 1.0:
                continue
            dd = np.linalg.norm(allp[:cnt] - p, axis=1)
            dd[i] = np.inf
            if dd.min() >= others_min:
                break
            if t % 50 == 49:
                scale *= 1.2
        out[i] = p
        allp[cnt] = p
    return out


def globule(n_atoms: int, rng, center=(0.0, 0.0, 0.0), density: float = 0.05,
            radius: float | None = None):
    """Protein-like random-walk globule: n/2 backbone beads (3.8 A steps,
    self-avoiding at 2.5 A, confined to the ball holding `density` atoms per
    A^3) plus one side atom jittered 1.5 A around each of the first n/2
    beads (the backbone takes the odd atom)."""
    nb = (n_atoms + 1) // 2
    ns = n_atoms - nb
    if radius is None:
        radius = (3.0 * n_atoms / (4.0 * math.pi * density)) ** (1.0 / 3.0)
        radius = max(radius, 2.0 * 3.8)     # room for a few 3.8 A steps
    center = np.asarray(center, np.float64)
    bb = _confined_walk(rng, nb, 3.8, radius, 2.5, center)
    side = _side_atoms(rng, bb[:ns], 2.0, 1.5)
    xyz = np.concatenate([bb, side], axis=0)
    bonds = [(i, i + 1) for i in range(nb - 1)] + [(i, nb + i) for i in range(ns)]
    bonds = np.asarray(bonds, np.int32)
    r0 = np.linalg.norm(xyz[bonds[:, 0]] - xyz[bonds[:, 1]], axis=1)
    return xyz, bonds, r0, radius


def _params(rng, n, temperature, net_charge):
    kbt = kbt_kj_per_mol(temperature)
    sigma = rng.uniform(3.0, 4.0, n)
    eps = rng.uniform(0.1, 0.9, n) / kbt
    q = rng.normal(0.0, 0.35, n)
    q += (net_charge - q.sum()) / n          # uniform shift to the net charge
    return sigma, eps, q


def protein_like(n_atoms: int = 2000, n: int = 256, h: float = 0.4,
                 seed: int = 0, temperature: float = 298.0,
                 net_charge: float = -3.0):
    """Synthetic protein-like solute: random-walk globule of n_atoms atoms,
    sigma ~ U[3, 4] A, eps ~ U[0.1, 0.9] kJ/mol, q ~ N(0, 0.35) shifted to
    the net charge, bonds A = 800 kBT/A^2 at their initial length, centred at
    the origin; default 256^3 grid at h = 0.4 A; tight initial surface with
    d_i = sigma_i."""
    rng = _rng(seed)
    xyz, bonds, r0, _ = globule(n_atoms, rng)
    xyz -= xyz.mean(axis=0)
    sigma, eps, q = _params(rng, n_atoms, temperature, net_charge)
    nn, hh, o = cubic_grid(n, h)
    return _system(xyz, sigma, eps, q, nn, hh, o,
                   {"kind": "tight", "d": sigma.copy()},
                   (bonds, np.full(len(bonds), 800.0), r0))


def small_protein(index: int, seed: int = 5, atoms=(60, 400), h: float = 0.4,
                  margin: float = 8.0):
    """The `index`-th solute of a seeded set of small protein-like solutes
    (the many-solute service the batched form is for): atom count
    log-uniform in `atoms`, the protein-like parameter distributions, and
    the smallest cubic grid at spacing h whose side is a multiple of 16
    cells and holds every atom `margin` A inside the box."""
    rng = np.random.default_rng([seed, index])
    na = int(round(np.exp(rng.uniform(np.log(atoms[0]), np.log(atoms[1])))))
    s = int(rng.integers(1 << 31))
    sd = protein_like(n_atoms=na, n=16, h=h, seed=s)
    ext = float(np.abs(sd["xyz"]).max()) + margin
    n = 16 * int(math.ceil(2.0 * ext / (16.0 * h)))
    return protein_like(n_atoms=na, n=n, h=h, seed=s)


def two_domain_complex(n_per: int = 10000, n: int = 384, h: float = 0.4,
                       seed: int = 2, gap: float = 6.0,
                       temperature: float = 298.0):
    """Two random-walk globules of n_per atoms each, their confinement balls
    `gap` apart along the body diagonal; 384^3 grid at h = 0.4 A."""
    rng = _rng(seed)
    radius = (3.0 * n_per / (4.0 * math.pi * 0.05)) ** (1.0 / 3.0)
    off = (radius + 0.5 * gap) / math.sqrt(3.0)
    parts, bl, r0l = [], [], []
    base = 0
    for s in (-1.0, 1.0):
        xyz, bonds, r0, _ = globule(n_per, rng, center=(s * off,) * 3,
                                    radius=radius)
        parts.append(xyz)
        bl.append(bonds + base)
        r0l.append(r0)
        base += n_per
    xyz = np.concatenate(parts)
    bonds = np.concatenate(bl)
    r0 = np.concatenate(r0l)
    sigma, eps, q = _params(rng, len(xyz), temperature, -3.0)
    nn, hh, o = cubic_grid(n, h)
    return _system(xyz, sigma, eps, q, nn, hh, o,
                   {"kind": "tight", "d": sigma.copy()},
                   (bonds, np.full(len(bonds), 800.0), r0))


def host_guest(index: int, seed: int = 1, h: float = 0.3, temperature: float = 298.0,
               density: float = 0.05):
    """System `index` (0..63) of the batched host-guest set: a host drawn
    log-uniform in [150, 4000] atoms and a guest in [20, 80] atoms, both
    confined random walks at the protein-like density; the guest's
    confinement ball sits in a random direction, U[5, 15] A beyond the
    host's.  The grid is the smallest multiple of 16 cells, at least 64, at
    spacing h whose half-width covers every atom plus 8 A.  At h = 0.3 A
    that is 160-320 cells per axis for indices 0..63 with seed 1 (a 4,000-
    atom host alone spans about 54 A, and even the smallest pair with its
    offset spans about 45 A).  Each system draws from its own stream spawned
    from `seed`; net charge 0, tight initial surface."""
    ss = np.random.SeedSequence(seed).spawn(index + 1)[index]
    rng = np.random.Generator(np.random.PCG64(ss))
    n_host = int(round(math.exp(rng.uniform(math.log(150.0), math.log(4000.0)))))
    n_guest = int(rng.integers(20, 81))
    offset = float(rng.uniform(5.0, 15.0))
    u = rng.normal(size=3)
    u /= np.linalg.norm(u)
    ball = lambda m: max((3.0 * m / (4.0 * math.pi * density)) ** (1.0 / 3.0), 2.0 * 3.8)
    dist = ball(n_host) + offset + ball(n_guest)
    hx, hb, hr0, _ = globule(n_host, rng, density=density)
    gx, gb, gr0, _ = globule(n_guest, rng, center=u * dist, density=density)
    xyz = np.concatenate([hx, gx], axis=0)
    lo, hi = xyz.min(axis=0), xyz.max(axis=0)
    xyz -= 0.5 * (lo + hi)
    need = float(np.abs(xyz).max()) + 8.0
    n = 64
    while 0.5 * n * h < need:
        n += 16
    bonds = np.concatenate([hb, gb + n_host], axis=0)
    r0 = np.concatenate([hr0, gr0])
    sigma, eps, q = _params(rng, n_host + n_guest, temperature, 0.0)
    nn, hh, o = cubic_grid(n, h)
    sysd = _system(xyz, sigma, eps, q, nn, hh, o, {"kind": "tight", "d": sigma.copy()},
                   (bonds, np.full(len(bonds), 800.0), r0))
    sysd.update(n_host=n_host, n_guest=n_guest)
    return sysd


def with_bends_torsions(sysd, B: float = 60.0, C=(0.0, 0.6, 0.2, 0.8, 0.0, 0.0, 0.0),
                        theta0_shift: float = 0.0):
    """A copy of a system with bending and torsion terms (Eq. Gss) on its
    bond graph: a bend for every pair of bonds sharing an atom (theta0 the
    current angle plus theta0_shift, B in kBT/rad^2), a torsion for every
    path i-j-k-l of three bonds (constants C_0..C_6 in kBT, phases 0 for odd
    and pi for even n, the convention the paper describes)."""
    out = dict(sysd)
    xyz = np.asarray(sysd["xyz"], np.float64)
    b = np.asarray(sysd["bonds"]).reshape(-1, 2)
    nb = [[] for _ in range(len(xyz))]
    for i, j in b:
        nb[int(i)].append(int(j))
        nb[int(j)].append(int(i))
    angles, th0 = [], []
    for j in range(len(xyz)):
        ns = sorted(nb[j])
        for x in range(len(ns)):
            for y in range(x + 1, len(ns)):
                i, k = ns[x], ns[y]
                u, v = xyz[i] - xyz[j], xyz[k] - xyz[j]
                c = np.dot(u, v) / (np.linalg.norm(u) * np.linalg.norm(v))
                angles.append((i, j, k))
                th0.append(min(math.pi, max(0.0, math.acos(min(1.0, max(-1.0, c))) + theta0_shift)))
    tors = []
    for j, k in b:
        j, k = int(j), int(k)
        for i in sorted(nb[j]):
            if i == k:
                continue
            for l in sorted(nb[k]):
                if l in (j, i):
                    continue
                tors.append((i, j, k, l))
    n_t = len(tors)
    psi = np.array([0.0 if n % 2 else math.pi for n in range(7)])
    out["angles"] = np.array(angles, np.int32).reshape(-1, 3)
    out["angle_B"] = np.full(len(angles), float(B))
    out["angle_theta0"] = np.array(th0, np.float64)
    out["torsions"] = np.array(tors, np.int32).reshape(-1, 4)
    out["torsion_C"] = np.tile(np.asarray(C, np.float64), (n_t, 1))
    out["torsion_psi"] = np.tile(psi, (n_t, 1))
    return out


def subset(sysd, idx):
    """The atoms `idx` of a system alone on the same grid (bonds between
    them kept, renumbered)."""
    idx = np.asarray(idx, np.int64)
    out = dict(sysd)
    for k in ("xyz", "sigma_sw", "eps_sw", "q", "sigma_ss", "eps_ss"):
        out[k] = np.asarray(sysd[k])[idx].copy()
    where = {int(a): i for i, a in enumerate(idx)}
    b = np.asarray(sysd["bonds"]).reshape(-1, 2)
    keep = [m for m in range(len(b)) if int(b[m, 0]) in where and int(b[m, 1]) in where]
    out["bonds"] = np.array([[where[int(b[m, 0])], where[int(b[m, 1])]] for m in keep],
                            np.int32).reshape(-1, 2)
    out["bond_k"] = np.asarray(sysd["bond_k"])[keep].copy()
    out["bond_r0"] = np.asarray(sysd["bond_r0"])[keep].copy()
    out["init"] = {"kind": "tight", "d": out["sigma_sw"].copy()}
    return out


def random_cluster(n_atoms: int, n: int, h: float, seed: int,
                   temperature: float = 298.0, net_charge: float = 0.0,
                   density: float = 0.05):
    """Small random-walk cluster centred in an n^3 box (test sizes)."""
    rng = _rng(seed)
    xyz, bonds, r0, _ = globule(n_atoms, rng, density=density)
    xyz -= xyz.mean(axis=0)
    sigma, eps, q = _params(rng, n_atoms, temperature, net_charge)
    nn, hh, o = cubic_grid(n, h)
    return _system(xyz, sigma, eps, q, nn, hh, o,
                   {"kind": "tight", "d": sigma.copy()},
                   (bonds, np.full(len(bonds), 800.0), r0))


def random_labels(n, seed: int, p: float = 0.5):
    """Uniform random 0/1 label field of shape n (z fastest)."""
    rng = _rng(seed)
    return (rng.random(tuple(int(v) for v in n)) < p).astype(np.uint8)


def random_field(n, seed: int, scale: float = 1.0):
    """Smooth-free random float32 field of shape n, N(0, scale^2)."""
    rng = _rng(seed)
    return (scale * rng.normal(size=tuple(int(v) for v in n))).astype(np.float32)
