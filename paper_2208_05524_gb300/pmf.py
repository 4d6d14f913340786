"""Potential of mean force of two solute groups (the paper's appendix,
"Potentials of Mean Force"; Sec. 5.1 for the two-plate curves).

At separation d the interface is relaxed with the atoms fixed (the flip
sweep from a tight or a loose start: the two branches of the paper's
hysteresis), and each part of the free energy is compared with its value
for the two groups relaxed alone (the d -> infinity limit):

  geom(d) = G_geom[Gamma_d] - G_geom[Gamma_I] - G_geom[Gamma_II]
  vdW(d)  = G_vdW[Gamma_d]  - (same for I, II) + cross-group solute LJ
  elec(d) = G_elec[Gamma_d] - (same for I, II) + cross-group Coulomb

with G_geom the surface term, G_vdW the solvent LJ term and G_elec the CFA
term inside the box; the far-field integral outside the box is reported as
its own part.  The cross-group pair sums are the system's solute-solute LJ
and Coulomb minus those of each group alone (bonds stay inside a group).
Every energy comes from the CUDA library; this module only combines the
returned numbers.
"""
from __future__ import annotations

import numpy as np

PARTS = ("geom", "vdw", "elec", "far")


def relaxed_parts(S, chi, U, E, xyz, start, radius=0.0, center=None, max_rounds=100000):
    """Moves the system's atoms to xyz, relaxes the labels from `start`
    ('tight' or 'loose': a sphere of `radius` about `center`), and returns
    the parts and the solute-solute pair sums of the relaxed state."""
    S.set_positions(xyz)
    S.energy_field(U, E)
    if start == "tight":
        S.init_labels(chi, "tight")
    else:
        S.init_labels(chi, "sphere", radius=radius, center=center)
    r = S.blsm_relax(chi, U, E, max_rounds=max_rounds)
    t = r["terms"]
    ss = S.ss_terms()
    return dict(geom=t["surf"], vdw=t["vdw"], elec=t["cfa"], far=t["far"],
                lj=ss["lj"], coulomb=ss["coulomb"], rounds=r["rounds"], total=t["total"])


def combine(pair, alone):
    """PMF parts at one separation from the pair's relaxed parts and the
    parts of each group relaxed alone (a list of two)."""
    out = {k: pair[k] - sum(a[k] for a in alone) for k in PARTS}
    out["vdw"] += pair["lj"] - sum(a["lj"] for a in alone)
    out["elec"] += pair["coulomb"] - sum(a["coulomb"] for a in alone)
    out["total"] = sum(out[k] for k in PARTS)
    return out


def two_atom_curve(S, S1, S2, chi, chi1, chi2, fields, separations, start, margin=2.0):
    """PMF of the two atoms of S along x at the given separations.  S1 and
    S2 hold one atom each on the same grid (the groups alone); `fields` is
    (U, E, U1, E1, U2, E2) device buffers.  The loose start is a sphere of
    radius d/2 + sigma + margin about the midpoint."""
    U, E, U1, E1, U2, E2 = fields
    sig = float(np.max(S.sigma))
    c = np.zeros((1, 3))
    a1 = relaxed_parts(S1, chi1, U1, E1, c, start, sig + margin, c[0])
    a2 = relaxed_parts(S2, chi2, U2, E2, c, start, sig + margin, c[0])
    rows = []
    for d in separations:
        xyz = np.array([[-0.5 * d, 0.0, 0.0], [0.5 * d, 0.0, 0.0]])
        p = relaxed_parts(S, chi, U, E, xyz, start, 0.5 * d + sig + margin, np.zeros(3))
        row = combine(p, [a1, a2])
        row["d"] = float(d)
        row["rounds"] = p["rounds"]
        rows.append(row)
    return rows
