"""Synthetic meshes for the 2D eddy-current (A_z) model.

These builders produce geometry and tags only: node coordinates, triangles,
material region per triangle, Dirichlet flags per node and the coil phase and
winding sign per triangle.  They hold none of the method's arithmetic (no
element integrals, no time stepping); both the CUDA path and the CPU oracle
consume the arrays they return.

Two families:

* ``unit_square(nx)``: structured P1 mesh of the unit square, every cell split
  by its (0,0)->(1,1) diagonal, with a central conductor that carries the
  source current (the small Monte Carlo workload).
* ``annulus(kind)``: a polar-structured "machine-shaped" annulus standing in
  for the 2D induction-machine model of Sec. III-B, which is not public here:
  rotor iron, 32 rotor bars, a 1 mm air gap, 36 stator slots with a 3-phase,
  4-pole winding, stator iron; homogeneous Dirichlet at both radii, periodic
  in the angle.  ``kind`` is "5k", "20k" or "80k" (node count).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

# Material region ids of the annulus.
ROTOR_IRON, ROTOR_BARS, AIR_GAP, STATOR_IRON, COIL_A, COIL_B, COIL_C = range(7)
ANNULUS_REGION_NAMES = ("rotor_iron", "rotor_bars", "air_gap", "stator_iron",
                        "coil_A", "coil_B", "coil_C")
# Region ids of the unit square.
SQUARE_BACKGROUND, SQUARE_CONDUCTOR = 0, 1


@dataclass
class Mesh:
    """A triangle mesh with material and source tags.

    xy         float64 [n_nodes, 2]   node coordinates (m)
    tri        int32   [n_tri, 3]     node ids, counter-clockwise
    region     int32   [n_tri]        material region id in [0, n_regions)
    dirichlet  uint8   [n_nodes]      1 where A_z = 0 is imposed
    src_phase  int32   [n_tri]        coil phase id in [0, n_phases), -1: no source
    src_coef   float64 [n_tri]        winding sign/fill of the source in that triangle
    """
    name: str
    xy: np.ndarray
    tri: np.ndarray
    region: np.ndarray
    dirichlet: np.ndarray
    src_phase: np.ndarray
    src_coef: np.ndarray
    n_regions: int
    n_phases: int
    region_names: tuple = field(default_factory=tuple)

    @property
    def n_nodes(self) -> int:
        return int(self.xy.shape[0])

    @property
    def n_tri(self) -> int:
        return int(self.tri.shape[0])

    @property
    def n_free(self) -> int:
        return int(self.n_nodes - int(self.dirichlet.sum()))


def unit_square(nx: int = 16, conductor: tuple = None) -> Mesh:
    """Structured nx x nx unit square, cells split along (0,0)->(1,1).

    Node (i, j) sits at (i/nx, j/nx) and has id j*(nx+1)+i.  The conductor is
    the block of cells [lo, hi) x [lo, hi); by default the central quarter of
    the side length (cells [6, 10) for nx = 16).  It is region 1, carries the
    source with phase 0 and sign +1; the rest is region 0.  All boundary nodes
    are Dirichlet.
    """
    if conductor is None:
        lo = (3 * nx) // 8
        hi = nx - lo
        conductor = (lo, hi)
    lo, hi = conductor
    n1 = nx + 1
    ii, jj = np.meshgrid(np.arange(n1), np.arange(n1), indexing="xy")
    xy = np.stack([ii.ravel() / nx, jj.ravel() / nx], axis=1).astype(np.float64)
    tris, regs = [], []
    for j in range(nx):
        for i in range(nx):
            n00 = j * n1 + i
            n10 = n00 + 1
            n01 = n00 + n1
            n11 = n01 + 1
            inside = lo <= i < hi and lo <= j < hi
            r = SQUARE_CONDUCTOR if inside else SQUARE_BACKGROUND
            tris.append((n00, n10, n11))   # lower-right triangle
            tris.append((n00, n11, n01))   # upper-left triangle
            regs += [r, r]
    tri = np.asarray(tris, dtype=np.int32)
    region = np.asarray(regs, dtype=np.int32)
    on_bnd = (ii.ravel() == 0) | (ii.ravel() == nx) | (jj.ravel() == 0) | (jj.ravel() == nx)
    src_phase = np.where(region == SQUARE_CONDUCTOR, 0, -1).astype(np.int32)
    src_coef = np.where(region == SQUARE_CONDUCTOR, 1.0, 0.0)
    return Mesh(name=f"square{nx}", xy=xy, tri=tri, region=region,
                dirichlet=on_bnd.astype(np.uint8), src_phase=src_phase,
                src_coef=src_coef, n_regions=2, n_phases=1,
                region_names=("background", "conductor"))


# Radial bands of the annulus: (r_inner, r_outer, layers) for the 20k mesh.
_BANDS_20K = ((0.020, 0.044, 16),   # rotor iron
              (0.044, 0.052, 8),    # rotor-bar band
              (0.052, 0.054, 2),    # rotor tip
              (0.054, 0.055, 3),    # air gap (1 mm)
              (0.055, 0.075, 20),   # stator slot band
              (0.075, 0.100, 20))   # yoke
_ANNULUS_KINDS = {
    # kind: (N_theta, layers per band)
    "5k": (288, (4, 2, 1, 1, 5, 4)),
    "20k": (288, tuple(b[2] for b in _BANDS_20K)),
    "80k": (576, tuple(2 * b[2] for b in _BANDS_20K)),
}
# Stator winding: 3-phase, 4-pole, 3 slots per pole and phase; 18-slot pattern
# repeated twice around 36 slots.  (phase, sign), phase 0/1/2 = A/B/C.
_SLOT_PATTERN = ((0, 1),) * 3 + ((2, -1),) * 3 + ((1, 1),) * 3 + \
                ((0, -1),) * 3 + ((2, 1),) * 3 + ((1, -1),) * 3
N_BARS, N_SLOTS = 32, 36


def annulus_radii(kind: str) -> np.ndarray:
    """Node ring radii (m) of an annulus kind, uniform within each band."""
    _, layers = _ANNULUS_KINDS[kind]
    rs = [_BANDS_20K[0][0]]
    for (r0, r1, _), m in zip(_BANDS_20K, layers):
        rs.extend(list(r0 + (r1 - r0) * np.arange(1, m + 1) / m))
    return np.asarray(rs, dtype=np.float64)


def annulus(kind: str = "20k") -> Mesh:
    """Polar-structured machine-shaped annulus over r in [0.02, 0.10] m.

    Node (ring i, angle j) has id j*N_r + i (radius fastest) and sits at
    (r_i cos t_j, r_i sin t_j), t_j = 2*pi*j/N_theta.  Each polar quad
    (i, j)-(i+1, j+1) is split along its (i, j)->(i+1, j+1) diagonal; the
    angle wraps periodically.  Regions are assigned from the triangle's
    centroid in (r, theta): bars span half the bar pitch, coil sides half the
    slot pitch.  Dirichlet on the innermost and outermost rings.
    """
    n_theta, _ = _ANNULUS_KINDS[kind]
    radii = annulus_radii(kind)
    n_r = radii.size
    dth = 2.0 * np.pi / n_theta
    jj, ii = np.meshgrid(np.arange(n_theta), np.arange(n_r), indexing="ij")
    th = jj.ravel() * dth
    rr = radii[ii.ravel()]
    xy = np.stack([rr * np.cos(th), rr * np.sin(th)], axis=1)

    i = np.arange(n_r - 1)
    j = np.arange(n_theta)
    J, I = np.meshgrid(j, i, indexing="ij")
    I = I.ravel()
    J = J.ravel()
    Jp = (J + 1) % n_theta
    n_ij = J * n_r + I
    n_i1j = J * n_r + I + 1
    n_i1j1 = Jp * n_r + I + 1
    n_ij1 = Jp * n_r + I
    t1 = np.stack([n_ij, n_i1j, n_i1j1], axis=1)
    t2 = np.stack([n_ij, n_i1j1, n_ij1], axis=1)
    tri = np.empty((2 * I.size, 3), dtype=np.int32)
    tri[0::2] = t1
    tri[1::2] = t2
    # centroids in (r, theta) with the angle unwrapped across the seam
    r_c = np.empty(tri.shape[0])
    th_c = np.empty(tri.shape[0])
    r_c[0::2] = (radii[I] + 2.0 * radii[I + 1]) / 3.0   # rings i, i+1, i+1
    r_c[1::2] = (2.0 * radii[I] + radii[I + 1]) / 3.0   # rings i, i+1, i
    th_c[0::2] = (J + 1.0 / 3.0) * dth   # vertices at t_j, t_j, t_{j+1}
    th_c[1::2] = (J + 2.0 / 3.0) * dth   # vertices at t_j, t_{j+1}, t_{j+1}

    region = np.full(tri.shape[0], ROTOR_IRON, dtype=np.int32)
    src_phase = np.full(tri.shape[0], -1, dtype=np.int32)
    src_coef = np.zeros(tri.shape[0])
    bar_pitch = 2.0 * np.pi / N_BARS
    slot_pitch = 2.0 * np.pi / N_SLOTS
    # bars centred on multiples of the bar pitch, half a pitch wide
    fb = th_c / bar_pitch
    in_bar = np.abs(fb - np.round(fb)) < 0.25
    band_bar = (r_c >= 0.044) & (r_c < 0.052)
    region[band_bar & in_bar] = ROTOR_BARS
    gap = (r_c >= 0.054) & (r_c < 0.055)
    region[gap] = AIR_GAP
    stator = r_c >= 0.055
    region[stator] = STATOR_IRON
    # slots centred on (s + 1/2) slot pitches, half a pitch wide
    fs = th_c / slot_pitch - 0.5
    slot_idx = np.round(fs).astype(np.int64) % N_SLOTS
    in_slot = (np.abs(fs - np.round(fs)) < 0.25) & (r_c >= 0.055) & (r_c < 0.075)
    pat = np.asarray(_SLOT_PATTERN)
    ph = pat[slot_idx % len(_SLOT_PATTERN), 0]
    sg = pat[slot_idx % len(_SLOT_PATTERN), 1]
    region[in_slot] = COIL_A + ph[in_slot]
    src_phase[in_slot] = ph[in_slot]
    src_coef[in_slot] = sg[in_slot]

    dirichlet = ((ii.ravel() == 0) | (ii.ravel() == n_r - 1)).astype(np.uint8)
    return Mesh(name=f"annulus{kind}", xy=xy, tri=tri, region=region,
                dirichlet=dirichlet, src_phase=src_phase, src_coef=src_coef,
                n_regions=7, n_phases=3, region_names=ANNULUS_REGION_NAMES)


def build(name: str) -> Mesh:
    """Mesh by name: 'square<nx>' or 'annulus<kind>' (e.g. 'annulus20k')."""
    if name.startswith("square"):
        return unit_square(int(name[len("square"):]))
    if name.startswith("annulus"):
        return annulus(name[len("annulus"):])
    raise ValueError(f"unknown mesh {name!r}")
