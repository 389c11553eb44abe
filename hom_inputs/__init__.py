"""Seeded synthetic inputs for filtered-property FFT homogenisation of periodic elastic cells.

This module is shared by the CPU oracle, the tests and the benchmark.  It only describes
*inputs*: cell geometry (disks, spheres, slabs), phase moduli and macroscopic load cases.
It holds none of the homogenisation arithmetic (no filters, no Green operator, no FFT).

The geometry follows the numerical experiment of Gélébart & Ouaki, section 2: a periodic
unit cell (side 1) holding one centred circular inclusion in a matrix, isotropic phases
with the same Poisson ratio nu = 0.3, elastic contrast = E_inclusion / E_matrix.  The 3D
and ensemble generators produce random non-overlapping spheres / disks of the same kind.

Coordinates are in cell units; a grid of n voxels per side has its grid points at the voxel
centres x_a = (a + 1/2) / n.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Sequence, Tuple

import numpy as np

# Primitive kinds and filter rules.  The integer values are part of the C ABI (include/hom.h).
PRIM_DISK = 0
PRIM_SPHERE = 1
PRIM_SLAB = 2

RULE_NONE = 0
RULE_VOIGT = 1
RULE_REUSS = 2
RULE_TWO_LAYER = 3

RULE_NAMES = {RULE_NONE: "none", RULE_VOIGT: "voigt", RULE_REUSS: "reuss", RULE_TWO_LAYER: "2-layers"}


@dataclasses.dataclass
class Primitive:
    """One analytic inclusion.

    kind    PRIM_DISK (2D), PRIM_SPHERE (3D) or PRIM_SLAB (any dimension)
    phase   phase index of the points inside the primitive
    centre  centre in cell units (3 values; the third is ignored in 2D)
    radius  disk/sphere radius in cell units; for a slab, its full thickness
    axis    slab normal axis (0 = x, 1 = y, 2 = z); unused for disks/spheres
    """
    kind: int
    phase: int
    centre: Tuple[float, float, float]
    radius: float
    axis: int = 0


@dataclasses.dataclass
class Cell:
    """A periodic unit cell on an n^dim voxel grid plus its filter settings."""
    dim: int
    n: int
    matrix_phase: int
    prims: List[Primitive]
    rule: int = RULE_NONE
    radius_px: float = 1.0
    subgrid: int = 16

    @property
    def nvox(self) -> int:
        return self.n ** self.dim


def lame_from_young(E: float, nu: float) -> Tuple[float, float]:
    """Lamé pair (lambda, mu) of an isotropic phase given Young's modulus and Poisson ratio."""
    lam = E * nu / ((1.0 + nu) * (1.0 - 2.0 * nu))
    mu = E / (2.0 * (1.0 + nu))
    return lam, mu


def mean_lame(phases: Sequence[Tuple[float, float]]) -> Tuple[float, float]:
    """Reference medium as the mean of the extreme phase Lamé constants (isotropic phases)."""
    lams = [p[0] for p in phases]
    mus = [p[1] for p in phases]
    return 0.5 * (min(lams) + max(lams)), 0.5 * (min(mus) + max(mus))


def geometric_lame(phases: Sequence[Tuple[float, float]], dim: int) -> Tuple[float, float]:
    """Reference medium for the Eyre-Milton scheme: geometric means of the extreme phase shear
    moduli and bulk moduli lambda + 2 mu / dim, returned as a Lame pair."""
    mus = [p[1] for p in phases]
    ks = [p[0] + 2.0 * p[1] / dim for p in phases]
    mu0 = math.sqrt(min(mus) * max(mus))
    k0 = math.sqrt(min(ks) * max(ks))
    return k0 - 2.0 * mu0 / dim, mu0


def ncomp(dim: int) -> int:
    """Number of independent strain components (Mandel vector length)."""
    return 3 if dim == 2 else 6


def unit_loads(dim: int) -> np.ndarray:
    """The nc unit Mandel macroscopic strains, one load case per row."""
    return np.eye(ncomp(dim))


# ---------------------------------------------------------------------------------------------
# Two-phase cells (phase 0 = matrix, phase 1 = inclusion)

def two_phases(contrast: float, nu: float = 0.3, E_matrix: float = 1.0):
    """Phase table [(lambda, mu)] for matrix (index 0) and inclusion (index 1)."""
    return [lame_from_young(E_matrix, nu), lame_from_young(E_matrix * contrast, nu)]


def centred_disk_cell(n: int, vf: float = 0.2, rule: int = RULE_VOIGT, radius_px: float = 1.0,
                      subgrid: int = 16, radius: float | None = None) -> Cell:
    """2D cell with one disk of volume fraction vf (or the given radius) at (0.5, 0.5)."""
    r = math.sqrt(vf / math.pi) if radius is None else radius
    return Cell(2, n, 0, [Primitive(PRIM_DISK, 1, (0.5, 0.5, 0.0), r)], rule, radius_px, subgrid)


def laminate_cell(n: int, dim: int, thickness: float, axis: int = 0, centre: float = 0.5,
                  rule: int = RULE_NONE, radius_px: float = 1.0, subgrid: int = 16) -> Cell:
    """Cell holding one slab of phase 1 (normal along `axis`) in a phase-0 matrix."""
    c = [0.5, 0.5, 0.5]
    c[axis] = centre
    return Cell(dim, n, 0, [Primitive(PRIM_SLAB, 1, tuple(c), thickness, axis)], rule, radius_px, subgrid)


def homogeneous_cell(n: int, dim: int) -> Cell:
    return Cell(dim, n, 0, [], RULE_NONE, 1.0, 8)


def _periodic_dist(a: np.ndarray, b: np.ndarray) -> float:
    d = np.abs(a - b)
    d = np.minimum(d, 1.0 - d)
    return float(np.sqrt(np.sum(d * d)))


def rsa_spheres_cell(n: int, seed: int, vf: float = 0.3, rmin: float = 0.05, rmax: float = 0.1,
                     rule: int = RULE_TWO_LAYER, radius_px: float = 1.0, subgrid: int = 8,
                     gap_voxels: float = 2.0, batches: int = 400) -> Cell:
    """3D random sequential addition of non-overlapping spheres (periodic minimum image).

    Radii are drawn uniformly in [rmin, rmax]; spheres are added until the total volume reaches
    vf, and the last radius is shrunk so that the total is exactly vf.  Two spheres keep a surface
    gap of at least gap_voxels / n.  Candidate centres are tried in seeded batches of 256; a
    sphere that finds no room after `batches` // 8 batches is shrunk by 5 % (not below rmin)."""
    rng = np.random.default_rng(seed)
    gap = gap_voxels / n
    centres = np.zeros((0, 3))
    radii = np.zeros(0)
    vol = 0.0
    while vol < vf - 1e-15:
        r = float(rng.uniform(rmin, rmax))
        rem = vf - vol
        if 4.0 / 3.0 * math.pi * r ** 3 >= rem:
            r = (rem * 3.0 / (4.0 * math.pi)) ** (1.0 / 3.0)
        placed = None
        for b in range(batches):
            if b > 0 and b % max(1, batches // 8) == 0:
                r = max(rmin, 0.95 * r) if r > rmin else r
            cand = rng.uniform(0.0, 1.0, size=(256, 3))
            if centres.shape[0] == 0:
                placed = cand[0]
                break
            d = np.abs(cand[:, None, :] - centres[None, :, :])
            d = np.minimum(d, 1.0 - d)
            dist = np.sqrt(np.sum(d * d, axis=-1))
            ok = np.all(dist >= r + radii[None, :] + gap, axis=1)
            if np.any(ok):
                placed = cand[int(np.argmax(ok))]
                break
        if placed is None:
            raise RuntimeError("sphere packing failed; lower vf or the gap")
        centres = np.vstack([centres, placed[None, :]])
        radii = np.append(radii, r)
        vol += 4.0 / 3.0 * math.pi * r ** 3
    prims = [Primitive(PRIM_SPHERE, 1, (float(c[0]), float(c[1]), float(c[2])), float(r))
             for c, r in zip(centres, radii)]
    return Cell(3, n, 0, prims, rule, radius_px, subgrid)


def random_disk_cell(seed: int, sizes=(45, 75, 135, 225, 405), kmin: int = 4, kmax: int = 40,
                     vfmin: float = 0.1, vfmax: float = 0.4, subgrid: int = 16,
                     radius_px: float = 1.0) -> Tuple[Cell, List[Tuple[float, float]]]:
    """One member of the random-disk ensemble: grid, disk set, contrast and filter rule drawn
    from the seed.  Returns the cell and its two-phase table."""
    rng = np.random.default_rng(seed)
    n = int(rng.choice(sizes))
    k = int(rng.integers(kmin, kmax + 1))
    vf = float(rng.uniform(vfmin, vfmax))
    contrast = float(10.0 ** rng.uniform(-2.0, 2.0))
    rule = int(rng.choice([RULE_REUSS, RULE_VOIGT, RULE_TWO_LAYER]))
    gap = 1.0 / n
    for _attempt in range(100):
        r0 = math.sqrt(vf / (k * math.pi))
        jit = rng.uniform(0.8, 1.2, size=k)
        radii = r0 * jit * math.sqrt(vf / (math.pi * float(np.sum((r0 * jit) ** 2))))
        centres: List[np.ndarray] = []
        ok = True
        for r in radii:
            for _t in range(5000):
                c = rng.uniform(0.0, 1.0, size=2)
                if all(_periodic_dist(c, cj) >= r + rj + gap for cj, rj in zip(centres, radii)):
                    centres.append(c)
                    break
            else:
                ok = False
                break
        if ok:
            prims = [Primitive(PRIM_DISK, 1, (float(c[0]), float(c[1]), 0.0), float(r))
                     for c, r in zip(centres, radii)]
            return Cell(2, n, 0, prims, rule, radius_px, subgrid), two_phases(contrast)
    raise RuntimeError("disk packing failed")


def resolution_sweep_cells(sizes=(45, 135, 405, 1215), contrasts=(10.0, 0.1),
                           rules=(RULE_NONE, RULE_VOIGT, RULE_REUSS, RULE_TWO_LAYER),
                           vf: float = 0.2, radius_px: float = 1.0, subgrid: int = 16):
    """The 2D resolution sweep of the centred-disk cell: every (size, contrast, rule) triple.

    Returns (cells, phases, cell_phase_offset) where the phase table holds one matrix /
    inclusion pair per contrast and each cell's primitive and matrix phases are remapped
    to its contrast's pair."""
    phases: List[Tuple[float, float]] = []
    base = {}
    for c in contrasts:
        base[c] = len(phases)
        phases.extend(two_phases(c))
    cells = []
    for n in sizes:
        for c in contrasts:
            for rule in rules:
                cell = centred_disk_cell(n, vf, rule, radius_px, subgrid)
                cell.matrix_phase = base[c]
                for p in cell.prims:
                    p.phase = base[c] + 1
                cells.append(cell)
    return cells, phases


def remap_phases(cell: Cell, offset: int) -> Cell:
    """Copy of `cell` with every phase index shifted by `offset`."""
    prims = [dataclasses.replace(p, phase=p.phase + offset) for p in cell.prims]
    return dataclasses.replace(cell, matrix_phase=cell.matrix_phase + offset, prims=prims)


def cell_phase_pair(cell: Cell) -> Tuple[int, int]:
    """(matrix phase, inclusion phase) of a two-phase cell."""
    inc = cell.prims[0].phase if cell.prims else cell.matrix_phase
    return cell.matrix_phase, inc
