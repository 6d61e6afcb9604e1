"""Seeded synthetic inputs shared by the CUDA path, the tests and the benchmark.

This module only *generates* inputs: atomic structures, network parameters,
initial velocities and the frozen input standardisation. It holds none of the
potential's arithmetic (no descriptor, network or force evaluation), so the CUDA
path and the CPU oracle can both consume it without sharing method code.

Workloads (the paper's datasets and trained weights are not available, so these
stand in for its two system types, liquid water and a multi-species amorphous
solid, Sec. IV.B):

* ``water``      -- H2O molecules on a jittered cubic lattice, O-H 0.96 A,
                    H-O-H 104.5 deg, random orientation; types O=0, H=1.
* ``amorphous``  -- four species placed by random sequential addition with a
                    periodic minimum distance; fractions 0.4/0.3/0.2/0.1.

Units are LAMMPS "metal" (eV, A, amu, ps), the unit system the paper's water
example uses (Sec. III, LAMMPS input).
"""
from __future__ import annotations

import json
import math
import os
from dataclasses import dataclass, field

import numpy as np

# Masses of the paper's LAMMPS water example (Sec. III): H and O in amu.
MASS_H = 1.007825
MASS_O = 15.999491
WATER_MOLAR_MASS = 18.015          # g/mol, for the 1.0 g/cm^3 box length
AVOGADRO = 6.02214076e23
KB_EV = 8.617333262e-5             # eV/K
EV_PER_AMU = 9648.533212           # (A/ps)^2 per (eV/amu): v^2 = E/m * this

WATER_BASIS = dict(rc_rad=6.0, order_rad=16, rc_ang=4.0, order_ang=8)
AMORPHOUS_BASIS = dict(rc_rad=8.0, order_rad=20, rc_ang=6.5, order_ang=6)

# Species weights s_t of the species-weighted descriptor copy: balanced
# non-zero integers in species order (O, H) and (A, B, C, D).
WATER_TYPE_WEIGHTS = (-1.0, 1.0)
AMORPHOUS_TYPE_WEIGHTS = (-2.0, -1.0, 1.0, 2.0)


def descriptor_dim(order_rad: int, order_ang: int) -> int:
    """Length of [radial, angular, radial_w, angular_w] = 2 (N_r+1 + N_a+1)."""
    return 2 * (order_rad + 1 + order_ang + 1)


@dataclass
class Structure:
    pos: np.ndarray            # [N, 3] float64, Angstrom (not necessarily wrapped)
    types: np.ndarray          # [N] int32, 0-based species index
    box: np.ndarray            # [3] float64, orthorhombic box lengths
    n_species: int

    @property
    def n(self) -> int:
        return int(self.pos.shape[0])


@dataclass
class Model:
    """Per-species feed-forward networks plus descriptor basis.

    ``params[t]`` is the flat concatenation W^1, b^1, W^2, b^2, ... of species t,
    each W^l row-major [n_l x n_{l-1}].
    """
    n_species: int
    type_weights: np.ndarray   # [n_species]
    rc_rad: float
    order_rad: int
    rc_ang: float
    order_ang: int
    widths: tuple              # (D, h1, ..., 1)
    params: np.ndarray         # [n_species, n_params] float64
    in_shift: np.ndarray       # [n_species, D] float64
    in_scale: np.ndarray       # [n_species, D] float64
    masses: np.ndarray = field(default_factory=lambda: np.zeros(0))

    @property
    def D(self) -> int:
        return descriptor_dim(self.order_rad, self.order_ang)

    @property
    def n_params(self) -> int:
        return n_params(self.widths)


def n_params(widths) -> int:
    return sum(widths[l] * widths[l - 1] + widths[l] for l in range(1, len(widths)))


# ----------------------------------------------------------------- structures

def water_box_length(n_mol: int, density_g_cm3: float = 1.0) -> float:
    per_a3 = density_g_cm3 * AVOGADRO / WATER_MOLAR_MASS / 1e24
    return (n_mol / per_a3) ** (1.0 / 3.0)


def _lattice_side(n: int) -> int:
    m = max(1, int(round(n ** (1.0 / 3.0))))
    while m ** 3 < n:
        m += 1
    while m > 1 and (m - 1) ** 3 >= n:
        m -= 1
    return m


def water(n_mol: int, box: float | None, seed: int, jitter: float = 0.2,
          r_oh: float = 0.96, angle_deg: float = 104.5) -> Structure:
    """n_mol rigid-geometry H2O on a jittered m^3 lattice (m = ceil(n^(1/3))).

    Draw order from ``np.random.default_rng(seed)``: site permutation (only when
    m^3 > n_mol), O jitter [n,3] uniform in (-jitter, jitter), orientation
    quaternions [n,4] standard normal. Atom order O, H, H per molecule.
    """
    if box is None:
        box = water_box_length(n_mol)
    rng = np.random.default_rng(seed)
    m = _lattice_side(n_mol)
    a = box / m
    g = np.arange(m)
    sites = np.stack(np.meshgrid(g, g, g, indexing="ij"), -1).reshape(-1, 3)
    if m ** 3 > n_mol:
        sites = sites[rng.permutation(m ** 3)[:n_mol]]
    centres = (sites + 0.5) * a
    o = centres + rng.uniform(-jitter, jitter, size=(n_mol, 3))
    q = rng.standard_normal((n_mol, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    w, x, y, z = q.T
    rot = np.empty((n_mol, 3, 3))
    rot[:, 0, 0] = 1 - 2 * (y * y + z * z)
    rot[:, 0, 1] = 2 * (x * y - z * w)
    rot[:, 0, 2] = 2 * (x * z + y * w)
    rot[:, 1, 0] = 2 * (x * y + z * w)
    rot[:, 1, 1] = 1 - 2 * (x * x + z * z)
    rot[:, 1, 2] = 2 * (y * z - x * w)
    rot[:, 2, 0] = 2 * (x * z - y * w)
    rot[:, 2, 1] = 2 * (y * z + x * w)
    rot[:, 2, 2] = 1 - 2 * (x * x + y * y)
    half = math.radians(angle_deg) / 2.0
    b1 = r_oh * np.array([math.sin(half), 0.0, math.cos(half)])
    b2 = r_oh * np.array([-math.sin(half), 0.0, math.cos(half)])
    h1 = o + rot @ b1
    h2 = o + rot @ b2
    pos = np.stack([o, h1, h2], axis=1).reshape(-1, 3)
    types = np.tile(np.array([0, 1, 1], dtype=np.int32), n_mol)
    return Structure(pos=np.ascontiguousarray(pos), types=types,
                     box=np.full(3, float(box)), n_species=2)


def amorphous(n_atoms: int, seed: int, density: float = 0.07, dmin: float = 1.6,
              fractions=(0.4, 0.3, 0.2, 0.1), max_tries: int = 10_000_000) -> Structure:
    """Random sequential addition of n_atoms points at ``density`` atoms/A^3 in a
    periodic cube, rejecting any point closer than ``dmin`` (minimum image) to an
    accepted one. Species from a seeded permutation of exact counts
    round(f_t N) for t >= 1, the remainder to species 0.

    Draw order: candidate points [3] uniform in [0, L) one at a time until all
    are placed, then the species permutation.
    """
    rng = np.random.default_rng(seed)
    L = (n_atoms / density) ** (1.0 / 3.0)
    ng = max(1, int(L // dmin))
    hc = L / ng
    cells: dict = {}
    pts = np.empty((n_atoms, 3))
    placed = 0
    tries = 0
    d2min = dmin * dmin
    offs = sorted({((dx % ng), (dy % ng), (dz % ng))
                   for dx in (-1, 0, 1) for dy in (-1, 0, 1) for dz in (-1, 0, 1)})
    batch = rng.uniform(0.0, L, size=(4096, 3))
    bi = 0
    while placed < n_atoms:
        if bi == len(batch):
            batch = rng.uniform(0.0, L, size=(4096, 3))
            bi = 0
        p = batch[bi]
        bi += 1
        tries += 1
        if tries > max_tries:
            raise RuntimeError("random sequential addition did not converge")
        c = (int(p[0] // hc) % ng, int(p[1] // hc) % ng, int(p[2] // hc) % ng)
        ok = True
        for o in offs:
            lst = cells.get(((c[0] + o[0]) % ng, (c[1] + o[1]) % ng, (c[2] + o[2]) % ng))
            if not lst:
                continue
            q = pts[lst]
            d = q - p
            d -= L * np.round(d / L)
            if np.any(np.einsum("ij,ij->i", d, d) < d2min):
                ok = False
                break
        if not ok:
            continue
        pts[placed] = p
        cells.setdefault(c, []).append(placed)
        placed += 1
    counts = [int(round(f * n_atoms)) for f in fractions]
    counts[0] = n_atoms - sum(counts[1:])
    perm = rng.permutation(n_atoms)
    types = np.empty(n_atoms, dtype=np.int32)
    start = 0
    for t, c in enumerate(counts):
        types[perm[start:start + c]] = t
        start += c
    return Structure(pos=pts, types=types, box=np.full(3, L), n_species=len(fractions))


# ---------------------------------------------------------------- parameters

def ann_params(widths, n_species: int, seed: int) -> np.ndarray:
    """Per-species W^l, b^l ~ N(0, 1/fan_in), drawn species by species and layer
    by layer (W^l then b^l) from ``np.random.default_rng(seed)``."""
    rng = np.random.default_rng(seed)
    out = np.empty((n_species, n_params(widths)))
    for t in range(n_species):
        chunks = []
        for l in range(1, len(widths)):
            sd = math.sqrt(1.0 / widths[l - 1])
            chunks.append(rng.normal(0.0, sd, size=widths[l] * widths[l - 1]))
            chunks.append(rng.normal(0.0, sd, size=widths[l]))
        out[t] = np.concatenate(chunks)
    return out


_SCALING_FILE = os.path.join(os.path.dirname(__file__), "input_scaling.json")


def input_scaling(family: str, n_species: int, D: int):
    """Frozen per-feature standardisation g = (G - shift) * scale of a basis
    family ("water" or "amorphous"); shared by all species. Identity when the
    stored file has no entry yet."""
    shift = np.zeros((n_species, D))
    scale = np.ones((n_species, D))
    if os.path.exists(_SCALING_FILE):
        with open(_SCALING_FILE) as f:
            data = json.load(f)
        if family in data:
            s = np.asarray(data[family]["shift"], dtype=np.float64)
            c = np.asarray(data[family]["scale"], dtype=np.float64)
            if s.shape == (D,) and c.shape == (D,):
                shift[:] = s
                scale[:] = c
    return shift, scale


def make_model(family: str, hidden=None, seed: int = 1, identity_scaling: bool = False, orders=None) -> Model:
    """Model of a basis family with seeded N(0, 1/fan_in) weights.

    water:     rad 6.0 A / order 16, ang 4.0 A / order 8, D = 52, 52-15-15-1
    amorphous: rad 8.0 A / order 20, ang 6.5 A / order 6, D = 56, 56-30-30-1

    ``orders`` = (N_r, N_a) replaces the basis orders (model-size sweeps); the
    input standardisation is then the identity, since stored statistics exist
    only for the families' own bases.
    """
    if family == "water":
        basis, tw, masses = WATER_BASIS, WATER_TYPE_WEIGHTS, np.array([MASS_O, MASS_H])
        hidden = (15, 15) if hidden is None else tuple(hidden)
    elif family == "amorphous":
        basis, tw, masses = AMORPHOUS_BASIS, AMORPHOUS_TYPE_WEIGHTS, np.ones(4)
        hidden = (30, 30) if hidden is None else tuple(hidden)
    else:
        raise ValueError(family)
    if orders is not None:
        basis = dict(basis, order_rad=int(orders[0]), order_ang=int(orders[1]))
        identity_scaling = True
    D = descriptor_dim(basis["order_rad"], basis["order_ang"])
    widths = (D,) + hidden + (1,)
    ns = len(tw)
    params = ann_params(widths, ns, seed)
    if identity_scaling:
        shift, scale = np.zeros((ns, D)), np.ones((ns, D))
    else:
        shift, scale = input_scaling(family, ns, D)
    return Model(n_species=ns, type_weights=np.asarray(tw, dtype=np.float64),
                 widths=widths, params=params, in_shift=shift, in_scale=scale,
                 masses=masses, **basis)


def maxwell_boltzmann(masses_per_atom: np.ndarray, temperature: float, seed: int) -> np.ndarray:
    """Velocities (A/ps) at ``temperature`` K: normal draws [N,3] scaled by
    sqrt(kB T / m), centre-of-mass drift removed, then rescaled so that the
    kinetic temperature over 3N-3 degrees of freedom is exactly ``temperature``."""
    rng = np.random.default_rng(seed)
    m = np.asarray(masses_per_atom, dtype=np.float64)[:, None]
    v = rng.standard_normal((m.shape[0], 3)) * np.sqrt(KB_EV * temperature * EV_PER_AMU / m)
    v -= (m * v).sum(0) / m.sum()
    ekin = 0.5 * (m * v * v).sum() / EV_PER_AMU
    dof = 3 * m.shape[0] - 3
    t_now = 2.0 * ekin / (dof * KB_EV)
    v *= math.sqrt(temperature / t_now)
    return v


# ----------------------------------------------------------------- workloads

def water_192(seed: int = 0) -> Structure:
    """64 H2O in a 12.42 A periodic cube (seed 0)."""
    return water(64, 12.42, seed)


def water_12288(seed: int = 10) -> Structure:
    """4,096 H2O at 1.0 g/cm^3 (L = 49.669 A, seed 10)."""
    return water(4096, None, seed)


def water_331776(seed: int = 40) -> Structure:
    """110,592 H2O at 1.0 g/cm^3 (L = 149.006 A, seed 40)."""
    return water(110592, None, seed)


def amorphous_27000(seed: int = 20) -> Structure:
    """27,000-atom 4-species amorphous solid at 0.07 atoms/A^3 (seed 20)."""
    return amorphous(27000, seed)


def batch_sizes(n_struct: int = 512, lo: int = 32, hi: int = 2048, seed: int = 30) -> np.ndarray:
    """Log-uniform atom counts in [lo, hi] for the batched workload."""
    rng = np.random.default_rng(seed)
    return np.rint(np.exp(rng.uniform(math.log(lo), math.log(hi), size=n_struct))).astype(np.int64)


def batch_structures(n_struct: int = 512, lo: int = 32, hi: int = 2048, seed: int = 30, limit=None):
    """The batched workload: log-uniform atom counts in [lo, hi]; the first half
    water at 1.0 g/cm^3 (n_mol = round(N/3)), the second half the 4-species
    amorphous solid; structure s uses seed 31 + s. Returns (water list,
    amorphous list) of Structures; ``limit`` keeps only the first structures of
    each half (for tests)."""
    sizes = batch_sizes(n_struct, lo, hi, seed)
    half = n_struct // 2
    wat, amo = [], []
    for s in range(n_struct):
        if limit is not None and (s % half) >= limit:
            continue
        if s < half:
            wat.append(water(max(1, int(round(sizes[s] / 3))), None, 31 + s))
        else:
            amo.append(amorphous(int(sizes[s]), 31 + s))
    return wat, amo


def concat(structures):
    """Flatten a list of Structures into (atom_offset [S+1], pos [N,3], types [N], boxes [S,3])."""
    off = np.zeros(len(structures) + 1, dtype=np.int64)
    off[1:] = np.cumsum([st.n for st in structures])
    pos = np.concatenate([st.pos for st in structures]) if structures else np.zeros((0, 3))
    types = np.concatenate([st.types for st in structures]).astype(np.int32) if structures else np.zeros(0, np.int32)
    boxes = np.stack([st.box for st in structures]) if structures else np.zeros((0, 3))
    return off, np.ascontiguousarray(pos), types, boxes
