"""Seeded synthetic inputs: molecular systems, model weights, initial velocities.

This module is the only code shared by the CUDA path and the FP64 oracle. It
draws inputs and holds none of the method's arithmetic: no neighbour list, no
model, no integrator, no mass repartitioning, no friction table. The paper's
workloads (bulk water boxes, solvated proteins, solvated small molecules,
Sec. 3) are not available, so seeded stand-ins with the same composition,
density and size are generated here:

* water boxes: rigid waters (O-H 0.9572 A, H-O-H 104.52 deg) on a cubic
  lattice, random orientation, N(0, 0.05 A) jitter on every coordinate;
* a solvated bead chain of protein size (C/N/O/H/S 32/9/10/48/1 %) on an
  excluded-volume walk with 1.5 A bonds, in water at about 1 g/cm^3;
* small molecules (heavy chain + hydrogen caps) in a water droplet with open
  boundaries, for the replica-serving workload.

Units: Angstrom, femtosecond, amu, kcal/mol, kelvin. Positions are rounded to
float32 so that both sides read bit-identical coordinates.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

SPECIES = ("H", "C", "N", "O", "S")
SP_H, SP_C, SP_N, SP_O, SP_S = range(5)
N_SPECIES = 5
# IUPAC conventional atomic weights (amu), indexed by species code.
ELEMENT_MASS = np.array([1.008, 12.011, 14.007, 15.999, 32.06])
# Valence used by the hydrogen-capping generator.
VALENCE = {SP_C: 4, SP_N: 3, SP_O: 2, SP_S: 2}

WATER_OH = 0.9572
WATER_HOH_DEG = 104.52
CHAIN_BOND = 1.5
CAP_BOND = 1.09
# Boltzmann constant (kcal/mol/K) and force->acceleration factor
# (A/fs^2 per (kcal/mol/A)/amu); used here only to draw initial velocities.
KB_KCAL = 8.314462618 / 4184.0
ACC_CONV = 4.184e-4
# Number density of liquid water atoms (3 atoms per 29.9 A^3).
WATER_ATOM_DENSITY = 3.0 / 29.9


@dataclasses.dataclass
class System:
    """One molecular system. Arrays are host numpy arrays."""

    name: str
    x: np.ndarray          # (N,3) float64 holding float32-representable values
    species: np.ndarray    # (N,) uint8 species code (SP_*)
    mol_id: np.ndarray     # (N,) int32 molecule index
    bonds: np.ndarray      # (B,2) int32 atom pairs
    bond_r0: np.ndarray    # (B,) float64 rest lengths
    box: np.ndarray        # (3,) float64 box edges; 0 on every axis = open boundary

    @property
    def n_atoms(self) -> int:
        return int(self.x.shape[0])

    def element_masses(self) -> np.ndarray:
        return ELEMENT_MASS[self.species.astype(np.int64)]


def _f32(a: np.ndarray) -> np.ndarray:
    return np.asarray(a, dtype=np.float32).astype(np.float64)


def _random_rotations(rng: np.random.Generator, n: int) -> np.ndarray:
    """Uniform random rotation matrices from uniform unit quaternions."""
    u1, u2, u3 = rng.random(n), rng.random(n), rng.random(n)
    a = np.sqrt(1.0 - u1) * np.sin(2 * np.pi * u2)
    b = np.sqrt(1.0 - u1) * np.cos(2 * np.pi * u2)
    c = np.sqrt(u1) * np.sin(2 * np.pi * u3)
    d = np.sqrt(u1) * np.cos(2 * np.pi * u3)
    R = np.empty((n, 3, 3))
    R[:, 0, 0] = 1 - 2 * (c * c + d * d)
    R[:, 0, 1] = 2 * (b * c - a * d)
    R[:, 0, 2] = 2 * (b * d + a * c)
    R[:, 1, 0] = 2 * (b * c + a * d)
    R[:, 1, 1] = 1 - 2 * (b * b + d * d)
    R[:, 1, 2] = 2 * (c * d - a * b)
    R[:, 2, 0] = 2 * (b * d - a * c)
    R[:, 2, 1] = 2 * (c * d + a * b)
    R[:, 2, 2] = 1 - 2 * (b * b + c * c)
    return R


def _water_template() -> np.ndarray:
    t = math.radians(WATER_HOH_DEG) / 2
    return np.array([[0.0, 0.0, 0.0],
                     [WATER_OH * math.sin(t), 0.0, WATER_OH * math.cos(t)],
                     [-WATER_OH * math.sin(t), 0.0, WATER_OH * math.cos(t)]])


def _place_waters(rng, sites, first_mol, first_atom, obstacles=None, box=None, h_min=1.8):
    """Rigid, randomly oriented waters with O on `sites`; returns arrays. With
    `obstacles`, orientations putting an H closer than h_min to an obstacle are
    re-drawn (up to 50 times)."""
    n = sites.shape[0]
    R = _random_rotations(rng, n)
    tmpl = _water_template()
    xw = sites[:, None, :] + np.einsum("nab,kb->nka", R, tmpl)
    if obstacles is not None and n > 0:
        from scipy.spatial import cKDTree
        tree = cKDTree(np.mod(obstacles, box), boxsize=box) if box is not None else cKDTree(obstacles)
        wrap = (lambda p: np.mod(p, box)) if box is not None else (lambda p: p)
        for _try in range(50):
            dh, _ = tree.query(wrap(xw[:, 1:, :].reshape(-1, 3)), k=1)
            bad = np.nonzero((dh.reshape(n, 2) < h_min).any(1))[0]
            if bad.size == 0:
                break
            Rb = _random_rotations(rng, bad.size)
            xw[bad] = sites[bad][:, None, :] + np.einsum("nab,kb->nka", Rb, tmpl)
    x = xw.reshape(-1, 3)
    species = np.tile(np.array([SP_O, SP_H, SP_H], np.uint8), n)
    mol = np.repeat(np.arange(first_mol, first_mol + n, dtype=np.int32), 3)
    o = first_atom + 3 * np.arange(n, dtype=np.int32)
    bonds = np.concatenate([np.stack([o, o + 1], 1), np.stack([o, o + 2], 1)], 0)
    bonds = bonds[np.argsort(bonds[:, 0] * 4 + bonds[:, 1] - bonds[:, 0], kind="stable")]
    r0 = np.full(bonds.shape[0], WATER_OH)
    return x, species, mol, bonds.astype(np.int32), r0


def water_box(n_mol: int, box_len: float, seed: int, n_lone_o: int = 0,
              jitter: float = 0.05, name: str = "water") -> System:
    """`n_mol` rigid waters (+ `n_lone_o` lone O atoms) on an n^3 lattice in a
    periodic cube of edge `box_len`: first sites of a seeded permutation,
    seeded orientations, N(0, jitter) on every coordinate."""
    rng = np.random.default_rng(seed)
    n_sites = n_mol + n_lone_o
    n = int(math.ceil(n_sites ** (1.0 / 3.0) - 1e-9))
    g = (np.arange(n) + 0.5) * (box_len / n)
    grid = np.stack(np.meshgrid(g, g, g, indexing="ij"), -1).reshape(-1, 3)
    sites = grid[rng.permutation(grid.shape[0])[:n_sites]]
    x, sp, mol, bonds, r0 = _place_waters(rng, sites[:n_mol], 0, 0)
    if n_lone_o:
        x = np.concatenate([x, sites[n_mol:]], 0)
        sp = np.concatenate([sp, np.full(n_lone_o, SP_O, np.uint8)])
        mol = np.concatenate([mol, np.arange(n_mol, n_mol + n_lone_o, dtype=np.int32)])
    x = x + rng.normal(0.0, jitter, size=x.shape)
    return System(name, _f32(x), sp, mol, bonds, r0, np.full(3, float(box_len)))


def _excluded_volume_walk(rng, n: int, bond: float, box=None, d_min: float = 2.5,
                          angle_deg: float = 109.47, max_backtracks: int = 20000) -> np.ndarray:
    """Chain of n beads in continuous space: bond length `bond`, bond angle
    `angle_deg`, seeded uniform dihedrals; beads three or more apart along the
    chain stay at least d_min apart (minimum image when `box` is given).
    Dead ends are resolved by seeded backtracking."""
    def mi(d):
        return d - box * np.rint(d / box) if box is not None else d
    pos = np.zeros((n, 3))
    centre = box / 2.0 if box is not None else np.zeros(3)
    pos[0] = centre
    u = rng.normal(size=3)
    pos[1] = pos[0] + bond * u / np.linalg.norm(u)
    k, backtracks = 2, 0
    theta = math.radians(angle_deg)
    while k < n:
        b1 = pos[k - 1] - pos[k - 2]
        b1 /= np.linalg.norm(b1)
        ref = pos[k - 2] - pos[k - 3] if k >= 3 else rng.normal(size=3)
        e2 = ref - (ref @ b1) * b1
        if np.linalg.norm(e2) < 1e-8:
            e2 = np.cross(b1, [1.0, 0.0, 0.0]) if abs(b1[0]) < 0.9 else np.cross(b1, [0.0, 1.0, 0.0])
        e2 /= np.linalg.norm(e2)
        e3 = np.cross(b1, e2)
        placed = False
        for _try in range(24):
            phi = rng.uniform(0, 2 * np.pi)
            d = -math.cos(theta) * b1 + math.sin(theta) * (math.cos(phi) * e2 + math.sin(phi) * e3)
            cand = pos[k - 1] + bond * d
            if k >= 3:
                dd = np.linalg.norm(mi(pos[: k - 2] - cand), axis=1)
                if dd.min() < d_min:
                    continue
            pos[k] = cand
            placed = True
            break
        if placed:
            k += 1
        else:
            backtracks += 1
            if backtracks > max_backtracks:
                raise RuntimeError("excluded-volume walk failed")
            k = max(2, k - int(rng.integers(1, 6)))
    return pos


def _largest_remainder(total: int, percents) -> list:
    raw = [total * p / 100.0 for p in percents]
    base = [int(math.floor(r)) for r in raw]
    rem = total - sum(base)
    order = sorted(range(len(raw)), key=lambda k: -(raw[k] - base[k]))
    for k in order[:rem]:
        base[k] += 1
    return base


def _min_image_dist_ok(points, obstacles, box, rmin):
    """True for each point farther than rmin from every obstacle (periodic)."""
    from scipy.spatial import cKDTree
    if box is not None:
        tree = cKDTree(np.mod(obstacles, box), boxsize=box)
        d, _ = tree.query(np.mod(points, box), k=1)
    else:
        tree = cKDTree(obstacles)
        d, _ = tree.query(points, k=1)
    return d > rmin


def solvated_chain(n_chain: int = 2489, n_water: int = 7023, box_len: float = 62.2,
                   seed: int = 301, jitter: float = 0.05,
                   composition=(("C", 32), ("N", 9), ("O", 10), ("H", 48), ("S", 1)),
                   name: str = "solvated_chain") -> System:
    """A bonded bead chain (seeded excluded-volume walk: 1.5 A bonds,
    tetrahedral bond angle, random dihedrals, beads three or more apart at
    least 2.5 A apart; species by largest-remainder rounding of
    `composition`, placed by a seeded shuffle) in a periodic water box. Water
    O sites closer than 2.5 A to a bead are rejected; the lattice is the
    smallest n^3 that leaves enough sites; the first `n_water` sites of a
    seeded permutation are used; water hydrogens are kept 1.8 A from beads by
    re-drawing the orientation."""
    rng = np.random.default_rng(seed)
    box = np.full(3, float(box_len))
    xc = _excluded_volume_walk(rng, n_chain, CHAIN_BOND, box=box)
    counts = _largest_remainder(n_chain, [p for _, p in composition])
    codes = []
    for (sym, _), cnt in zip(composition, counts):
        codes += [SPECIES.index(sym)] * cnt
    sp_c = np.array(codes, np.uint8)[rng.permutation(n_chain)]
    bonds_c = np.stack([np.arange(n_chain - 1), np.arange(1, n_chain)], 1).astype(np.int32)
    r0_c = np.full(n_chain - 1, CHAIN_BOND)
    n = int(math.ceil(n_water ** (1.0 / 3.0)))
    while True:
        g = (np.arange(n) + 0.5) * (box_len / n)
        grid = np.stack(np.meshgrid(g, g, g, indexing="ij"), -1).reshape(-1, 3)
        ok = _min_image_dist_ok(grid, xc, box, 2.5)
        if ok.sum() >= n_water:
            break
        n += 1
    acc = grid[ok]
    sites = acc[rng.permutation(acc.shape[0])[:n_water]]
    xw, spw, molw, bw, r0w = _place_waters(rng, sites, 1, n_chain, obstacles=xc, box=box)
    x = np.concatenate([xc, xw], 0)
    x = x + rng.normal(0.0, jitter, size=x.shape)
    sp = np.concatenate([sp_c, spw])
    mol = np.concatenate([np.zeros(n_chain, np.int32), molw])
    bonds = np.concatenate([bonds_c, bw], 0).astype(np.int32)
    r0 = np.concatenate([r0_c, r0w])
    return System(name, _f32(x), sp, mol, bonds, r0, box)


def capped_molecule_in_droplet(n_solute: int, seed: int, jitter: float = 0.05,
                               name: str = "droplet") -> System:
    """Small molecule of exactly `n_solute` atoms (heavy self-avoiding chain,
    species drawn 32:9:10:1 from C:N:O:S, hydrogen caps up to valence as far
    as the count allows, each cap placed 1.6 A or more from other atoms when
    possible) surrounded by `n_solute` waters (3x its atom count
    in water atoms) packed around it at about 1 g/cm^3; open boundary."""
    rng = np.random.default_rng(seed)
    heavy_p = np.array([32, 9, 10, 1], np.float64)
    heavy_codes = np.array([SP_C, SP_N, SP_O, SP_S])
    # number of heavy atoms: grow until heavy + caps reaches n_solute
    n_heavy = 1
    sp_heavy = [int(rng.choice(heavy_codes, p=heavy_p / heavy_p.sum()))]
    def n_caps(sp_list):
        tot = 0
        for k, s in enumerate(sp_list):
            nb = (k > 0) + (k < len(sp_list) - 1)
            tot += max(VALENCE[s] - nb, 0)
        return tot
    while n_heavy + n_caps(sp_heavy) < n_solute:
        sp_heavy.append(int(rng.choice(heavy_codes, p=heavy_p / heavy_p.sum())))
        n_heavy += 1
    walk = _excluded_volume_walk(rng, n_heavy, CHAIN_BOND) if n_heavy > 1 else np.zeros((1, 3))
    xh = walk - walk.mean(0)
    xs, sps, bonds, r0 = [*xh], [*sp_heavy], [], []
    for k in range(n_heavy - 1):
        bonds.append((k, k + 1))
        r0.append(CHAIN_BOND)
    budget = n_solute - n_heavy
    for k, s in enumerate(sp_heavy):
        nb = (k > 0) + (k < n_heavy - 1)
        for _c in range(max(VALENCE[s] - nb, 0)):
            if budget == 0:
                break
            # cap direction: best of up to 200 seeded draws (first one that
            # keeps the cap 1.6 A from every other atom placed so far)
            placed = np.array(xs)
            best, best_d = None, -1.0
            for _try in range(200):
                u = rng.normal(size=3)
                u /= np.linalg.norm(u)
                c_ = xh[k] + CAP_BOND * u
                d = np.linalg.norm(placed - c_, axis=1)
                d[k] = 9.0
                if d.min() > best_d:
                    best, best_d = c_, d.min()
                if d.min() >= 1.6:
                    break
            cand = best
            xs.append(cand)
            sps.append(SP_H)
            bonds.append((k, len(xs) - 1))
            r0.append(CAP_BOND)
            budget -= 1
    xs = np.array(xs)
    sps = np.array(sps, np.uint8)
    n_w = n_solute
    spacing = (3.0 / WATER_ATOM_DENSITY) ** (1.0 / 3.0)
    rad = (np.abs(xs).max() + 3.0)
    while True:
        m = int(math.ceil(2 * rad / spacing)) + 1
        g = (np.arange(m) - (m - 1) / 2.0) * spacing
        grid = np.stack(np.meshgrid(g, g, g, indexing="ij"), -1).reshape(-1, 3)
        grid = grid[np.linalg.norm(grid, axis=1) <= rad]
        ok = _min_image_dist_ok(grid, xs, None, 2.5)
        if ok.sum() >= n_w:
            break
        rad += spacing
    acc = grid[ok]
    acc = acc[np.argsort(np.linalg.norm(acc, axis=1), kind="stable")][:n_w]
    xw, spw, molw, bw, r0w = _place_waters(rng, acc, 1, n_solute, obstacles=xs)
    x = np.concatenate([xs, xw], 0)
    x = x + rng.normal(0.0, jitter, size=x.shape)
    sp = np.concatenate([sps, spw])
    mol = np.concatenate([np.zeros(n_solute, np.int32), molw])
    b = np.concatenate([np.array(bonds, np.int32).reshape(-1, 2), bw], 0).astype(np.int32)
    rr = np.concatenate([np.array(r0), r0w])
    return System(name, _f32(x), sp, mol, b, rr, np.zeros(3))


def maxwell_boltzmann(masses: np.ndarray, temperature: float, seed: int) -> np.ndarray:
    """Velocities (A/fs) drawn from Maxwell-Boltzmann at `temperature` for the
    given simulation masses, with the mass-weighted centre-of-mass velocity
    removed; rounded to float32."""
    rng = np.random.default_rng(seed)
    sig = np.sqrt(KB_KCAL * temperature * ACC_CONV / masses)
    v = rng.normal(size=(masses.shape[0], 3)) * sig[:, None]
    vcm = (masses[:, None] * v).sum(0) / masses.sum()
    return _f32(v - vcm)


# --------------------------------------------------------------------------
# Model weights. Both models are random-init stand-ins (no trained weights are
# available); the layout of the flat blobs is the one the C ABI documents.
# --------------------------------------------------------------------------

def expected_neighbours(rc: float) -> float:
    return WATER_ATOM_DENSITY * 4.0 / 3.0 * math.pi * rc ** 3


@dataclasses.dataclass
class ModelSpec:
    """Hyper-parameters of a message-passing model (conservative or NC)."""

    L: int                 # message-passing layers
    C: int                 # channels
    lmax: int              # highest spherical-harmonic order
    K: int                 # Bessel functions (= n_s scalar heads for the NC head)
    rc: float              # cutoff (A)
    p: int                 # polynomial envelope exponent
    nu: float              # message normalisation (multiplies the neighbour sum)
    scale: float           # output scale (energy for conservative, force for NC)
    n_c: int = 0           # NC: attention dimension
    n_l: int = 0           # NC: tensor heads
    n_species: int = N_SPECIES
    bf16: bool = False     # MLP contractions in bf16 on the tensor cores (fp32 accumulate)
    bf16_plain: bool = False   # with bf16: one bf16 rounding per operand instead of hi + lo pairs


def cons_spec(L, C, lmax, K=8, rc=5.0, p=6, scale=1e-2, bf16=False, bf16_plain=False) -> ModelSpec:
    return ModelSpec(L, C, lmax, K, rc, p, 1.0 / math.sqrt(expected_neighbours(rc)), scale,
                     bf16=bf16, bf16_plain=bf16_plain)


def nc_spec(C, K=8, rc=4.0, p=5, n_c=8, n_l=2, scale=1e-2, bf16=False, bf16_plain=False) -> ModelSpec:
    return ModelSpec(1, C, 1, K, rc, p, 1.0 / math.sqrt(expected_neighbours(rc)), scale,
                     n_c=n_c, n_l=n_l, bf16=bf16, bf16_plain=bf16_plain)


def _xavier(rng, fan_out, fan_in, shape=None, gain=1.0):
    a = gain * math.sqrt(6.0 / (fan_in + fan_out))
    return rng.uniform(-a, a, size=shape if shape is not None else (fan_out, fan_in))


def cons_weights(spec: ModelSpec, seed: int) -> np.ndarray:
    """Flat float64 blob for the conservative model:
    emb[S][C]; per layer: wrad[lmax+1][K][C], w1[C][(lmax+1)C], b1[C],
    w2[C][C], b2[C]; readout: wr[C][C], br[C], wo[C]."""
    rng = np.random.default_rng(seed)
    S, C, L, nl1, K = spec.n_species, spec.C, spec.L, spec.lmax + 1, spec.K
    parts = [rng.uniform(-math.sqrt(3), math.sqrt(3), size=(S, C))]
    for _t in range(L):
        parts.append(rng.uniform(-2.0, 2.0, size=(nl1, K, C)))
        parts.append(_xavier(rng, C, nl1 * C))
        parts.append(np.zeros(C))
        parts.append(_xavier(rng, C, C))
        parts.append(np.zeros(C))
    parts.append(_xavier(rng, C, C))
    parts.append(np.zeros(C))
    parts.append(_xavier(rng, 1, C, shape=(C,)))
    return np.concatenate([p.ravel() for p in parts]).astype(np.float32).astype(np.float64)


def nc_weights(spec: ModelSpec, seed: int) -> np.ndarray:
    """Flat float64 blob for the NC model:
    emb[S][C]; layer: wrad[2][K][C], w1[C][2C], b1[C], w2[C][C], b2[C];
    U[n_l][C]; Wq[H][n_c][C]; Wk[H][n_c][C] with H = K + n_l."""
    rng = np.random.default_rng(seed)
    S, C, K = spec.n_species, spec.C, spec.K
    H = K + spec.n_l
    parts = [rng.uniform(-math.sqrt(3), math.sqrt(3), size=(S, C)),
             rng.uniform(-2.0, 2.0, size=(2, K, C)),
             _xavier(rng, C, 2 * C), np.zeros(C), _xavier(rng, C, C), np.zeros(C),
             _xavier(rng, spec.n_l, C),
             _xavier(rng, spec.n_c, C, shape=(H, spec.n_c, C)),
             _xavier(rng, spec.n_c, C, shape=(H, spec.n_c, C))]
    return np.concatenate([p.ravel() for p in parts]).astype(np.float32).astype(np.float64)


def cons_blob_len(spec: ModelSpec) -> int:
    S, C, L, nl1, K = spec.n_species, spec.C, spec.L, spec.lmax + 1, spec.K
    return S * C + L * (nl1 * K * C + nl1 * C * C + C + C * C + C) + C * C + 2 * C


def nc_blob_len(spec: ModelSpec) -> int:
    S, C, K = spec.n_species, spec.C, spec.K
    H = K + spec.n_l
    return S * C + 2 * K * C + 2 * C * C + C + C * C + C + spec.n_l * C + 2 * H * spec.n_c * C


# --------------------------------------------------------------------------
# Workload recipes (sizes and seeds of the synthetic stand-ins).
# --------------------------------------------------------------------------

@dataclasses.dataclass
class IntegratorSpec:
    dt_outer: float            # Delta (fs); for single-time-step runs, the step
    n_inner: int               # n (1 for single-time-step runs)
    temperature: float         # K
    gamma_ps: tuple            # friction per species code (1/ps)
    hmr_delta: float           # amu added to every H (0 = off)
    seed: int                  # Philox key


def water_192(seed=101):
    return water_box(64, 12.42, seed, name="water_192")


def water_12288(seed=201):
    return water_box(4096, 49.7, seed, name="water_12288")


def solvated_chain_23558(seed=301):
    return solvated_chain(seed=seed, name="solvated_chain_23558")


def water_100000(seed=501):
    return water_box(33333, 99.8, seed, n_lone_o=1, name="water_100000")


WORKLOADS = {
    "water_192": dict(system=water_192, sys_seed=101, w_seed=102, rng_seed=103,
                      cons=lambda: cons_spec(2, 64, 1), nc=lambda: nc_spec(32, rc=3.5),
                      dmts=IntegratorSpec(4.0, 4, 300.0, (1.0,) * 5, 0.0, 103),
                      sts=IntegratorSpec(1.0, 1, 300.0, (1.0,) * 5, 0.0, 103)),
    "water_12288": dict(system=water_12288, sys_seed=201, w_seed=202, rng_seed=203,
                        cons=lambda: cons_spec(3, 128, 2, bf16=True),
                        nc=lambda: nc_spec(64, rc=4.0, bf16=True),
                        dmts=IntegratorSpec(10.0, 5, 300.0, (20.0, 1.0, 1.0, 1.0, 1.0), 3.0, 203),
                        sts=IntegratorSpec(1.0, 1, 300.0, (1.0,) * 5, 0.0, 203)),
    "solvated_chain_23558": dict(system=solvated_chain_23558, sys_seed=301, w_seed=302,
                                 rng_seed=303,
                                 cons=lambda: cons_spec(3, 128, 2, bf16=True),
                                 nc=lambda: nc_spec(64, rc=4.0, bf16=True),
                                 dmts=IntegratorSpec(10.0, 5, 300.0, (20.0, 1.0, 1.0, 1.0, 1.0),
                                                     3.0, 303),
                                 sts=IntegratorSpec(1.0, 1, 300.0, (1.0,) * 5, 0.0, 303)),
    "water_100000": dict(system=water_100000, sys_seed=501, w_seed=502, rng_seed=503,
                         cons=lambda: cons_spec(3, 128, 2, bf16=True),
                         nc=lambda: nc_spec(64, rc=4.0, bf16=True),
                         dmts=IntegratorSpec(10.0, 5, 300.0, (20.0, 1.0, 1.0, 1.0, 1.0), 3.0, 503),
                         sts=IntegratorSpec(1.0, 1, 300.0, (1.0,) * 5, 0.0, 503)),
}


def serving_requests(n_req: int = 512, seed: int = 401, rate_per_s: float = 200.0,
                     atoms_lo: int = 20, atoms_hi: int = 400,
                     steps_lo: int = 50, steps_hi: int = 2000):
    """Replica requests: solute size and outer-step count log-uniform, Poisson
    arrivals (exponential gaps). Returns a list of dicts (systems built lazily
    by `capped_molecule_in_droplet(n_solute, seed)`)."""
    rng = np.random.default_rng(seed)
    n_sol = np.rint(np.exp(rng.uniform(math.log(atoms_lo), math.log(atoms_hi), n_req))).astype(int)
    n_steps = np.rint(np.exp(rng.uniform(math.log(steps_lo), math.log(steps_hi), n_req))).astype(int)
    gaps = rng.exponential(1.0 / rate_per_s, n_req)
    t = np.cumsum(gaps) - gaps[0]
    return [dict(id=k, n_solute=int(n_sol[k]), n_outer=int(n_steps[k]), arrival_s=float(t[k]),
                 sys_seed=seed * 1000 + k, rng_seed=403 * 10 ** 6 + k) for k in range(n_req)]
