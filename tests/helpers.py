"""Shared fixtures for the GPU tests: workloads, oracle references, tolerances."""
import copy

import numpy as np

from paper_2602_14975_gb300 import synth as S

# Tolerances stated for the path: FP32 forces within 1e-5 relative max-abs of
# the oracle; BF16 paths within 2e-3 of the force RMS; positions within 1e-4 A
# after 10 outer steps.
TOL_F32 = 1e-5
TOL_BF16_RMS = 2e-3
TOL_POS = 1e-4


def rel_maxabs(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-30))


def with_x(sy, x):
    s2 = copy.deepcopy(sy)
    s2.x = np.asarray(x, np.float64)
    return s2


def pair_set(row_ptr, col, offset=0):
    row_ptr = np.asarray(row_ptr)
    col = np.asarray(col)
    out = set()
    for i in range(len(row_ptr) - 1):
        for j in col[row_ptr[i]:row_ptr[i + 1]]:
            out.add((i + offset, int(j) + offset))
    return out


def band_pairs(sy, pairs, rcut, eps=1e-4):
    """Pairs whose |d|^2 lies within eps of rcut^2 (FP32 vs FP64 may differ)."""
    out = set()
    for (i, j) in pairs:
        d = sy.x[j] - sy.x[i]
        if sy.box[0] > 0:
            d = d - sy.box * np.rint(d / sy.box)
        if abs(float(d @ d) - rcut * rcut) < eps:
            out.add((i, j))
    return out


def cluster_around(sy, center, radius):
    """Atoms within `radius` (minimum image) of atom `center`, unwrapped
    around it, as an open-boundary system; bonds inside the cluster kept.
    Returns (system, index of the centre in it)."""
    d = sy.x - sy.x[center]
    d -= sy.box * np.round(d / sy.box)
    keep = np.nonzero((d ** 2).sum(1) < radius ** 2)[0]
    remap = -np.ones(sy.n_atoms, np.int64)
    remap[keep] = np.arange(keep.size)
    b = sy.bonds
    bm = (remap[b[:, 0]] >= 0) & (remap[b[:, 1]] >= 0)
    sub = S.System(f"{sy.name}_around_{center}", sy.x[center] + d[keep], sy.species[keep], sy.mol_id[keep],
                   remap[b[bm]].astype(np.int32), sy.bond_r0[bm], np.zeros(3))
    return sub, int(remap[center])
