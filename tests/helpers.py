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
