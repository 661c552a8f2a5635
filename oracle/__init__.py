"""FP64 CPU oracle of the DMTS-NC hot path (test infrastructure).

Only the tests, the smoke check and the CPU-baseline leg of the benchmark may
import this package. The product path never does. The C source
`dmts_oracle.c` is compiled with gcc into `oracle/_build/` on first use (or by
`build()`), without -ffast-math so that IEEE double semantics hold.

Every wrapper takes numpy arrays and a `synth.ModelSpec`-like object and returns
float64 results.
"""
from __future__ import annotations

import ctypes as ct
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "dmts_oracle.c")
_OUT = os.path.join(_HERE, "_build", "libdmts_oracle.so")
_lock = threading.Lock()
_lib = None

# prior constants: bond k (kcal/mol/A^2), LJ epsilon (kcal/mol), sigma (A),
# LJ switch radius (A), LJ switch exponent, repulsion switch radius (A),
# repulsion switch exponent
PRIOR = np.array([450.0, 0.15, 3.15, 5.0, 6.0, 3.5, 6.0])
BONDS, LJ, REP = 1, 2, 4


def build(force: bool = False) -> str:
    os.makedirs(os.path.dirname(_OUT), exist_ok=True)
    if force or not os.path.exists(_OUT) or os.path.getmtime(_OUT) < os.path.getmtime(_SRC):
        tmp = _OUT + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-std=c11", "-D_DEFAULT_SOURCE",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _OUT)
    return _OUT


def lib():
    global _lib
    with _lock:
        if _lib is None:
            _lib = ct.CDLL(build())
            _declare(_lib)
    return _lib


_D = ct.POINTER(ct.c_double)
_I = ct.POINTER(ct.c_int)
_U8 = ct.POINTER(ct.c_uint8)
_U32 = ct.POINTER(ct.c_uint32)
_U64 = ct.POINTER(ct.c_uint64)


def _declare(L):
    L.orc_nbr_brute.restype = ct.c_long
    L.orc_nbr_brute.argtypes = [ct.c_int, _D, _D, ct.c_double, _I, _I, ct.c_long]
    for name in ("orc_cons_energy", "orc_cons_energy_forces"):
        f = getattr(L, name)
        f.restype = ct.c_double
        f.argtypes = [ct.c_int, _D, _U8, _D, _I, _D, _D, _D]
    L.orc_prior.restype = ct.c_double
    L.orc_prior.argtypes = [ct.c_int, _D, _U8, _I, _D, ct.c_int, _I, _D, _D, ct.c_int, _D, _D]
    L.orc_nc_forces.restype = None
    L.orc_nc_forces.argtypes = [ct.c_int, _D, _U8, _D, _I, _D, _D, ct.c_int, _I, _D, _D, ct.c_int, _D, _D, _D]
    L.orc_zbl_phi.restype = ct.c_double
    L.orc_zbl_phi.argtypes = [ct.c_double]
    L.orc_rep_pair.restype = ct.c_double
    L.orc_rep_pair.argtypes = [ct.c_int, ct.c_int, ct.c_double, ct.c_double, ct.c_double, _D]
    L.orc_philox4x32_10.restype = None
    L.orc_philox4x32_10.argtypes = [_U32, _U32, _U32]
    L.orc_noise_words.restype = None
    L.orc_noise_words.argtypes = [ct.c_uint64, ct.c_uint32, ct.c_uint64, ct.c_uint32, _U32]
    L.orc_gauss3.restype = None
    L.orc_gauss3.argtypes = [ct.c_uint64, ct.c_uint32, ct.c_uint64, ct.c_uint32, _D]
    L.orc_hmr_masses.restype = None
    L.orc_hmr_masses.argtypes = [ct.c_int, _U8, _I, _D, ct.c_double, _D]
    L.orc_gamma_table.restype = None
    L.orc_gamma_table.argtypes = [ct.c_int, _D, ct.c_double, ct.c_double, _D, _D]
    for name in ("orc_bessel", "orc_dbessel"):
        f = getattr(L, name)
        f.restype = ct.c_double
        f.argtypes = [ct.c_int, ct.c_double, ct.c_double]
    for name in ("orc_envelope", "orc_denvelope"):
        f = getattr(L, name)
        f.restype = ct.c_double
        f.argtypes = [ct.c_double, ct.c_double]
    L.orc_sph.restype = None
    L.orc_sph.argtypes = [_D, _D]
    L.orc_respa_run.restype = ct.c_double
    L.orc_respa_run.argtypes = [_I, _D, ct.c_uint64, _U8, _I, _D, _I, _D, _D,
                                _I, _D, _D, _I, _D, _D, _D, _D,
                                ct.c_int, _D, _D, _D, _D, _U64, _I, _D, _D, _D, _D]
    L.orc_baro_mass.restype = ct.c_double
    L.orc_baro_mass.argtypes = [ct.c_int, ct.c_double, ct.c_double]
    L.orc_baro_force.restype = ct.c_double
    L.orc_baro_force.argtypes = [ct.c_int, ct.c_double, ct.c_double, _D, ct.c_double]
    L.orc_kinetic.restype = ct.c_double
    L.orc_kinetic.argtypes = [ct.c_int, _D, _D]
    L.orc_baro_drift.restype = None
    L.orc_baro_drift.argtypes = [ct.c_int, _D, _D, _D, ct.c_double, ct.c_double, ct.c_double]
    L.orc_sts_run.restype = ct.c_double
    L.orc_sts_run.argtypes = [_I, _D, ct.c_uint64, _U8, _I, _D, _I, _D, _D,
                              _I, _D, _D, _D, _D, ct.c_int, _D, _D, _D, _U64, _I]


def _d(a):
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a, a.ctypes.data_as(_D)


def _i(a):
    a = np.ascontiguousarray(a, dtype=np.int32)
    return a, a.ctypes.data_as(_I)


def _u8(a):
    a = np.ascontiguousarray(a, dtype=np.uint8)
    return a, a.ctypes.data_as(_U8)


def model_ints(spec) -> np.ndarray:
    return np.array([spec.L, spec.C, spec.lmax, spec.K, spec.n_species, spec.n_c, spec.n_l],
                    np.int32)


def model_reals(spec) -> np.ndarray:
    return np.array([spec.rc, float(spec.p), spec.nu, spec.scale], np.float64)


# ---------------------------------------------------------------- wrappers --

def nbr_brute(x, box, rcut):
    """Full neighbour list (row_ptr, col), rows ascending in j."""
    L = lib()
    x, px = _d(x)
    box, pb = _d(box)
    n = x.shape[0]
    cap = max(16, n * 64)
    while True:
        rp = np.zeros(n + 1, np.int32)
        col = np.zeros(cap, np.int32)
        e = L.orc_nbr_brute(n, px, pb, float(rcut), rp.ctypes.data_as(_I), col.ctypes.data_as(_I), cap)
        if e >= 0:
            return rp, col[:e].copy()
        cap = -e


def cons_energy(sys, spec, blob, per_atom=False):
    L = lib()
    x, px = _d(sys.x)
    sp, ps = _u8(sys.species)
    box, pb = _d(sys.box)
    mi, pmi = _i(model_ints(spec))
    mr, pmr = _d(model_reals(spec))
    w, pw = _d(blob)
    e = np.zeros(x.shape[0])
    E = L.orc_cons_energy(x.shape[0], px, ps, pb, pmi, pmr, pw, e.ctypes.data_as(_D))
    return (E, e) if per_atom else E


def cons_energy_forces(sys, spec, blob):
    L = lib()
    x, px = _d(sys.x)
    sp, ps = _u8(sys.species)
    box, pb = _d(sys.box)
    mi, pmi = _i(model_ints(spec))
    mr, pmr = _d(model_reals(spec))
    w, pw = _d(blob)
    F = np.zeros((x.shape[0], 3))
    E = L.orc_cons_energy_forces(x.shape[0], px, ps, pb, pmi, pmr, pw, F.ctypes.data_as(_D))
    return E, F


def prior(sys, with_lj=True, consts=PRIOR, terms=None):
    """Analytic terms of U: bonds | LJ | screened repulsion (default all
    three; with_lj=False keeps bonds + repulsion)."""
    if terms is None:
        terms = BONDS | REP | (LJ if with_lj else 0)
    L = lib()
    x, px = _d(sys.x)
    sp, ps = _u8(sys.species)
    mol, pm = _i(sys.mol_id)
    box, pb = _d(sys.box)
    b, pbd = _i(sys.bonds.reshape(-1, 2))
    r0, pr0 = _d(sys.bond_r0)
    c, pc = _d(consts)
    F = np.zeros((x.shape[0], 3))
    E = L.orc_prior(x.shape[0], px, ps, pm, pb, b.shape[0], pbd, pr0, pc, int(terms),
                    F.ctypes.data_as(_D), None)
    return E, F


def prior_virial(sys, terms, consts=PRIOR):
    """Virial proxy -sum_i F_i . q_i of the analytic terms, in pair form
    (sum over pairs of r dE/dr)."""
    L = lib()
    x, px = _d(sys.x)
    sp, ps = _u8(sys.species)
    mol, pm = _i(sys.mol_id)
    box, pb = _d(sys.box)
    b, pbd = _i(sys.bonds.reshape(-1, 2))
    r0, pr0 = _d(sys.bond_r0)
    c, pc = _d(consts)
    W = ct.c_double(0.0)
    L.orc_prior(x.shape[0], px, ps, pm, pb, b.shape[0], pbd, pr0, pc, int(terms), None, ct.byref(W))
    return W.value


def nc_forces(sys, spec, blob, with_bonds=True, consts=PRIOR, fast_terms=None, with_virial=False):
    """Returns (F after mean subtraction, net force before subtraction), and
    the virial proxy sum_i sum_j F_ij . r_ij (+ pair form of the fast terms)
    as a third value with with_virial.
    fast_terms: prior terms added to the NC force (default bonds + repulsion,
    none when with_bonds is False)."""
    if fast_terms is None:
        fast_terms = (BONDS | REP) if with_bonds else 0
    L = lib()
    x, px = _d(sys.x)
    sp, ps = _u8(sys.species)
    box, pb = _d(sys.box)
    mi, pmi = _i(model_ints(spec))
    mr, pmr = _d(model_reals(spec))
    w, pw = _d(blob)
    b, pbd = _i(sys.bonds.reshape(-1, 2))
    r0, pr0 = _d(sys.bond_r0)
    c, pc = _d(consts)
    F = np.zeros((x.shape[0], 3))
    net = np.zeros(3)
    W = ct.c_double(0.0)
    L.orc_nc_forces(x.shape[0], px, ps, pb, pmi, pmr, pw, b.shape[0], pbd,
                    pr0, pc, int(fast_terms), F.ctypes.data_as(_D), net.ctypes.data_as(_D), ct.byref(W))
    return (F, net, W.value) if with_virial else (F, net)


def philox4x32_10(ctr, key):
    L = lib()
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, np.uint32)
    L.orc_philox4x32_10(c.ctypes.data_as(_U32), k.ctypes.data_as(_U32), out.ctypes.data_as(_U32))
    return out


def noise_words(seed, replica, step, atom):
    out = np.zeros(4, np.uint32)
    lib().orc_noise_words(seed, replica, step, atom, out.ctypes.data_as(_U32))
    return out


def gauss3(seed, replica, step, atom):
    g = np.zeros(3)
    lib().orc_gauss3(seed, replica, step, atom, g.ctypes.data_as(_D))
    return g


def hmr_masses(species, mol_id, masses, delta_h):
    L = lib()
    sp, ps = _u8(species)
    mol, pm = _i(mol_id)
    m, pmm = _d(masses)
    out = np.zeros(m.shape[0])
    L.orc_hmr_masses(m.shape[0], ps, pm, pmm, float(delta_h), out.ctypes.data_as(_D))
    return out


def gamma_table(gamma_ps, dt_fs, T):
    g, pg = _d(gamma_ps)
    c1 = np.zeros(g.shape[0])
    c2 = np.zeros(g.shape[0])
    lib().orc_gamma_table(g.shape[0], pg, float(dt_fs), float(T), c1.ctypes.data_as(_D),
                          c2.ctypes.data_as(_D))
    return c1, c2


def bessel(k, r, rc):
    return lib().orc_bessel(k, r, rc)


def dbessel(k, r, rc):
    return lib().orc_dbessel(k, r, rc)


def envelope(u, p):
    return lib().orc_envelope(u, float(p))


def denvelope(u, p):
    return lib().orc_denvelope(u, float(p))


def zbl_phi(x):
    return lib().orc_zbl_phi(float(x))


def rep_pair(si, sj, r, rc=PRIOR[5], p=PRIOR[6]):
    """(E_rep, dE/dr) of one pair."""
    d = ct.c_double(0.0)
    e = lib().orc_rep_pair(int(si), int(sj), float(r), float(rc), float(p), ct.byref(d))
    return e, d.value


def sph(n):
    n, pn = _d(n)
    Y = np.zeros(9)
    lib().orc_sph(pn, Y.ctypes.data_as(_D))
    return Y


class MDState:
    """Host FP64 state carried between oracle integrator calls."""

    def __init__(self, sys, v, masses):
        self.x = np.array(sys.x, dtype=np.float64)
        self.v = np.array(v, dtype=np.float64)
        self.F = np.zeros_like(self.x)
        self.F_nc = np.zeros_like(self.x)
        self.masses = np.array(masses, dtype=np.float64)
        self.step = ct.c_uint64(0)
        self.first = ct.c_int(1)


LANGEVIN, FFL = 0, 1


def respa_run(state, sys, cons_spec, cons_blob, nc_spec, nc_blob, dt_outer, n_inner, T,
              gamma_ps, seed, n_outer, replica=0, inner_mode=0, outer_mode=0, consts=PRIOR,
              thermostat=LANGEVIN, virial_avg=None, barostat=None):
    """Algorithm 1 for n_outer outer steps; returns the last potential energy.
    virial_avg (a ctypes double, optional) receives the average virial proxy
    of the fast force over the inner steps of the last outer step.
    barostat (optional): (P_ext atm, tau_P ps, box, baro) with box a float64
    [3] array the piston moves and baro = [p_eps, G, have_G] float64, both
    updated in place (a periodic system only).
    inner_mode: 0 NC + bonds, 1 full -grad U (collapse to BAOAB), 2 bonds only.
    outer_mode: 0 -grad(U_MP + prior), 1 bonds only.
    thermostat: LANGEVIN or FFL (Fast Forward Langevin O-step)."""
    L = lib()
    ints, pi = _i([sys.n_atoms, sys.bonds.shape[0], inner_mode, outer_mode, n_inner, replica, thermostat])
    reals, pr = _d([dt_outer, T])
    sp, ps = _u8(sys.species)
    mol, pm = _i(sys.mol_id)
    box, pb = _d(sys.box)
    b, pbd = _i(sys.bonds.reshape(-1, 2))
    r0, pr0 = _d(sys.bond_r0)
    c, pc = _d(consts)
    cmi, pcmi = _i(model_ints(cons_spec))
    cmr, pcmr = _d(model_reals(cons_spec))
    cb, pcb = _d(cons_blob)
    nmi, pnmi = _i(model_ints(nc_spec))
    nmr, pnmr = _d(model_reals(nc_spec))
    nb, pnb = _d(nc_blob)
    m, pmm = _d(state.masses)
    g, pg = _d(gamma_ps)
    return L.orc_respa_run(pi, pr, ct.c_uint64(seed), ps, pm, pb, pbd, pr0, pc,
                           pcmi, pcmr, pcb, pnmi, pnmr, pnb, pmm, pg, int(n_outer),
                           state.x.ctypes.data_as(_D), state.v.ctypes.data_as(_D),
                           state.F.ctypes.data_as(_D), state.F_nc.ctypes.data_as(_D),
                           ct.byref(state.step), ct.byref(state.first),
                           ct.byref(virial_avg) if virial_avg is not None else None,
                           *_baro_args(barostat))


def _baro_args(barostat):
    if barostat is None:
        return None, None, None
    p_atm, tau_ps, box_io, baro = barostat
    assert box_io.dtype == np.float64 and baro.dtype == np.float64 and box_io.flags.c_contiguous
    par = np.array([p_atm, tau_ps], np.float64)
    _baro_args.keep = par
    return par.ctypes.data_as(_D), box_io.ctypes.data_as(_D), baro.ctypes.data_as(_D)


def baro_mass(n, T, tau_p_fs):
    L = lib()
    return L.orc_baro_mass(int(n), float(T), float(tau_p_fs))


def baro_force(n, K, wvir, box, p_atm):
    b, pb = _d(box)
    return lib().orc_baro_force(int(n), float(K), float(wvir), pb, float(p_atm))


def kinetic(v, mass):
    vv, pv = _d(np.asarray(v).reshape(-1))
    m, pm = _d(mass)
    return lib().orc_kinetic(len(m), pv, pm)


def baro_drift(x, v, box, h, b, a):
    """In place on float64 arrays x [n,3], v [n,3], box [3]."""
    lib().orc_baro_drift(x.shape[0], x.ctypes.data_as(_D), v.ctypes.data_as(_D), box.ctypes.data_as(_D),
                         float(h), float(b), float(a))


def sts_run(state, sys, cons_spec, cons_blob, dt, T, gamma_ps, seed, n_steps, replica=0,
            outer_mode=0, consts=PRIOR, thermostat=LANGEVIN):
    """Single-time-step BAOAB for n_steps steps; returns the last potential energy."""
    L = lib()
    ints, pi = _i([sys.n_atoms, sys.bonds.shape[0], outer_mode, replica, thermostat])
    reals, pr = _d([dt, T])
    sp, ps = _u8(sys.species)
    mol, pm = _i(sys.mol_id)
    box, pb = _d(sys.box)
    b, pbd = _i(sys.bonds.reshape(-1, 2))
    r0, pr0 = _d(sys.bond_r0)
    c, pc = _d(consts)
    cmi, pcmi = _i(model_ints(cons_spec))
    cmr, pcmr = _d(model_reals(cons_spec))
    cb, pcb = _d(cons_blob)
    m, pmm = _d(state.masses)
    g, pg = _d(gamma_ps)
    return L.orc_sts_run(pi, pr, ct.c_uint64(seed), ps, pm, pb, pbd, pr0, pc,
                         pcmi, pcmr, pcb, pmm, pg, int(n_steps),
                         state.x.ctypes.data_as(_D), state.v.ctypes.data_as(_D),
                         state.F.ctypes.data_as(_D), ct.byref(state.step), ct.byref(state.first))
