"""ctypes mirror of include/dmts.h and the loader of libdmts.so.

The library is the in-tree build of the CUDA sources; there is no fallback:
if it cannot be built or loaded, every call raises.
"""
from __future__ import annotations

import ctypes as ct
import os
import threading

_lock = threading.Lock()
_lib = None

MAX_SPECIES = 8

OK, E_INVALID, E_OOM, E_CUDA, E_NBR_OVERFLOW, E_NONFINITE, E_TIMEOUT, E_BUSY = range(8)
FIT_QK, FIT_MLP, FIT_LAYER = 1, 2, 4   # nc_distill_step: weights to fit
STATUS_NAMES = {0: "OK", 1: "E_INVALID", 2: "E_OOM", 3: "E_CUDA", 4: "E_NBR_OVERFLOW",
                5: "E_NONFINITE", 6: "E_TIMEOUT", 7: "E_BUSY"}
FP32, BF16, BF16_PLAIN = 0, 1, 2
MODE_RESPA, MODE_STS = 0, 1
LANGEVIN, FFL = 0, 1
WITH_PRIOR = 1
WITH_BONDS = 1


class Model(ct.Structure):
    _fields_ = [("L", ct.c_int), ("C", ct.c_int), ("lmax", ct.c_int), ("K", ct.c_int),
                ("n_species", ct.c_int), ("n_c", ct.c_int), ("n_l", ct.c_int),
                ("rc", ct.c_float), ("p_env", ct.c_float), ("nu", ct.c_float), ("scale", ct.c_float),
                ("precision", ct.c_int), ("weights", ct.POINTER(ct.c_double)),
                ("n_weights", ct.c_longlong)]


class Prior(ct.Structure):
    _fields_ = [("k_bond", ct.c_float), ("lj_eps", ct.c_float), ("lj_sigma", ct.c_float),
                ("lj_rc", ct.c_float), ("lj_p", ct.c_float), ("rep_rc", ct.c_float), ("rep_p", ct.c_float)]


class System(ct.Structure):
    _fields_ = [("n_atoms", ct.c_int), ("n_replicas", ct.c_int), ("rep_off", ct.c_void_p),
                ("box", ct.c_void_p), ("x", ct.c_void_p), ("species", ct.c_void_p),
                ("mol_id", ct.c_void_p), ("bond_ptr", ct.c_void_p), ("bond_idx", ct.c_void_p),
                ("bond_r0", ct.c_void_p)]


class Nbr(ct.Structure):
    _fields_ = [("row_ptr", ct.c_void_p), ("col", ct.c_void_p), ("capacity", ct.c_longlong),
                ("r_list", ct.c_float)]


class Integrator(ct.Structure):
    _fields_ = [("dt_outer", ct.c_float), ("n_inner", ct.c_int), ("temperature", ct.c_float),
                ("gamma_ps", ct.c_double * MAX_SPECIES), ("mode", ct.c_int), ("skin", ct.c_float),
                ("thermostat", ct.c_int), ("barostat", ct.c_int), ("pressure_atm", ct.c_float),
                ("tau_p_ps", ct.c_float)]


class Guard(ct.Structure):
    _fields_ = [("threshold", ct.c_float), ("chunk_outer", ct.c_int), ("sts_steps", ct.c_int),
                ("sts_dt", ct.c_float)]


class GuardStats(ct.Structure):
    _fields_ = [("n_rewinds", ct.c_int), ("n_chunks", ct.c_int), ("chunk_max", ct.c_void_p),
                ("chunk_cap", ct.c_int), ("rewind_at", ct.c_void_p), ("rewind_cap", ct.c_int)]


class State(ct.Structure):
    _fields_ = [("sys", System), ("v", ct.c_void_p), ("f_nc", ct.c_void_p), ("f_cons", ct.c_void_p),
                ("masses", ct.c_void_p), ("energy", ct.c_void_p), ("step", ct.c_void_p),
                ("seed", ct.c_void_p), ("replica_id", ct.c_void_p), ("first_step", ct.c_int),
                ("internal", ct.c_void_p), ("virial_nc", ct.c_void_p), ("virial_cons", ct.c_void_p),
                ("virial_est", ct.c_void_p), ("baro", ct.c_void_p), ("thermo", ct.c_void_p),
                ("thermo_trace", ct.c_void_p), ("thermo_trace_rows", ct.c_int)]


class Request(ct.Structure):
    _fields_ = [("n_atoms", ct.c_int), ("x", ct.c_void_p), ("v", ct.c_void_p), ("species", ct.c_void_p),
                ("mol_id", ct.c_void_p), ("n_bonds", ct.c_int), ("bonds", ct.c_void_p),
                ("bond_r0", ct.c_void_p), ("masses", ct.c_void_p), ("box", ct.c_float * 3),
                ("n_outer", ct.c_int), ("seed", ct.c_uint64), ("replica_id", ct.c_uint32),
                ("arrival_s", ct.c_double)]


class ServeCfg(ct.Structure):
    _fields_ = [("hbm_budget_bytes", ct.c_longlong), ("max_slots", ct.c_int), ("realtime", ct.c_int)]


class Result(ct.Structure):
    _fields_ = [("x", ct.c_void_p), ("v", ct.c_void_p), ("energy", ct.c_double),
                ("t_arrival_s", ct.c_double), ("t_admit_s", ct.c_double), ("t_done_s", ct.c_double),
                ("status", ct.c_int)]


class ServeStats(ct.Structure):
    _fields_ = [("tick_ms", ct.c_void_p), ("tick_cap", ct.c_int), ("n_ticks", ct.c_int),
                ("wall_s", ct.c_double), ("atom_outer_steps", ct.c_double), ("max_resident", ct.c_int),
                ("tick_atoms", ct.c_void_p)]


# every entry point declared in include/dmts.h
EXPORTS = ("dmts_create", "dmts_destroy", "dmts_last_error", "dmts_sync", "nbr_build",
           "energy_forces_cons", "forces_nc", "respa_step", "dmts_state_release", "dmts_state_lists", "nc_distill_step", "run_replicas",
           "dmts_masses_hmr", "dmts_bond_table", "dmts_philox_words", "dmts_gaussians",
           "dmts_replica_footprint", "dmts_profile_enable", "dmts_profile_read", "nbr_build_noalloc",
           "dmts_contract_bf16", "dmts_kernel_launches", "respa_guarded", "dmts_check_bounded_wait")


def lib_path() -> str:
    return os.path.join(os.path.dirname(os.path.abspath(__file__)), "_build", "libdmts.so")


def _declare(L):
    vp, i, f, d = ct.c_void_p, ct.c_int, ct.c_float, ct.c_double
    L.dmts_create.restype = i
    L.dmts_create.argtypes = [ct.POINTER(vp), ct.POINTER(Model), ct.POINTER(Model), ct.POINTER(Prior), i]
    L.dmts_destroy.restype = None
    L.dmts_kernel_launches.restype = ct.c_ulonglong
    L.dmts_kernel_launches.argtypes = []
    L.dmts_destroy.argtypes = [vp]
    L.dmts_last_error.restype = ct.c_char_p
    L.dmts_last_error.argtypes = [vp]
    L.dmts_sync.restype = i
    L.dmts_sync.argtypes = [vp, vp]
    L.nbr_build.restype = i
    L.nbr_build.argtypes = [vp, ct.POINTER(System), ct.POINTER(Nbr), ct.POINTER(ct.c_longlong), vp]
    L.energy_forces_cons.restype = i
    L.energy_forces_cons.argtypes = [vp, ct.POINTER(System), ct.POINTER(Nbr), vp, vp, vp, i, vp]
    L.forces_nc.restype = i
    L.forces_nc.argtypes = [vp, ct.POINTER(System), ct.POINTER(Nbr), vp, vp, vp, i, vp]
    L.respa_step.restype = i
    L.respa_step.argtypes = [vp, ct.POINTER(State), ct.POINTER(Integrator), i, vp]
    L.respa_guarded.restype = i
    L.respa_guarded.argtypes = [vp, ct.POINTER(State), ct.POINTER(Integrator), ct.POINTER(Guard), i,
                                ct.POINTER(GuardStats), vp]
    L.dmts_state_release.restype = None
    L.dmts_state_release.argtypes = [vp, ct.POINTER(State)]
    L.nc_distill_step.restype = i
    L.nc_distill_step.argtypes = [vp, ct.POINTER(System), ct.POINTER(Nbr), vp, i, ct.c_float, i, vp, vp, vp]
    L.dmts_state_lists.restype = i
    L.dmts_state_lists.argtypes = [vp, ct.POINTER(State), i, vp, vp, ct.c_longlong, ct.POINTER(ct.c_longlong),
                                   ct.POINTER(ct.c_float), vp]
    L.run_replicas.restype = i
    L.run_replicas.argtypes = [vp, ct.POINTER(Request), i, ct.POINTER(Integrator), ct.POINTER(ServeCfg),
                               ct.POINTER(Result), ct.POINTER(ServeStats)]
    L.dmts_masses_hmr.restype = None
    L.dmts_masses_hmr.argtypes = [i, vp, vp, vp, d, vp]
    L.dmts_bond_table.restype = i
    L.dmts_bond_table.argtypes = [i, i, vp, vp, vp, vp, vp]
    L.dmts_philox_words.restype = i
    L.dmts_philox_words.argtypes = [vp, ct.c_uint64, ct.c_uint32, ct.c_uint64, ct.c_uint32, i, vp, vp]
    L.dmts_gaussians.restype = i
    L.dmts_gaussians.argtypes = [vp, ct.c_uint64, ct.c_uint32, ct.c_uint64, ct.c_uint32, i, vp, vp]
    L.dmts_replica_footprint.restype = ct.c_longlong
    L.dmts_replica_footprint.argtypes = [vp, i]
    L.dmts_contract_bf16.restype = i
    L.dmts_contract_bf16.argtypes = [vp, i, i, i, vp, vp, vp, i, vp]
    L.dmts_check_bounded_wait.restype = i
    L.dmts_check_bounded_wait.argtypes = [vp, i, vp]
    L.nbr_build_noalloc.restype = i
    L.nbr_build_noalloc.argtypes = [ct.POINTER(System), ct.POINTER(Nbr), ct.POINTER(ct.c_longlong), vp]
    L.dmts_profile_enable.restype = i
    L.dmts_profile_enable.argtypes = [vp, i]
    L.dmts_profile_read.restype = i
    L.dmts_profile_read.argtypes = [vp, i, ct.c_char_p, i, ct.POINTER(ct.c_longlong), ct.POINTER(ct.c_double)]


def lib(build_if_missing: bool = True):
    """Loads libdmts.so (building it in-tree if needed). Raises if it cannot."""
    global _lib
    with _lock:
        if _lib is None:
            path = lib_path()
            if build_if_missing:
                from . import buildlib as _build
                path = _build.build()
            if not os.path.exists(path):
                raise RuntimeError(f"libdmts.so not found at {path}; run build()")
            L = ct.CDLL(path)
            _declare(L)
            _lib = L
    return _lib


class DmtsError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


def check(status, ctx=None):
    if status != OK:
        msg = lib().dmts_last_error(ctx)
        raise DmtsError(status, msg.decode() if msg else "")
