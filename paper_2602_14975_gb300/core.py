"""Torch-facing binding of the C ABI (argument marshalling only).

Every step of the DMTS-NC path runs in libdmts.so; PyTorch provides device
memory and the current CUDA stream. Names follow the C ABI: nbr_build,
energy_forces_cons, forces_nc, respa_step, run_replicas.
"""
from __future__ import annotations

import ctypes as ct
import math

import numpy as np
import torch

from . import _lib as L


def _ptr(t):
    return ct.c_void_p(t.data_ptr()) if t is not None else ct.c_void_p(0)


def _stream(device=None):
    return ct.c_void_p(torch.cuda.current_stream(device).cuda_stream)


def _require_cuda(t: torch.Tensor, name: str):
    if not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")


def precision_of(spec) -> int:
    """dmts_precision of a model spec: fp32, split-bf16 or plain bf16."""
    if not spec.bf16:
        return L.FP32
    return L.BF16_PLAIN if getattr(spec, "bf16_plain", False) else L.BF16


def model_struct(spec, blob) -> tuple:
    w = np.ascontiguousarray(blob, dtype=np.float64)
    m = L.Model(spec.L, spec.C, spec.lmax, spec.K, spec.n_species, spec.n_c, spec.n_l,
                float(spec.rc), float(spec.p), float(spec.nu), float(spec.scale),
                precision_of(spec), w.ctypes.data_as(ct.POINTER(ct.c_double)), w.size)
    return m, w


# bond k, LJ eps, LJ sigma, LJ switch radius, LJ switch exponent, repulsion
# switch radius, repulsion switch exponent
DEFAULT_PRIOR = (450.0, 0.15, 3.15, 5.0, 6.0, 3.5, 6.0)


class Context:
    """Owns a dmts_ctx: both models uploaded to `device`."""

    def __init__(self, cons=None, nc=None, prior=DEFAULT_PRIOR, device: int = 0):
        self.lib = L.lib()
        self.device = device
        h = ct.c_void_p()
        keep = []
        cm = nm = None
        if cons is not None:
            cm, w = model_struct(*cons)
            keep.append(w)
        if nc is not None:
            nm, w = model_struct(*nc)
            keep.append(w)
        pr = L.Prior(*prior)
        st = self.lib.dmts_create(ct.byref(h), ct.byref(cm) if cm else None, ct.byref(nm) if nm else None,
                                  ct.byref(pr), device)
        L.check(st, None)
        self.handle = h
        self.cons_spec = cons[0] if cons is not None else None
        self.nc_spec = nc[0] if nc is not None else None
        self.nc_blob_len = len(nc[1]) if nc is not None else 0
        self.prior = prior

    def close(self):
        if getattr(self, "handle", None):
            self.lib.dmts_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def sync(self):
        L.check(self.lib.dmts_sync(self.handle, _stream()), self.handle)


def bond_table(n_atoms, bonds, r0):
    """Per-atom CSR bond table (both directions) built by the library's host helper."""
    bonds = np.ascontiguousarray(np.asarray(bonds, np.int32).reshape(-1, 2))
    r0 = np.ascontiguousarray(np.asarray(r0, np.float32))
    nb = bonds.shape[0]
    ptr = np.zeros(n_atoms + 1, np.int32)
    idx = np.zeros(max(1, 2 * nb), np.int32)
    rr = np.zeros(max(1, 2 * nb), np.float32)
    st = L.lib().dmts_bond_table(n_atoms, nb, bonds.ctypes.data, r0.ctypes.data, ptr.ctypes.data,
                                 idx.ctypes.data, rr.ctypes.data)
    L.check(st)
    return ptr, idx, rr


def masses_hmr(species, mol_id, masses, delta_h):
    """Hydrogen mass repartitioning by the library's host helper (FP64)."""
    sp = np.ascontiguousarray(species, np.uint8)
    mo = np.ascontiguousarray(mol_id, np.int32)
    m = np.ascontiguousarray(masses, np.float64)
    out = np.zeros_like(m)
    L.lib().dmts_masses_hmr(m.shape[0], sp.ctypes.data, mo.ctypes.data, m.ctypes.data, float(delta_h),
                            out.ctypes.data)
    return out


class DeviceSystem:
    """A batch of replicas resident on the device (concatenated atoms)."""

    def __init__(self, systems, device="cuda"):
        if not isinstance(systems, (list, tuple)):
            systems = [systems]
        self.systems = list(systems)
        counts = [s.n_atoms for s in systems]
        self.n_atoms = int(sum(counts))
        self.n_replicas = len(systems)
        off = np.concatenate([[0], np.cumsum(counts)]).astype(np.int32)
        self.rep_off_host = off
        x = np.concatenate([s.x for s in systems], 0).astype(np.float32)
        sp = np.concatenate([s.species for s in systems]).astype(np.uint8)
        mol = np.concatenate([s.mol_id for s in systems]).astype(np.int32)
        bonds = np.concatenate([s.bonds.reshape(-1, 2) + off[k] for k, s in enumerate(systems)], 0)
        r0 = np.concatenate([s.bond_r0 for s in systems])
        ptr, idx, rr = bond_table(self.n_atoms, bonds, r0)
        dev = torch.device(device)
        self.x = torch.from_numpy(x).to(dev)
        self.species = torch.from_numpy(sp).to(dev)
        self.mol_id = torch.from_numpy(mol).to(dev)
        self.rep_off = torch.from_numpy(off).to(dev)
        self.box = torch.from_numpy(np.stack([s.box for s in systems]).astype(np.float32)).to(dev)
        self.bond_ptr = torch.from_numpy(ptr).to(dev)
        self.bond_idx = torch.from_numpy(idx).to(dev)
        self.bond_r0 = torch.from_numpy(rr).to(dev)

    def struct(self) -> L.System:
        return L.System(self.n_atoms, self.n_replicas, _ptr(self.rep_off), _ptr(self.box), _ptr(self.x),
                        _ptr(self.species), _ptr(self.mol_id), _ptr(self.bond_ptr), _ptr(self.bond_idx),
                        _ptr(self.bond_r0))


class NbrList:
    def __init__(self, row_ptr, col, r_list):
        self.row_ptr, self.col, self.r_list = row_ptr, col, float(r_list)

    def struct(self):
        return L.Nbr(_ptr(self.row_ptr), _ptr(self.col), self.col.numel(), self.r_list)


def nbr_build(ctx: Context, dsys: DeviceSystem, r_list: float, capacity: int | None = None) -> NbrList:
    """Cell-list neighbour build; grows the capacity and retries on overflow."""
    dev = dsys.x.device
    if capacity is None:
        capacity = max(1024, 80 * dsys.n_atoms)
    while True:
        row = torch.empty(dsys.n_atoms + 1, dtype=torch.int32, device=dev)
        col = torch.empty(max(1, capacity), dtype=torch.int32, device=dev)
        nb = NbrList(row, col, r_list)
        s = dsys.struct()
        nbs = nb.struct()
        npairs = ct.c_longlong(0)
        st = ctx.lib.nbr_build(ctx.handle, ct.byref(s), ct.byref(nbs), ct.byref(npairs), _stream(dev))
        if st == L.E_NBR_OVERFLOW:
            capacity = int(npairs.value * 1.2) + 1024
            continue
        L.check(st, ctx.handle)
        nb.col = col[: max(1, npairs.value)]
        nb.n_pairs = int(npairs.value)
        return nb


def energy_forces_cons(ctx: Context, dsys: DeviceSystem, nbr: NbrList, with_prior=True, forces=True,
                       with_virial=False):
    """Returns (energy f64 [n_replicas], forces f32 [N,3] or None), and with
    with_virial the virial -sum_i F_i . q_i (pair form) f64 [n_replicas] as
    a third value."""
    dev = dsys.x.device
    E = torch.empty(dsys.n_replicas, dtype=torch.float64, device=dev)
    F = torch.empty(dsys.n_atoms, 3, dtype=torch.float32, device=dev) if forces else None
    W = torch.empty(dsys.n_replicas, dtype=torch.float64, device=dev) if with_virial else None
    s, nbs = dsys.struct(), nbr.struct()
    st = ctx.lib.energy_forces_cons(ctx.handle, ct.byref(s), ct.byref(nbs), _ptr(E), _ptr(F), _ptr(W),
                                    L.WITH_PRIOR if with_prior else 0, _stream(dev))
    L.check(st, ctx.handle)
    return (E, F, W) if with_virial else (E, F)


def nc_distill_step(ctx: Context, dsys: DeviceSystem, nbr: NbrList, target, lr: float = 0.0, step: int = 1,
                    params: int = L.FIT_QK | L.FIT_MLP | L.FIT_LAYER, with_grad: bool = False):
    """One distillation step of the NC model toward target forces (f32 [N,3]
    on the device), fitting `params` (L.FIT_QK: the head's q/k projection,
    L.FIT_MLP: its MLP, L.FIT_LAYER: the layer's radial weights and tensor-head
    mix): returns (loss f64 [n_replicas], the gradient f32 in
    the NC weight blob's layout or None); lr > 0 applies an Adam update."""
    dev = dsys.x.device
    target = torch.as_tensor(target, dtype=torch.float32, device=dev).contiguous()
    loss = torch.empty(dsys.n_replicas, dtype=torch.float64, device=dev)
    grad = None
    if with_grad:
        grad = torch.empty(int(ctx.nc_blob_len), dtype=torch.float32, device=dev)
    s, nbs = dsys.struct(), nbr.struct()
    st = ctx.lib.nc_distill_step(ctx.handle, ct.byref(s), ct.byref(nbs), _ptr(target), int(params), float(lr),
                                 int(step), _ptr(loss), _ptr(grad), _stream(dev))
    L.check(st, ctx.handle)
    return loss, grad


def forces_nc(ctx: Context, dsys: DeviceSystem, nbr: NbrList, with_bonds=True, with_virial=False):
    """Returns (F_NC f32 [N,3] mean-subtracted, net force f64 [R,3] before
    subtraction), and with with_virial the virial proxy f64 [R] as a third
    value."""
    dev = dsys.x.device
    F = torch.empty(dsys.n_atoms, 3, dtype=torch.float32, device=dev)
    net = torch.empty(dsys.n_replicas, 3, dtype=torch.float64, device=dev)
    W = torch.empty(dsys.n_replicas, dtype=torch.float64, device=dev) if with_virial else None
    s, nbs = dsys.struct(), nbr.struct()
    st = ctx.lib.forces_nc(ctx.handle, ct.byref(s), ct.byref(nbs), _ptr(F), _ptr(net), _ptr(W),
                           L.WITH_BONDS if with_bonds else 0, _stream(dev))
    L.check(st, ctx.handle)
    return (F, net, W) if with_virial else (F, net)


def integrator(dt_outer, n_inner, temperature, gamma_ps, mode=L.MODE_RESPA, skin=0.5,
               thermostat=L.LANGEVIN, barostat=False, pressure_atm=1.0, tau_p_ps=2.0) -> L.Integrator:
    """Integrator parameters; thermostat L.LANGEVIN or L.FFL (Fast Forward
    Langevin); barostat: the stochastic piston at pressure_atm with relaxation
    time tau_p_ps (the state needs virial=True, barostat=True)."""
    g = (ct.c_double * L.MAX_SPECIES)(*([float(v) for v in gamma_ps] + [0.0] * (L.MAX_SPECIES - len(gamma_ps))))
    return L.Integrator(float(dt_outer), int(n_inner), float(temperature), g, int(mode), float(skin),
                        int(thermostat), int(bool(barostat)), float(pressure_atm), float(tau_p_ps))


class MDState:
    """Device-resident dynamic state of a batch (positions live in dsys.x)."""

    def __init__(self, dsys: DeviceSystem, v, masses, seeds, replica_ids=None, steps=None, virial=False,
                 barostat=False, thermo=False, trace_rows=0):
        dev = dsys.x.device
        self.dsys = dsys
        self.v = torch.as_tensor(np.asarray(v, np.float32)).to(dev).contiguous()
        self.masses = torch.as_tensor(np.asarray(masses, np.float32)).to(dev).contiguous()
        R = dsys.n_replicas
        self.f_nc = torch.zeros(dsys.n_atoms, 3, dtype=torch.float32, device=dev)
        self.f_cons = torch.zeros(dsys.n_atoms, 3, dtype=torch.float32, device=dev)
        self.energy = torch.zeros(R, dtype=torch.float64, device=dev)
        seeds = np.broadcast_to(np.asarray(seeds, np.uint64), (R,)).copy()
        self.seed = torch.from_numpy(seeds.view(np.int64)).to(dev)
        rid = np.arange(R, dtype=np.uint32) if replica_ids is None else np.asarray(replica_ids, np.uint32)
        self.replica_id = torch.from_numpy(rid.view(np.int32)).to(dev)
        st0 = np.zeros(R, np.uint64) if steps is None else np.asarray(steps, np.uint64)
        self.step = torch.from_numpy(st0.view(np.int64)).to(dev)
        # with virial=True: average virial proxy of the fast force over the
        # inner steps of the last outer step (RESPA), the virial of the full
        # force at its last evaluation, and the estimator that combines them
        # at the end of each outer step, per replica
        self.virial_nc = torch.zeros(R, dtype=torch.float64, device=dev) if virial else None
        self.virial_cons = torch.zeros(R, dtype=torch.float64, device=dev) if virial else None
        self.virial_est = torch.zeros(R, dtype=torch.float64, device=dev) if virial else None
        # with barostat=True: per replica the piston momentum, its last force and a set flag
        self.baro = torch.zeros(R, 3, dtype=torch.float64, device=dev) if barostat else None
        # with thermo=True: per replica (K, U + K, T) at the end of each call,
        # FP64 on the device; with trace_rows > 0 also after every outer step
        # of a call (rows = outer steps, at most trace_rows per call)
        self.thermo = torch.zeros(R, 3, dtype=torch.float64, device=dev) if (thermo or trace_rows) else None
        self.thermo_trace = (torch.zeros(trace_rows, R, 3, dtype=torch.float64, device=dev)
                             if trace_rows else None)
        self.c = L.State(dsys.struct(), _ptr(self.v), _ptr(self.f_nc), _ptr(self.f_cons), _ptr(self.masses),
                         _ptr(self.energy), _ptr(self.step), _ptr(self.seed), _ptr(self.replica_id), 1, None,
                         _ptr(self.virial_nc), _ptr(self.virial_cons), _ptr(self.virial_est), _ptr(self.baro),
                         _ptr(self.thermo), _ptr(self.thermo_trace), int(trace_rows))
        self.ctx = None

    def lists(self, which: int) -> NbrList:
        """The neighbour list the state holds (0: conservative, 1: NC), as
        last built on the device; valid after the first respa_step."""
        if self.ctx is None:
            raise ValueError("the state holds no lists before its first respa_step")
        dev = self.dsys.x.device
        row = torch.empty(self.dsys.n_atoms + 1, dtype=torch.int32, device=dev)
        npairs, rl = ct.c_longlong(0), ct.c_float(0.0)
        st = self.ctx.lib.dmts_state_lists(self.ctx.handle, ct.byref(self.c), int(which), _ptr(row), None, 0,
                                           ct.byref(npairs), ct.byref(rl), _stream(dev))
        if st not in (L.OK, L.E_NBR_OVERFLOW):
            L.check(st, self.ctx.handle)
        col = torch.empty(max(1, npairs.value), dtype=torch.int32, device=dev)
        st = self.ctx.lib.dmts_state_lists(self.ctx.handle, ct.byref(self.c), int(which), _ptr(row), _ptr(col),
                                           col.numel(), ct.byref(npairs), ct.byref(rl), _stream(dev))
        L.check(st, self.ctx.handle)
        nb = NbrList(row, col[: max(1, npairs.value)], float(rl.value))
        nb.n_pairs = int(npairs.value)
        return nb

    def release(self):
        if self.ctx is not None and self.c.internal:
            self.ctx.lib.dmts_state_release(self.ctx.handle, ct.byref(self.c))


def respa_step(ctx: Context, state: MDState, integ: L.Integrator, n_outer: int):
    state.ctx = ctx
    st = ctx.lib.respa_step(ctx.handle, ct.byref(state.c), ct.byref(integ), int(n_outer),
                            _stream(state.v.device))
    L.check(st, ctx.handle)


def respa_guarded(ctx: Context, state: MDState, integ: L.Integrator, n_outer: int, threshold: float,
                  chunk_outer: int, sts_steps: int, sts_dt: float, cap: int = 4096) -> dict:
    """Algorithm 1 under the rewind guard (saved frame every chunk_outer
    outer steps; on max |F - F_S| > threshold or a non-finite value: back to
    the frame, sts_steps STS steps of sts_dt, then Algorithm 1 again).
    Returns {"n_rewinds", "n_chunks", "chunk_max", "rewind_at"}."""
    state.ctx = ctx
    g = L.Guard(float(threshold), int(chunk_outer), int(sts_steps), float(sts_dt))
    cm = np.zeros(cap, np.float32)
    ra = np.zeros(cap, np.float32)
    stats = L.GuardStats(0, 0, cm.ctypes.data, cap, ra.ctypes.data, cap)
    st = ctx.lib.respa_guarded(ctx.handle, ct.byref(state.c), ct.byref(integ), ct.byref(g), int(n_outer),
                               ct.byref(stats), _stream(state.v.device))
    L.check(st, ctx.handle)
    return {"n_rewinds": stats.n_rewinds, "n_chunks": stats.n_chunks,
            "chunk_max": cm[:min(stats.n_chunks, cap)].copy(), "rewind_at": ra[:min(stats.n_rewinds, cap)].copy()}


def philox_words(ctx, seed, replica, step, atom0, count):
    out = torch.empty(4 * count, dtype=torch.int32, device=f"cuda:{ctx.device}")
    L.check(ctx.lib.dmts_philox_words(ctx.handle, seed, replica, step, atom0, count, _ptr(out), _stream()),
            ctx.handle)
    return out


def gaussians(ctx, seed, replica, step, atom0, count):
    out = torch.empty(3 * count, dtype=torch.float32, device=f"cuda:{ctx.device}")
    L.check(ctx.lib.dmts_gaussians(ctx.handle, seed, replica, step, atom0, count, _ptr(out), _stream()),
            ctx.handle)
    return out


class ConsEnergy(torch.autograd.Function):
    """U(x) of the conservative model (+ prior) with the hand-written adjoint
    as its backward: forward returns the per-replica energies, backward
    returns -F * grad_output (F from the same call, per replica)."""

    @staticmethod
    def forward(fn_ctx, x, ctx: Context, dsys: DeviceSystem, nbr: NbrList, with_prior: bool = True):
        if x.data_ptr() != dsys.x.data_ptr():
            dsys.x.copy_(x.detach())
        E, F = energy_forces_cons(ctx, dsys, nbr, with_prior=with_prior, forces=True)
        fn_ctx.save_for_backward(F, dsys.rep_off)
        return E

    @staticmethod
    def backward(fn_ctx, gE):
        F, rep_off = fn_ctx.saved_tensors
        counts = (rep_off[1:] - rep_off[:-1]).long()
        g = torch.repeat_interleave(gE.to(F.dtype), counts)
        return -F * g[:, None], None, None, None, None


def profile_enable(ctx: Context, on: bool = True, every: int = 1):
    """Per-kernel CUDA-event timing inside the library (measurement support);
    with every = N > 1 only every N-th outer step of respa_step is timed."""
    L.check(ctx.lib.dmts_profile_enable(ctx.handle, max(1, int(every)) if on else 0), ctx.handle)


def kernel_launches(ctx: Context) -> int:
    """Kernels the library has launched in this process so far (all
    contexts); the difference of two reads counts a region's launches."""
    return int(ctx.lib.dmts_kernel_launches())


def profile_read(ctx: Context) -> dict:
    """{kernel: (launches, total_ms)} since the last profile_enable(True)."""
    n = ctx.lib.dmts_profile_read(ctx.handle, -1, None, 0, None, None)
    out = {}
    buf = ct.create_string_buffer(64)
    for k in range(max(n, 0)):
        la = ct.c_longlong(0)
        ms = ct.c_double(0.0)
        ctx.lib.dmts_profile_read(ctx.handle, k, buf, 64, ct.byref(la), ct.byref(ms))
        out[buf.value.decode()] = (int(la.value), float(ms.value))
    return out


class ReplicaRequest:
    """One serving request: a system, its initial velocities and simulation
    masses, the number of outer steps, its noise seed and id, and its arrival
    time (s, relative to the start of the run)."""

    def __init__(self, system, v, masses, n_outer, seed, replica_id, arrival_s=0.0):
        self.system = system
        self.x = np.ascontiguousarray(system.x, np.float32)
        self.v = np.ascontiguousarray(v, np.float32)
        self.species = np.ascontiguousarray(system.species, np.uint8)
        self.mol_id = np.ascontiguousarray(system.mol_id, np.int32)
        self.bonds = np.ascontiguousarray(system.bonds.reshape(-1, 2), np.int32)
        self.bond_r0 = np.ascontiguousarray(system.bond_r0, np.float32)
        self.masses = np.ascontiguousarray(masses, np.float32)
        self.n_outer, self.seed, self.replica_id = int(n_outer), int(seed), int(replica_id)
        self.arrival_s = float(arrival_s)

    def struct(self):
        box = (ct.c_float * 3)(*[float(b) for b in self.system.box])
        return L.Request(self.x.shape[0], self.x.ctypes.data, self.v.ctypes.data, self.species.ctypes.data,
                         self.mol_id.ctypes.data, self.bonds.shape[0], self.bonds.ctypes.data,
                         self.bond_r0.ctypes.data, self.masses.ctypes.data, box, self.n_outer,
                         self.seed, self.replica_id, self.arrival_s)


def run_replicas(ctx: Context, requests, integ: L.Integrator, hbm_budget_bytes: int = 64 << 30,
                 max_slots: int = 512, realtime: bool = False, tick_cap: int = 1 << 20):
    """Continuous-batching serving loop. Returns (results, stats): results[k]
    = dict(x, v, energy, t_arrival_s, t_admit_s, t_done_s, status); stats =
    dict(tick_ms, tick_atoms, n_ticks, wall_s, atom_outer_steps, max_resident),
    tick_atoms being the atoms of the packed batch each tick integrated."""
    n = len(requests)
    reqs = (L.Request * max(1, n))(*[r.struct() for r in requests])
    xs = [np.zeros_like(r.x) for r in requests]
    vs = [np.zeros_like(r.v) for r in requests]
    res = (L.Result * max(1, n))()
    for k in range(n):
        res[k].x = xs[k].ctypes.data
        res[k].v = vs[k].ctypes.data
    ticks = np.zeros(tick_cap, np.float64)
    tick_atoms = np.zeros(tick_cap, np.int32)
    stats = L.ServeStats(ticks.ctypes.data, tick_cap, 0, 0.0, 0.0, 0, tick_atoms.ctypes.data)
    cfg = L.ServeCfg(int(hbm_budget_bytes), int(max_slots), 1 if realtime else 0)
    st = ctx.lib.run_replicas(ctx.handle, reqs, n, ct.byref(integ), ct.byref(cfg), res, ct.byref(stats))
    L.check(st, ctx.handle)
    out = [dict(x=xs[k], v=vs[k], energy=res[k].energy, t_arrival_s=res[k].t_arrival_s,
                t_admit_s=res[k].t_admit_s, t_done_s=res[k].t_done_s, status=res[k].status) for k in range(n)]
    nt = min(stats.n_ticks, tick_cap)
    return out, dict(tick_ms=ticks[:nt].copy(), tick_atoms=tick_atoms[:nt].copy(), n_ticks=stats.n_ticks,
                     wall_s=stats.wall_s,
                     atom_outer_steps=stats.atom_outer_steps, max_resident=stats.max_resident)


def replica_footprint(ctx: Context, n_atoms: int) -> int:
    return int(ctx.lib.dmts_replica_footprint(ctx.handle, int(n_atoms)))


def contract_bf16(ctx: Context, act: torch.Tensor, wt: torch.Tensor, split: bool = False) -> torch.Tensor:
    """out = act @ wt.T on the tensor cores (bf16 operands, fp32 accumulate).

    split=True: act [M][2K] and wt [N][2K] hold hi | lo pairs per row and
    out = act_hi wt_hi^T + act_lo wt_hi^T + act_hi wt_lo^T."""
    assert act.dtype == torch.bfloat16 and wt.dtype == torch.bfloat16
    act, wt = act.contiguous(), wt.contiguous()
    M, K = act.shape
    N = wt.shape[0]
    if split:
        K //= 2
    out = torch.empty(M, N, dtype=torch.float32, device=act.device)
    L.check(ctx.lib.dmts_contract_bf16(ctx.handle, M, N, K, _ptr(act), _ptr(wt), _ptr(out), int(split),
                                       _stream(act.device)), ctx.handle)
    return out


def check_bounded_wait(ctx: Context, limit_us: int) -> int:
    """Runs the library's bounded mbarrier wait on a barrier nothing arrives
    on (limit_us microseconds) and returns the status dmts_sync then reports
    (DMTS_E_TIMEOUT expected); the sticky error word is cleared."""
    L.check(ctx.lib.dmts_check_bounded_wait(ctx.handle, int(limit_us), _stream()), ctx.handle)
    return int(ctx.lib.dmts_sync(ctx.handle, _stream()))
