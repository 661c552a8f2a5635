"""Benchmark of the DMTS-NC hot path on one GB300 (or N, one replica each).

One step = one outer step of Algorithm 1 (one conservative evaluation with
its adjoint forces, n = 5 NC evaluations, the fused integrator, neighbour
rebuilds) on the 23,558-atom solvated bead chain in water. The same GPU also
runs single-time-step BAOAB (1 fs, no HMR) for the ns/day ratio.

Prints one JSON line (rank 0). `--impl reference` times the FP64 CPU oracle
instead, on a bounded cut-out of the same workload.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

WORKLOAD = "solvated_chain_23558"
LARGE_WORKLOAD = "water_100000"

# DRAM traffic per launch of the roofline kernel, dram__bytes_read.sum +
# dram__bytes_write.sum from one ncu capture of this bench's workload (the
# capture command and the counters are in profiles/). It is reported only
# while the kernel's sources hash to the recorded value; after any change to
# them it is null until a new capture is taken.
PROF_EVERY = 4   # time every 4th outer step of the timed region per kernel
KCAL_A3_PER_ATM = 101325.0 * 6.02214076e23 * 1e-30 / 4184.0   # 1 atm in kcal/mol/A^3

NCU_TRAFFIC = {
    "mp_bwd": {"bytes_per_launch": (153792768 + 14773248 + 154217472 + 12226560 + 141881088 + 280320) / 3,
               # the adjoint's code: channel-pack helpers, kernel and launch, the
               # argument structs, the device helpers
               "sources": [("paper_2602_14975_gb300/csrc/mp.cu", ("// ---- channel packs", "// ---- forward")),
                           ("paper_2602_14975_gb300/csrc/mp.cu", ("// ---- adjoint", "// In the forward pass")),
                           ("paper_2602_14975_gb300/csrc/mp.cu", ("template <int C, int LMAX, bool VIR, bool SG>",
                                                                  "#define DMTS_DISPATCH")),
                           ("paper_2602_14975_gb300/csrc/mp.cuh", ("struct EdgeGeom {", "template <int CPW>")),
                           ("paper_2602_14975_gb300/csrc/common.cuh", None)],
               "sha256": "3796c7e6556c549033dba13f00650618a0defe87a98c4c586074b1306b886a7e"},
}


def _kernel_text(text, name):
    """Source text of the __global__ function `name` (from its template line
    to the closing brace at column 0)."""
    at = text.index(f" {name}(")
    beg = text.rindex("template", 0, at)
    end = text.index("\n}\n", at) + 3
    return text[beg:end]


def _region(text, start, end):
    """Text from the line holding `start` up to the line holding `end`; both
    markers are matched after collapsing runs of dashes in comment rules."""
    import re
    norm = re.sub(r"-{4,}", "----", text)
    beg = norm.index(start)
    beg = norm.rindex("\n", 0, beg) + 1
    stop = norm.index(end, beg + len(start))
    return norm[beg:stop]


def sources_sha256(sources):
    """Hash of the code a recorded capture depends on: a whole file (None), a
    __global__ function by name, or a region between two markers."""
    import hashlib
    h = hashlib.sha256()
    for path, spec in sources:
        with open(os.path.join(ROOT, path), encoding="utf-8") as f:
            text = f.read()
        if spec is None:
            part = text
        elif isinstance(spec, tuple):
            part = _region(text, *spec)
        else:
            part = _kernel_text(text, spec)
        h.update(part.encode())
    return h.hexdigest()


def ncu_traffic(kernel):
    rec = NCU_TRAFFIC.get(kernel)
    if not rec or rec["bytes_per_launch"] is None:
        return None
    return rec["bytes_per_launch"] if sources_sha256(rec["sources"]) == rec["sha256"] else None


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default=WORKLOAD)
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU-baseline leg")
    return ap.parse_args()


def ns_per_day(fs_per_step, steps_per_s):
    return fs_per_step * steps_per_s * 86400.0 / 1e6


# ----------------------------------------------------------------- clocks --
class ClockSampler:
    """nvidia-smi sampling of SM clock and throttle reasons during a region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append((float(parts[1]), float(parts[2]), parts[5:9]))
            except ValueError:
                continue
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for _, _, flags in rows for k, f in enumerate(flags) if f == "Active"})
        return {"sm_mhz": float(np.median([r[0] for r in rows])), "sm_max_mhz": max(r[1] for r in rows),
                "samples": len(rows), "reasons": reasons}


# ------------------------------------------------------------- CPU oracle --
def cutout(sy, frac_edge):
    """Atoms of whole molecules whose first atom lies in [0, frac_edge*L)^3
    (wrapped); bonds re-indexed; same box."""
    from paper_2602_14975_gb300 import synth as S
    xw = np.mod(sy.x, sy.box)
    lim = frac_edge * sy.box
    keep_mol = set()
    seen = set()
    for i in range(sy.n_atoms):
        m = int(sy.mol_id[i])
        if m in seen:
            continue
        seen.add(m)
        if np.all(xw[i] < lim):
            keep_mol.add(m)
    keep = np.array([int(sy.mol_id[i]) in keep_mol for i in range(sy.n_atoms)])
    if sy.mol_id[0] == 0 and 0 not in keep_mol:
        # the chain is one molecule: keep its beads inside the cut-out region
        keep |= (sy.mol_id == 0) & np.all(xw < lim, axis=1)
    idx = np.nonzero(keep)[0]
    remap = -np.ones(sy.n_atoms, np.int64)
    remap[idx] = np.arange(idx.size)
    b = sy.bonds
    bm = keep[b[:, 0]] & keep[b[:, 1]]
    return S.System(sy.name + "_cutout", sy.x[idx], sy.species[idx], sy.mol_id[idx],
                    remap[b[bm]].astype(np.int32), sy.bond_r0[bm], sy.box)


def oracle_outer_step_seconds(sy, W, frac_edge):
    """Times the oracle's force evaluations of one DMTS-NC outer step (one
    conservative energy+forces, n NC evaluations) on a cut-out; returns
    (seconds per outer step scaled to the full system, sample description)."""
    import oracle as O
    from paper_2602_14975_gb300 import synth as S
    sub = cutout(sy, frac_edge)
    cs, ns = W["cons"](), W["nc"]()
    cb, nb = S.cons_weights(cs, W["w_seed"]), S.nc_weights(ns, W["w_seed"])
    n_in = W["dmts"].n_inner
    t0 = time.perf_counter()
    O.cons_energy_forces(sub, cs, cb)
    O.prior(sub)
    t1 = time.perf_counter()
    O.nc_forces(sub, ns, nb)
    t2 = time.perf_counter()
    per_outer = (t1 - t0) + n_in * (t2 - t1)
    scale = sy.n_atoms / sub.n_atoms
    desc = (f"oracle (FP64 C, 1 thread): 1 conservative E+F + 1 NC evaluation timed on a "
            f"{sub.n_atoms}-atom cut-out ({frac_edge:.3f} of the box edge) of {sy.name}; "
            f"outer step = t_cons + {n_in} t_nc, scaled x{scale:.2f} to {sy.n_atoms} atoms")
    return per_outer * scale, desc


def workload_config(sy, I, cs, ns):
    """The `config` of the JSON line (the same for both arms)."""
    return {"workload": sy.name, "n_atoms": sy.n_atoms,
            "integrator": f"DMTS-NC outer {I.dt_outer} fs / {I.n_inner} inner, HMR +{I.hmr_delta} amu on H, "
                          f"gamma_H {I.gamma_ps[0]}/ps, gamma_heavy {I.gamma_ps[1]}/ps",
            "cons_model": f"L={cs.L} C={cs.C} lmax={cs.lmax} K={cs.K} rc={cs.rc}",
            "nc_model": f"C={ns.C} lmax=1 rc={ns.rc} n_c={ns.n_c} n_l={ns.n_l}",
            "precision": ("bf16 MLP contractions on the tensor cores (tcgen05, fp32 accumulate), "
                          "fp32 everywhere else, fp64 per-replica sums") if cs.bf16 else "fp32",
            "l2": "inputs larger than L2: about 0.5 GB of node and edge data per outer step",
            "parallelism": "replicas only (one replica per GPU)"}


# Bytes per atom that one k_integrate launch reads and writes (fp32 vectors
# of 12 B): an inner step reads the mass (4), v, F_NC, x, the
# replica index (4), the species (1) and the rebuild check's reference
# positions and writes x and v: 57 + 24; the launch that also applies the
# outer kick reads the cached full force too (69 + 24); the closing launch of
# a call reads mass, v, F_NC and the full force and writes v (40 + 12).
INTEG_B_INNER, INTEG_B_KICK, INTEG_B_CLOSE = 81, 93, 52


def integ_bytes_per_outer_step(n_inner, with_close):
    return INTEG_B_KICK + INTEG_B_INNER * (n_inner - 1) + (INTEG_B_CLOSE if with_close else 0)


def serving_roofline(prof, atom_outer_steps, n_inner, cs):
    """Per-kernel rates inside the serving loop, where one launch covers every
    resident replica (often 10^5 atoms or more): the integrator against HBM
    (one call per outer step: n_inner launches and the closing one) and the
    conservative contractions against the bf16 tensor peak."""
    pk = {}
    pk_path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(pk_path):
        pk = json.load(open(pk_path))
    out = {}
    t_int = prof.get("integrate", (0, 0.0))[1] * 1e-3
    if t_int > 0:
        gbs = integ_bytes_per_outer_step(n_inner, True) * atom_outer_steps / t_int / 1e9
        out["integrate"] = {"row": "a8", "bound": "hbm", "gbs": gbs,
                            "frac_hbm": gbs / pk["hbm_gbs"] if pk.get("hbm_gbs") else None}
    t_g = prof.get("gemm_tc", (0, 0.0))[1] * 1e-3
    if t_g > 0:
        nl = cs.lmax + 1
        tf = 2.0 * cs.C * cs.C * (2 * cs.L * (nl + 1) + 2) * atom_outer_steps / t_g / 1e12
        out["gemm_tc"] = {"row": "a4", "bound": "tensor", "tflops": tf,
                          "frac_bf16_sustained": tf / pk["bf16_tflops_sustained"] if pk.get("bf16_tflops_sustained") else None}
    tot = sum(v[1] for v in prof.values()) or 1.0
    out["shares"] = {k: round(v[1] / tot, 4) for k, v in sorted(prof.items(), key=lambda kv: -kv[1][1])}
    return out


# ------------------------------------------------------------------ main --
def main():
    args = parse()
    from paper_2602_14975_gb300 import dist as D
    from paper_2602_14975_gb300 import synth as S
    world, rank, local = D.world()
    W = S.WORKLOADS[args.workload]
    I = W["dmts"]

    if args.impl == "reference":
        if rank != 0:
            return 0
        sy = W["system"]()
        # size the per-step cut-out so that warm-up + timed steps take about
        # two minutes (cost grows linearly with the cut-out's atom count)
        t_cal, _ = oracle_outer_step_seconds(sy, W, 0.25)
        n_cal = cutout(sy, 0.25).n_atoms
        t_cal_sample = t_cal * n_cal / sy.n_atoms
        budget = 120.0 / max(1, args.steps + args.warmup)
        frac = min(1.0 / 3.0, 0.25 * (budget / max(t_cal_sample, 1e-3)) ** (1.0 / 3.0))
        for _ in range(args.warmup):
            oracle_outer_step_seconds(sy, W, frac)
        t0 = time.perf_counter()
        per = []
        for _ in range(args.steps):
            s, desc = oracle_outer_step_seconds(sy, W, frac)
            per.append(s)
        wall = time.perf_counter() - t0
        t_outer = float(np.mean(per))
        val = ns_per_day(I.dt_outer, 1.0 / t_outer)
        line = {"impl": "reference", "metric": "ns/day (DMTS-NC)", "value": val, "unit": "ns/day",
                "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": t_outer * 1e3, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                "config": workload_config(sy, I, W["cons"](), W["nc"]()),
                "cpu_baseline": {"value": val, "unit": "ns/day", "cores": 1, "kind": "oracle", "sample": desc},
                "e2e": {"value": val, "unit": "ns/day", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
                "wall_s": wall}
        print(json.dumps(line), flush=True)
        return 0

    import torch
    torch.cuda.set_device(local)
    D.init("nccl", torch.device(f"cuda:{local}"))
    from paper_2602_14975_gb300 import core

    sy = W["system"]()
    cs, ns = W["cons"](), W["nc"]()    # bf16 MLP contractions on the tensor cores
    cb, nb = S.cons_weights(cs, W["w_seed"]), S.nc_weights(ns, W["w_seed"])
    ctx = core.Context(cons=(cs, cb), nc=(ns, nb), device=local)

    dev = torch.device(f"cuda:{local}")

    def barrier():
        D.barrier(dev)

    def max_over_ranks(v):
        return D.max_over_ranks(v, dev)

    # algorithmic work of the dominant kernels (active edges within the cutoffs)
    d0 = core.DeviceSystem(sy)
    e_cons = core.nbr_build(ctx, d0, cs.rc).n_pairs
    e_nc = core.nbr_build(ctx, d0, ns.rc).n_pairs
    del d0

    # ---------------------------------------------------------- DMTS-NC
    m_hmr = core.masses_hmr(sy.species, sy.mol_id, sy.element_masses(), I.hmr_delta)
    v0 = S.maxwell_boltzmann(m_hmr, I.temperature, W["rng_seed"])
    dsys = core.DeviceSystem(sy)
    st = core.MDState(dsys, v0, m_hmr.astype(np.float32), seeds=I.seed, replica_ids=[D.replica_id(rank, 0)])
    skin = 0.5    # Verlet skin (A); rebuilds are gated on half-skin displacement
    integ = core.integrator(I.dt_outer, I.n_inner, I.temperature, I.gamma_ps, skin=skin)
    core.respa_step(ctx, st, integ, args.warmup)
    ctx.sync()
    clocks = ClockSampler(local)
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    # per-kernel events on every PROF_EVERY-th outer step of the timed
    # region (events on every step cost about 4 % of the step time)
    core.profile_enable(ctx, True, every=PROF_EVERY)
    n_prof = (args.steps + PROF_EVERY - 1) // PROF_EVERY
    barrier()
    clocks.start()
    torch.cuda.nvtx.range_push("dmts_outer_steps")    # the timed region, for ncu --nvtx-include
    launches0 = core.kernel_launches(ctx)
    e0.record(stream)
    core.respa_step(ctx, st, integ, args.steps)
    e1.record(stream)
    n_launches = core.kernel_launches(ctx) - launches0
    torch.cuda.nvtx.range_pop()
    barrier()
    ck = clocks.stop()
    ctx.sync()
    prof = core.profile_read(ctx)
    core.profile_enable(ctx, False)
    ms_dmts = max_over_ranks(e0.elapsed_time(e1)) / args.steps
    st.release()

    # ------------------------------------- rewind guard, FFL thermostat
    # the same outer step under the rewind guard (saved frame and monitor
    # read every 50 outer steps, no disagreement), and with the Fast Forward
    # Langevin O-step
    n_side = max(10, args.steps // 2)
    side = {}
    for label, th in (("guarded", 0), ("ffl", 1)):
        dg = core.DeviceSystem(W["system"]())
        sg = core.MDState(dg, v0, m_hmr.astype(np.float32), seeds=I.seed, replica_ids=[D.replica_id(rank, 0)])
        ig = core.integrator(I.dt_outer, I.n_inner, I.temperature, I.gamma_ps, skin=skin,
                             thermostat=core.L.FFL if th else core.L.LANGEVIN)
        core.respa_step(ctx, sg, ig, 2)
        ctx.sync()
        barrier()
        e0.record(stream)
        if label == "guarded":
            gs = core.respa_guarded(ctx, sg, ig, n_side, math.inf, 50, 4 * I.n_inner, I.dt_outer / I.n_inner)
        else:
            core.respa_step(ctx, sg, ig, n_side)
        e1.record(stream)
        barrier()
        ctx.sync()
        ms = max_over_ranks(e0.elapsed_time(e1)) / n_side
        side[label] = {"ns_per_day": ns_per_day(I.dt_outer, 1e3 / ms) * world, "ms_per_step": ms, "steps": n_side}
        if label == "guarded":
            side[label].update({"chunk_outer": 50, "rewinds": gs["n_rewinds"],
                                "max_force_disagreement": float(np.max(gs["chunk_max"])) if gs["n_chunks"] else None})
        sg.release()

    # --------------------------------------------------------------- NPT
    # the same outer step with the barostat (piston relaxation time 2 ps as in
    # the paper's NPT runs). The random-weight stand-in models sit far from
    # 1 atm, so the target is their instantaneous pressure at the start (the
    # full force's virial and the kinetic energy), which keeps the box near
    # its size over the run
    dn = core.DeviceSystem(W["system"]())
    sn = core.MDState(dn, v0, m_hmr.astype(np.float32), seeds=I.seed, replica_ids=[D.replica_id(rank, 0)],
                      virial=True, barostat=True)
    i_init = core.integrator(I.dt_outer, I.n_inner, I.temperature, I.gamma_ps, skin=skin, barostat=True)
    core.respa_step(ctx, sn, i_init, 0)      # lists (with the piston's cell margin) and first forces
    ctx.sync()
    k_start = 0.5 * float((m_hmr[:, None] * v0 ** 2).sum()) / 4.184e-4
    p_start = (2 * k_start - float(sn.virial_cons[0].item())) / (3 * float(np.prod(sy.box))) / KCAL_A3_PER_ATM
    i_npt = core.integrator(I.dt_outer, I.n_inner, I.temperature, I.gamma_ps, skin=skin, barostat=True,
                            pressure_atm=p_start, tau_p_ps=2.0)
    core.respa_step(ctx, sn, i_npt, 2)
    ctx.sync()
    barrier()
    e0.record(stream)
    core.respa_step(ctx, sn, i_npt, n_side)
    e1.record(stream)
    barrier()
    ctx.sync()
    ms = max_over_ranks(e0.elapsed_time(e1)) / n_side
    box_end = dn.box.cpu().numpy().reshape(-1)
    side["npt"] = {"ns_per_day": ns_per_day(I.dt_outer, 1e3 / ms) * world, "ms_per_step": ms, "steps": n_side,
                   "pressure_atm": p_start, "tau_p_ps": 2.0,
                   "box_change": float(box_end[0] / sy.box[0] - 1.0)}
    sn.release()

    # ------------------------------------------------------- distillation
    # on-box distillation of the NC model (every weight but the embedding)
    # toward the full force: frames 10 single time steps apart from a BAOAB run of the
    # conservative model, 4 for training and 1 held out; |F_L| = |F - F_S| on
    # the held-out frame before and after 60 Adam steps
    ctxD = core.Context(cons=(cs, cb), nc=(ns, nb))
    dF = core.DeviceSystem(W["system"]())
    sF = core.MDState(dF, v0, m_hmr.astype(np.float32), seeds=I.seed + 7, replica_ids=[D.replica_id(rank, 0)])
    iF = core.integrator(1.0, 1, I.temperature, I.gamma_ps, mode=1, skin=skin)
    frames = []
    for _ in range(5):
        core.respa_step(ctxD, sF, iF, 10)
        df = core.DeviceSystem(W["system"]())
        df.x.copy_(dF.x)
        nbc = core.nbr_build(ctxD, df, cs.rc + 0.5)
        _, tf = core.energy_forces_cons(ctxD, df, nbc, with_prior=True)
        frames.append((df, core.nbr_build(ctxD, df, ns.rc + 0.5), tf))
    sF.release()
    ctx.sync()

    def f_l_rms(fr):
        lv, _ = core.nc_distill_step(ctxD, fr[0], fr[1], fr[2], lr=0.0)
        return math.sqrt(lv.item() / (3 * fr[0].n_atoms))

    rms0 = f_l_rms(frames[4])
    n_dist = 60
    barrier()
    e0.record(stream)
    for k in range(n_dist):
        fr = frames[k % 4]
        core.nc_distill_step(ctxD, fr[0], fr[1], fr[2], lr=1e-3, step=k + 1)
    e1.record(stream)
    barrier()
    ctx.sync()
    ms_dist = max_over_ranks(e0.elapsed_time(e1)) / n_dist
    rms1 = f_l_rms(frames[4])
    side["distill"] = {"what": "every NC weight but the species embedding (W_rad, U, W1, b1, W2, b2, W_qk) fitted to "
                               "the full force (Adam, lr 1e-3)",
                       "train_frames": 4, "steps": n_dist, "ms_per_step": ms_dist,
                       "f_l_rms_held_out_before": rms0, "f_l_rms_held_out_after": rms1,
                       "unit": "kcal/mol/A"}
    del frames, ctxD

    # --------------------------------------------------------------- STS
    sts = W["sts"]
    m_el = sy.element_masses()
    sy2 = W["system"]()
    d2 = core.DeviceSystem(sy2)
    st2 = core.MDState(d2, S.maxwell_boltzmann(m_el, sts.temperature, W["rng_seed"]),
                       m_el.astype(np.float32), seeds=sts.seed, replica_ids=[D.replica_id(rank, 0)])
    integ2 = core.integrator(sts.dt_outer, 1, sts.temperature, sts.gamma_ps, mode=1, skin=skin)
    n_sts = max(10, args.steps)
    core.respa_step(ctx, st2, integ2, args.warmup)
    ctx.sync()
    barrier()
    e0.record(stream)
    core.respa_step(ctx, st2, integ2, n_sts)
    e1.record(stream)
    barrier()
    ctx.sync()
    ms_sts = max_over_ranks(e0.elapsed_time(e1)) / n_sts
    st2.release()

    # --------------------------------------------------------------- e2e
    # state held on the host (pinned): every step copies x, v in, runs one
    # outer step through the public API and reads x, v and the energy back
    d3 = core.DeviceSystem(W["system"]())
    st3 = core.MDState(d3, v0, m_hmr.astype(np.float32), seeds=I.seed, replica_ids=[D.replica_id(rank, 0)])
    hx = torch.from_numpy(sy.x.astype(np.float32)).pin_memory()
    hv = torch.from_numpy(v0.astype(np.float32)).pin_memory()
    he = torch.zeros(1, dtype=torch.float64).pin_memory()
    core.respa_step(ctx, st3, integ, 2)
    ctx.sync()
    n_e2e = max(5, args.steps // 4)
    barrier()
    t0 = time.perf_counter()
    e0.record(stream)
    for _ in range(n_e2e):
        d3.x.copy_(hx, non_blocking=True)
        st3.v.copy_(hv, non_blocking=True)
        core.respa_step(ctx, st3, integ, 1)
        hx.copy_(d3.x, non_blocking=True)
        hv.copy_(st3.v, non_blocking=True)
        he.copy_(st3.energy[:1], non_blocking=True)
    e1.record(stream)
    barrier()
    ctx.sync()
    ms_e2e = max_over_ranks(e0.elapsed_time(e1)) / n_e2e
    st3.release()
    bytes_in = 2 * sy.n_atoms * 12
    bytes_out = 2 * sy.n_atoms * 12 + 8

    # ------------------------------------------------ 100,000-atom box
    # the largest synthetic system: same models, the integrator and list
    # kernels at a size where they stream enough bytes to be HBM-bound
    WL = S.WORKLOADS[LARGE_WORKLOAD]
    syL = WL["system"]()
    csL, nsL = WL["cons"](), WL["nc"]()
    ctxL = core.Context(cons=(csL, S.cons_weights(csL, WL["w_seed"])), nc=(nsL, S.nc_weights(nsL, WL["w_seed"])),
                        device=local)
    IL = WL["dmts"]
    mL = core.masses_hmr(syL.species, syL.mol_id, syL.element_masses(), IL.hmr_delta)
    dL = core.DeviceSystem(syL)
    stL = core.MDState(dL, S.maxwell_boltzmann(mL, IL.temperature, WL["rng_seed"]), mL.astype(np.float32),
                       seeds=IL.seed, replica_ids=[D.replica_id(rank, 0)])
    integL = core.integrator(IL.dt_outer, IL.n_inner, IL.temperature, IL.gamma_ps, skin=skin)
    n_large = max(5, min(20, args.steps // 10))
    core.respa_step(ctxL, stL, integL, 3)
    ctxL.sync()
    core.profile_enable(ctxL, True)
    barrier()
    e0.record(stream)
    core.respa_step(ctxL, stL, integL, n_large)
    e1.record(stream)
    barrier()
    ctxL.sync()
    profL = core.profile_read(ctxL)
    core.profile_enable(ctxL, False)
    ms_large = max_over_ranks(e0.elapsed_time(e1)) / n_large
    stL.release()
    stsL = WL["sts"]
    mLe = syL.element_masses()
    dL2 = core.DeviceSystem(syL)
    stL2 = core.MDState(dL2, S.maxwell_boltzmann(mLe, stsL.temperature, WL["rng_seed"]), mLe.astype(np.float32),
                        seeds=stsL.seed, replica_ids=[D.replica_id(rank, 0)])
    integL2 = core.integrator(stsL.dt_outer, 1, stsL.temperature, stsL.gamma_ps, mode=1, skin=skin)
    core.respa_step(ctxL, stL2, integL2, 3)
    ctxL.sync()
    barrier()
    e0.record(stream)
    core.respa_step(ctxL, stL2, integL2, 2 * n_large)
    e1.record(stream)
    barrier()
    ctxL.sync()
    ms_large_sts = max_over_ranks(e0.elapsed_time(e1)) / (2 * n_large)
    stL2.release()
    del ctxL

    # ----------------------------------------------------------- serving
    # (1) the 23,558-atom system as a request of the serving loop
    r3 = core.ReplicaRequest(sy, v0, m_hmr, args.steps, I.seed, D.replica_id(rank, 0))
    out3, st3s = core.run_replicas(ctx, [r3], integ)
    ms_serve = float(np.sum(st3s["tick_ms"])) / max(1, st3s["n_ticks"])
    # (2) the replica-serving workload: Poisson arrivals of small solvated
    # molecules, continuous batching, per-tick latency
    n_req = int(os.environ.get("DMTS_BENCH_REQUESTS", "512"))
    spec = S.serving_requests(n_req=n_req, seed=401)
    reqs = []
    for q in spec:
        sq = S.capped_molecule_in_droplet(q["n_solute"], seed=q["sys_seed"])
        mq = core.masses_hmr(sq.species, sq.mol_id, sq.element_masses(), I.hmr_delta)
        vq = S.maxwell_boltzmann(mq, I.temperature, q["sys_seed"] + 1)
        reqs.append(core.ReplicaRequest(sq, vq, mq, q["n_outer"], q["rng_seed"], D.replica_id(rank, 1 + q["id"]),
                                        q["arrival_s"]))
    barrier()
    core.profile_enable(ctx, True)
    outs, sst = core.run_replicas(ctx, reqs, integ, realtime=True)
    prof_serve = core.profile_read(ctx)
    core.profile_enable(ctx, False)
    barrier()
    tk = sst["tick_ms"]
    lat = np.array([o["t_done_s"] - o["t_arrival_s"] for o in outs])
    serving = {
        "workload": f"{n_req} Poisson requests (200/s), 80-1600 atoms each, 50-2000 outer steps, open droplets",
        "p50_ms_per_outer_step": float(np.percentile(tk, 50)), "p99_ms_per_outer_step": float(np.percentile(tk, 99)),
        "ticks": int(sst["n_ticks"]), "wall_s": sst["wall_s"], "max_resident": int(sst["max_resident"]),
        "atom_outer_steps_per_s": sst["atom_outer_steps"] / sst["wall_s"] * world,
        "request_latency_s_p50": float(np.percentile(lat, 50)), "request_latency_s_p99": float(np.percentile(lat, 99)),
        "failed": int(sum(o["status"] != 0 for o in outs)),
        "kernel_roofline": serving_roofline(prof_serve, sst["atom_outer_steps"], I.n_inner, cs),
        "solvated_chain_23558_in_loop": {"ns_per_day": ns_per_day(I.dt_outer, 1e3 / ms_serve) * world,
                                         "ms_per_outer_step": ms_serve,
                                         "vs_sts": ns_per_day(I.dt_outer, 1e3 / ms_serve) / ns_per_day(sts.dt_outer, 1e3 / ms_sts)},
    }

    # ---------------------------------------------------------- roofline
    peaks = {}
    pk_path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(pk_path):
        peaks = json.load(open(pk_path))
    C = cs.C
    # algorithmic FLOP per active edge (one layer), counted as 2 per FMA:
    # forward: radial 3*8 FMA + 3 mul + 9 FMA per channel;
    # adjoint: radial and derivative 48 FMA + 18 + 9 + 3 + 9 + 9 + 3 per
    # channel, plus 30 FMA per lane for the direction derivatives; layer 0
    # has no sender-role gradient (its inputs are the species embedding), so
    # 87 FMA per channel there. mp_bwd is the average over the L launches of
    # one evaluation, as the per-launch time is.
    Lc = cs.L
    flop_edge = {"mp_fwd": 2 * 36 * C,
                 "mp_bwd": (2 * 99 * C * (Lc - 1) + 2 * 87 * C) / Lc + 2 * 30 * 32}
    fp32_peak_tflops = 152 * 128 * 2 * 2.070e9 / 1e12   # SMs x FP32 lanes x FMA x max clock
    fp32_src = "152 SMs x 128 FP32 lanes x 2 FLOP x 2.07 GHz (nominal unit counts and max clock)"

    def per_launch_s(pr, k):
        v = pr.get(k)
        return v[1] / v[0] * 1e-3 if v and v[0] else None

    ranked = sorted(((k, v) for k, v in prof.items() if k in flop_edge), key=lambda kv: -kv[1][1])
    name = ranked[0][0] if ranked else "mp_bwd"
    pl = per_launch_s(prof, name)
    achieved = flop_edge[name] * e_cons / pl / 1e12 if pl else None
    roof = {"kernel": name, "bound": "alu", "achieved": achieved, "peak": fp32_peak_tflops,
            "unit": "TFLOP/s", "frac": achieved / fp32_peak_tflops if achieved else None,
            "traffic": ncu_traffic(name), "peak_source": fp32_src,
            "work_per_launch": f"{flop_edge[name]} FLOP x {e_cons} active edges",
            "algorithmic_bytes_per_launch": None}
    # node arrays once (fp32 unless noted) and the active-edge stream (4 B of
    # column index per active entry): forward reads s, x and writes A, q
    # (+ its bf16 copy); the adjoint reads s, gA, g_s and x and writes g_s
    # (+ bf16 copy) and F
    nlm = (cs.lmax + 1) ** 2
    n_at = sy.n_atoms
    alg_bytes = {"mp_fwd": n_at * (4 * C + 12 + 4 * nlm * C + 6 * (cs.lmax + 1) * C) + 4 * e_cons,
                 "mp_bwd": n_at * (4 * C + 4 * nlm * C + 12 + 12 + (Lc - 1) / Lc * (4 * C + 6 * C)) + 4 * e_cons}
    roof["algorithmic_bytes_per_launch"] = alg_bytes[name]

    # every hot kernel against its own bound (per-launch averages over the
    # timed region; algorithmic work counts each node array once and each
    # edge stream once)
    hbm = peaks.get("hbm_gbs")
    bf16_pk = peaks.get("bf16_tflops_sustained")
    N, NL = sy.n_atoms, cs.lmax + 1
    gemm_flop_cons = 2.0 * N * C * C * (2 * cs.L * (NL + 1) + 2)
    Cn, qkw = ns.C, 2 * (ns.K + ns.n_l) * ns.n_c
    gemm_flop_nc = 2.0 * N * Cn * (2 * Cn + Cn + qkw)

    def rate(work, seconds, unit_scale):
        return work / seconds / unit_scale if seconds else None

    t_gemm = prof.get("gemm_tc", (0, 0.0))[1] * 1e-3 / n_prof
    t_ncg = prof.get("nc_gemm_tc", (0, 0.0))[1] * 1e-3 / n_prof
    nc_bytes = N * (qkw * 4 + ns.n_l * 12 + 12 + 12) + 4 * e_nc
    kr = {}
    for k in ("mp_fwd", "mp_bwd"):
        a = rate(flop_edge[k] * e_cons, per_launch_s(prof, k), 1e12)
        kr[k] = {"row": "a2+a3" if k == "mp_fwd" else "a5", "bound": "alu", "tflops": a,
                 "frac_fp32_peak": a / fp32_peak_tflops if a else None}
    g = rate(gemm_flop_cons, t_gemm, 1e12)
    kr["gemm_tc"] = {"row": "a4", "bound": "tensor", "tflops": g, "frac_bf16_sustained": g / bf16_pk if g and bf16_pk else None,
                     "flop_per_step": gemm_flop_cons}
    g = rate(gemm_flop_nc * I.n_inner, t_ncg, 1e12)
    kr["nc_gemm_tc"] = {"row": "a4 (NC)", "bound": "tensor", "tflops": g,
                        "frac_bf16_sustained": g / bf16_pk if g and bf16_pk else None}
    # the NC layer's forward: radial K(l_max+1) FMA + (l_max+1) mul +
    # (l_max+1)^2 FMA per (edge, channel), as for the conservative layer
    nnl = ns.lmax + 1
    flop_nc_edge = 2 * (ns.K * nnl + nnl + nnl * nnl) * Cn
    a = rate(flop_nc_edge * e_nc, per_launch_s(prof, "nc_mp_fwd"), 1e12)
    kr["nc_mp_fwd"] = {"row": "a7 (NC layer: a2+a3 at NC sizes)", "bound": "alu", "tflops": a,
                       "frac_fp32_peak": a / fp32_peak_tflops if a else None, "flop_per_edge": flop_nc_edge}
    b = rate(nc_bytes, per_launch_s(prof, "nc_head"), 1e9)
    kr["nc_head"] = {"row": "a7", "bound": "hbm", "gbs": b, "frac_hbm": b / hbm if b and hbm else None,
                     "bytes_per_launch": nc_bytes}
    # average over the n_inner launches of an outer step (the one closing
    # launch of a long call is left out)
    ib = integ_bytes_per_outer_step(I.n_inner, False) / I.n_inner
    b = rate(ib * N, per_launch_s(prof, "integrate"), 1e9)
    kr["integrate"] = {"row": "a8", "bound": "hbm", "gbs": b, "frac_hbm": b / hbm if b and hbm else None,
                       "bytes_per_launch": ib * N}
    b = rate(ib * syL.n_atoms, per_launch_s(profL, "integrate"), 1e9)
    kr["integrate_100k"] = {"row": "a8", "bound": "hbm", "gbs": b, "frac_hbm": b / hbm if b and hbm else None,
                            "bytes_per_launch": ib * syL.n_atoms}
    shares = {k: {"launches": v[0], "ms_per_step": v[1] / n_prof,
                  "share": v[1] / max(sum(x[1] for x in prof.values()), 1e-9)} for k, v in prof.items()}

    val = ns_per_day(I.dt_outer, 1e3 / ms_dmts) * world
    sts_val = ns_per_day(sts.dt_outer, 1e3 / ms_sts) * world
    line = {
        "metric": "ns/day (DMTS-NC)", "value": val, "unit": "ns/day", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_dmts, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32+bf16" if cs.bf16 else "f32", "data": "synthetic",
        "config": workload_config(sy, I, cs, ns),
        "atom_steps_per_s": sy.n_atoms * 1e3 / ms_dmts * world,
        "sts": {"ns_per_day": sts_val, "ms_per_step": ms_sts, "dt_fs": sts.dt_outer,
                "atom_steps_per_s": sy.n_atoms * 1e3 / ms_sts * world},
        "speedup_vs_sts": val / sts_val,
        "e2e": {"value": ns_per_day(I.dt_outer, 1e3 / ms_e2e) * world, "unit": "ns/day",
                "h2d_bytes_per_step": bytes_in, "d2h_bytes_per_step": bytes_out, "steps": n_e2e},
        "serving": serving,
        "gpu_launches": n_launches,
        "clocks": ck,
        "roofline": roof,
        "kernels": shares,
        "kernel_roofline": kr,
        "rewind_guard": side["guarded"],
        "ffl": side["ffl"],
        "npt": side["npt"],
        "distill": side["distill"],
        "large_system": {"workload": syL.name, "n_atoms": syL.n_atoms, "steps": n_large,
                         "ns_per_day": ns_per_day(IL.dt_outer, 1e3 / ms_large) * world, "ms_per_step": ms_large,
                         "sts_ns_per_day": ns_per_day(stsL.dt_outer, 1e3 / ms_large_sts) * world,
                         "sts_ms_per_step": ms_large_sts,
                         "speedup_vs_sts": ns_per_day(IL.dt_outer, 1e3 / ms_large) / ns_per_day(stsL.dt_outer, 1e3 / ms_large_sts),
                         "kernels_ms_per_step": {k: v[1] / n_large for k, v in profL.items()}},
        "active_edges": {"cons": e_cons, "nc": e_nc},
    }
    if rank == 0 and not args.no_cpu and world == 1:
        t_outer, desc = oracle_outer_step_seconds(sy, W, 0.6)
        line["cpu_baseline"] = {"value": ns_per_day(I.dt_outer, 1.0 / t_outer), "unit": "ns/day",
                                "cores": 1, "kind": "oracle", "sample": desc}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
