"""Benchmark of the DMTS-NC hot path on one GB300 (or N, one replica each).

One step = one outer step of Algorithm 1 (one conservative evaluation with
its adjoint forces, n = 5 NC evaluations, the fused integrator, neighbour
rebuilds) on the 23,558-atom solvated bead chain in water. The same GPU also
runs single-time-step BAOAB (1 fs, no HMR) for the ns/day ratio.

Prints one JSON line (rank 0), the headline first; `--detail PATH` also
writes every leg's figures (per-kernel shares and rooflines, the other
configurations, serving latencies, rewind guard, FFL, NPT, distillation) to
a JSON file. `--impl reference` times the FP64 CPU oracle instead, on
periodic samples of the same workload.
"""
from __future__ import annotations

import argparse
import dataclasses
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
    "mp_bwd": {"bytes_per_launch": (154229760 + 19248896 + 154260992 + 16390400 + 139650304 + 268544) / 3,
               # the adjoint's code: channel-pack helpers, kernel and launch, the
               # argument structs, the device helpers
               "sources": [("paper_2602_14975_gb300/csrc/mp.cu", ("// ---- channel packs", "// ---- forward")),
                           ("paper_2602_14975_gb300/csrc/mp.cu", ("// ---- adjoint", "// In the forward pass")),
                           ("paper_2602_14975_gb300/csrc/mp.cu", ("template <int C, int LMAX, bool VIR, bool SG>",
                                                                  "#define DMTS_DISPATCH")),
                           ("paper_2602_14975_gb300/csrc/mp.cuh", ("struct EdgeGeom {", "template <int CPW>")),
                           ("paper_2602_14975_gb300/csrc/common.cuh", None)],
               "sha256": "8c1a3a7c5d60e748369169f7e9198032650ff7e2427e60f09026a2b70bc7c32c"},
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
    ap.add_argument("--detail", default="", help="also write every leg's figures to this JSON file")
    ap.add_argument("--next3", action="store_true",
                    help="the distillation study on the 12,288-atom water box instead (NEXT-3): held-out |F_L| "
                         "before and after, and DMTS-NC kinetic temperatures against (T/d) chi^2(d)")
    ap.add_argument("--main-only", action="store_true",
                    help="only the timed DMTS-NC leg (for profiler captures); prints its time and kernel shares")
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
def host_cpu():
    """(CPUs this process may run on, CPU model) of the host the oracle runs on."""
    n = usable_cpus()
    model = ""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            k, _, v = line.partition(":")
            if k.strip() == "Model name" and v.strip():
                model = v.strip()
                break
    except (OSError, subprocess.SubprocessError):
        pass
    if not model:
        try:
            for line in open("/proc/cpuinfo"):
                k, _, v = line.partition(":")
                if k.strip() == "model name":
                    model = v.strip()
                    break
        except OSError:
            pass
    import platform
    return n, model or platform.machine()


def cutout(sy, frac_edge):
    """A periodic sample of the system at its own density: the molecules
    whose first atom lies in [0, f L)^3 (wrapped), each kept whole next to
    that atom, in a periodic box of edge f L, so that every atom has about
    as many neighbours as in the full system (an open cut-out would lose
    those beyond its faces and look cheaper per atom). Chain beads inside
    the region are kept with the bonds between them."""
    from paper_2602_14975_gb300 import synth as S
    xw = np.mod(sy.x, sy.box)
    lim = frac_edge * sy.box
    first = {}
    for i in range(sy.n_atoms):
        first.setdefault(int(sy.mol_id[i]), i)
    keep = np.zeros(sy.n_atoms, bool)
    xk = np.array(sy.x, np.float64)
    chain = set(int(m) for m, c in zip(*np.unique(sy.mol_id, return_counts=True)) if c > 3)
    for i in range(sy.n_atoms):
        m = int(sy.mol_id[i])
        if m in chain:
            keep[i] = bool(np.all(xw[i] < lim))
            xk[i] = xw[i]
        else:
            f = first[m]
            if np.all(xw[f] < lim):
                keep[i] = True
                d = sy.x[i] - sy.x[f]
                xk[i] = xw[f] + d - sy.box * np.rint(d / sy.box)
    idx = np.nonzero(keep)[0]
    remap = -np.ones(sy.n_atoms, np.int64)
    remap[idx] = np.arange(idx.size)
    b = sy.bonds
    bm = keep[b[:, 0]] & keep[b[:, 1]]
    return S.System(sy.name + "_cutout", xk[idx], sy.species[idx], sy.mol_id[idx],
                    remap[b[bm]].astype(np.int32), sy.bond_r0[bm], np.array(sy.box) * frac_edge)


def _oracle_sample_times(sub, cs, cb, ns, nb):
    """(seconds of one conservative E+F with the prior, of one NC
    evaluation) of the oracle on the system `sub`."""
    import oracle as O
    t0 = time.perf_counter()
    O.cons_energy_forces(sub, cs, cb)
    O.prior(sub)
    t1 = time.perf_counter()
    O.nc_forces(sub, ns, nb)
    t2 = time.perf_counter()
    return t1 - t0, t2 - t1


def _oracle_copy(job):
    """One copy of the all-cores leg (runs in a spawned process)."""
    return _oracle_sample_times(*job)


def usable_cpus():
    try:
        return len(os.sched_getaffinity(0))
    except (AttributeError, OSError):
        return os.cpu_count() or 1


def oracle_all_cores(sy, W, frac_edge):
    """The oracle, as it stands, as one copy per usable host core at once
    (spawned processes, each timing the same periodic sample): the sum of
    the copies' outer-step rates, scaled to the full system, is the host's
    aggregate throughput and an upper bound for any all-core parallel form
    of the oracle's force loops on one system (perfect scaling, measured
    under the same memory and cache contention)."""
    import multiprocessing as mp
    from paper_2602_14975_gb300 import synth as S
    sub = cutout(sy, frac_edge)
    cs, ns = W["cons"](), W["nc"]()
    job = (sub, cs, S.cons_weights(cs, W["w_seed"]), ns, S.nc_weights(ns, W["w_seed"]))
    n_in = W["dmts"].n_inner
    p = usable_cpus()
    t0 = time.perf_counter()
    with mp.get_context("spawn").Pool(p) as pool:
        times = pool.map(_oracle_copy, [job] * p)
    wall = time.perf_counter() - t0
    scale = sy.n_atoms / sub.n_atoms
    per_outer = [(tc + n_in * tn) * scale for tc, tn in times]
    rate = sum(1.0 / t for t in per_outer)           # full-system outer steps per second
    return rate, p, wall, (f"{p} concurrent copies of the oracle (FP64 C, as it stands, 1 thread each), each timing "
                           f"1 conservative E+F + 1 NC evaluation on a periodic {sub.n_atoms}-atom sample of "
                           f"{sy.name} scaled x{scale:.2f}; value = the sum of their outer-step rates")


def oracle_outer_step_seconds(sy, W, frac_edge):
    """Times the oracle's force evaluations of one DMTS-NC outer step (one
    conservative energy + forces with the prior, n NC evaluations) on a
    periodic sample; returns (seconds per outer step scaled to the full
    system, seconds the sample took, sample description)."""
    from paper_2602_14975_gb300 import synth as S
    sub = cutout(sy, frac_edge) if frac_edge < 1.0 else sy
    cs, ns = W["cons"](), W["nc"]()
    cb, nb = S.cons_weights(cs, W["w_seed"]), S.nc_weights(ns, W["w_seed"])
    n_in = W["dmts"].n_inner
    t_cons, t_nc = _oracle_sample_times(sub, cs, cb, ns, nb)
    per_outer = t_cons + n_in * t_nc
    scale = sy.n_atoms / sub.n_atoms
    what = (f"a periodic {sub.n_atoms}-atom sample ({frac_edge:.3f} of the box edge, same density) of {sy.name}, "
            f"scaled x{scale:.2f}") if sub is not sy else f"the whole {sy.name}"
    desc = (f"oracle (FP64 C, as it stands, 1 thread): 1 conservative E+F + 1 NC evaluation timed on {what}; "
            f"outer step = t_cons + {n_in} t_nc")
    return per_outer * scale, t_cons + t_nc, desc


def workload_config(sy, I, cs, ns):
    """The `config` of the JSON line (the same for both arms)."""
    return {"workload": sy.name, "n_atoms": sy.n_atoms,
            "integrator": f"DMTS-NC outer {I.dt_outer} fs / {I.n_inner} inner, HMR +{I.hmr_delta} Da on H "
                          f"(the paper's HMR; the configurations' 'H mass 3 amu' read as this), "
                          f"gamma_H {I.gamma_ps[0]}/ps, gamma_heavy {I.gamma_ps[1]}/ps",
            "cons_model": f"L={cs.L} C={cs.C} lmax={cs.lmax} K={cs.K} rc={cs.rc}",
            "nc_model": f"C={ns.C} lmax=1 rc={ns.rc} n_c={ns.n_c} n_l={ns.n_l}",
            "precision": ("split-bf16 MLP contractions on the tensor cores (tcgen05, fp32 accumulate), "
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


def serving_tail(tick_ms, tick_atoms):
    """What sets the per-tick latency percentiles: a least-squares fit
    ms = a + b * atoms over all ticks, and the batch sizes of the p50 and p99
    ticks (a tick's cost follows the atoms resident in it)."""
    t = np.asarray(tick_ms, np.float64)
    n = np.asarray(tick_atoms, np.float64)
    if t.size < 2 or np.ptp(n) == 0:
        return None
    b, a = np.polyfit(n, t, 1)
    resid = t - (a + b * n)
    p50, p99 = np.percentile(t, 50), np.percentile(t, 99)
    near = lambda p: float(np.median(n[np.abs(t - p) <= 0.05 * p])) if np.any(np.abs(t - p) <= 0.05 * p) else None  # noqa: E731
    return {"fit_ms": {"intercept": float(a), "per_1000_atoms": float(b * 1e3)},
            "fit_residual_ms_p99_abs": float(np.percentile(np.abs(resid), 99)),
            "atoms_at_p50_tick": near(p50), "atoms_at_p99_tick": near(p99),
            "atoms_p50": float(np.percentile(n, 50)), "atoms_max": float(n.max())}


# ----------------------------------------------------------------- NEXT-3 --
def next3_study(core, S, D, rank):
    """Distillation of the NC model (Sec. 2, "Model training") on frames of a
    single-time-step run of the 12,288-atom water box with the conservative
    model (20 training frames and 4 held out, 50 fs apart), 2,000 Adam steps
    on all frames at once with a cosine learning rate from 2e-3; then
    DMTS-NC at Delta = 10 fs with the distilled model for n = 5, 10, 20 inner
    steps: kinetic temperatures every 0.5 ps after 5 ps against
    (T/d) chi^2(d), d = 3N (Sec. 3), and the largest |F - F_S| the rewind
    guard sees with the random and the distilled NC model."""
    from scipy import stats
    import torch
    W = S.WORKLOADS["water_12288"]
    sy = W["system"]()
    cs, ns = W["cons"](), W["nc"]()
    cb, nb = S.cons_weights(cs, W["w_seed"]), S.nc_weights(ns, W["w_seed"])
    ctx = core.Context(cons=(cs, cb), nc=(ns, nb))
    ctx0 = core.Context(cons=(cs, cb), nc=(ns, nb))
    I = W["dmts"]
    m_el = sy.element_masses()
    d = core.DeviceSystem(sy)
    st = core.MDState(d, S.maxwell_boltzmann(m_el, 300.0, 7), m_el.astype(np.float32), seeds=11)
    ig = core.integrator(1.0, 1, 300.0, (1.0,) * 5, mode=core.L.MODE_STS, skin=0.5)
    core.respa_step(ctx, st, ig, 200)
    frames = []
    for _ in range(24):
        core.respa_step(ctx, st, ig, 50)
        frames.append(d.x.cpu().numpy().astype(np.float64))
    st.release()

    def batch(xs):
        db = core.DeviceSystem([S.System(sy.name, x, sy.species, sy.mol_id, sy.bonds, sy.bond_r0, sy.box)
                                for x in xs])
        _, T = core.energy_forces_cons(ctx, db, core.nbr_build(ctx, db, cs.rc + 0.5), with_prior=True)
        return db, core.nbr_build(ctx, db, ns.rc + 0.5), T

    train, hold = batch(frames[:20]), batch(frames[20:])

    def rms(b):
        loss, _ = core.nc_distill_step(ctx, b[0], b[1], b[2], lr=0.0)
        return math.sqrt(loss.sum().item() / (3 * b[0].n_atoms))

    r0 = (rms(train), rms(hold))
    n_steps = 2000
    t0 = time.perf_counter()
    for k in range(n_steps):
        lr = 2e-3 * 0.5 * (1.0 + math.cos(math.pi * k / n_steps))
        core.nc_distill_step(ctx, train[0], train[1], train[2], lr=lr, step=k + 1)
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0
    r1 = (rms(train), rms(hold))
    m = core.masses_hmr(sy.species, sy.mol_id, sy.element_masses(), I.hmr_delta)
    dof = 3 * sy.n_atoms
    runs = []
    for n_in in (5, 10, 20):
        dd = core.DeviceSystem(sy)
        s2 = core.MDState(dd, S.maxwell_boltzmann(m, 300.0, 9), m.astype(np.float32), seeds=13, thermo=True)
        ii = core.integrator(I.dt_outer, n_in, I.temperature, I.gamma_ps, skin=0.5)
        Ts = []
        for _ in range(60):
            core.respa_step(ctx, s2, ii, 50)
            Ts.append(float(s2.thermo.cpu().numpy()[0, 2]))
        s2.release()
        T = np.array(Ts[10:])
        runs.append({"n_inner": n_in, "delta_fs": I.dt_outer / n_in, "T_mean": float(T.mean()),
                     "T_std": float(T.std()), "T_std_chi2": 300.0 * math.sqrt(2.0 / dof), "samples": int(T.size),
                     "ks_p": float(stats.kstest(T * dof / 300.0, stats.chi2(dof).cdf).pvalue)})
    guard = {}
    for label, cx in (("random", ctx0), ("distilled", ctx)):
        dg = core.DeviceSystem(sy)
        sg = core.MDState(dg, S.maxwell_boltzmann(m, 300.0, 9), m.astype(np.float32), seeds=13)
        gs = core.respa_guarded(cx, sg, core.integrator(I.dt_outer, I.n_inner, I.temperature, I.gamma_ps, skin=0.5),
                                200, math.inf, 50, 4 * I.n_inner, I.dt_outer / I.n_inner)
        guard[label] = float(np.max(gs["chunk_max"]))
        sg.release()
    return {"study": "NEXT-3 distillation", "workload": sy.name, "train_frames": 20, "held_out_frames": 4,
            "adam_steps": n_steps, "train_s": t_train, "f_l_rms_train": [r0[0], r1[0]],
            "f_l_rms_held_out": [r0[1], r1[1]], "unit": "kcal/mol/A", "temperatures": runs,
            "max_force_disagreement_200_outer_steps": guard}


# ------------------------------------------------------------------ main --
def reference_arm(args, W, I):
    """The FP64 oracle, as it stands, on the host cores: every step times one
    outer step's force evaluations on a periodic sample of the workload sized
    so that warm-up and timed steps take about two minutes together."""
    sy = W["system"]()
    t_full, t_cal, _ = oracle_outer_step_seconds(sy, W, 0.25)
    budget = 120.0 / max(1, args.steps + args.warmup)
    frac = min(0.6, 0.25 * (budget / max(t_cal, 1e-3)) ** (1.0 / 3.0))
    frac = max(frac, 0.2)
    for _ in range(args.warmup):
        oracle_outer_step_seconds(sy, W, frac)
    t0 = time.perf_counter()
    per, wall_each = [], []
    for _ in range(args.steps):
        s_full, s_sample, desc = oracle_outer_step_seconds(sy, W, frac)
        per.append(s_full)
        wall_each.append(s_sample)
    wall = time.perf_counter() - t0
    t_outer = float(np.mean(per))
    val = ns_per_day(I.dt_outer, 1.0 / t_outer)
    ncpu, model = host_cpu()
    return {"impl": "reference", "metric": "ns/day (DMTS-NC)", "value": val, "unit": "ns/day",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": float(np.mean(wall_each)) * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": workload_config(sy, I, W["cons"](), W["nc"]()),
            "cpu_baseline": {"value": val, "unit": "ns/day", "cores": 1, "kind": "oracle", "sample": desc,
                             "host_cpus": ncpu, "cpu_model": model,
                             "full_system_s_per_outer_step": t_outer},
            "e2e": {"value": val, "unit": "ns/day", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "wall_s": wall}


def fp32_peak_tflops(props, peaks):
    """FP32 FMA peak: SMs (from the device) x 128 FP32 lanes per SM x 2 FLOP
    x the maximum SM clock (the measured-peaks file, else nvidia-smi)."""
    mhz = peaks.get("sm_max_mhz")
    src = "measured-peaks file"
    if not mhz:
        try:
            out = subprocess.run(["nvidia-smi", "--query-gpu=clocks.max.sm", "--format=csv,noheader,nounits"],
                                 capture_output=True, text=True, timeout=20).stdout.split()
            mhz, src = float(out[0]), "nvidia-smi"
        except (OSError, subprocess.SubprocessError, ValueError, IndexError):
            mhz, src = 2070.0, "nominal"
    sms = props.multi_processor_count
    return sms * 128 * 2 * mhz * 1e6 / 1e12, f"{sms} SMs x 128 FP32 lanes x 2 FLOP x {mhz:.0f} MHz ({src} clock)"


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
        print(json.dumps(reference_arm(args, W, I)), flush=True)
        return 0

    import torch
    torch.cuda.set_device(local)
    D.init("nccl", torch.device(f"cuda:{local}"))
    from paper_2602_14975_gb300 import core

    if args.next3:
        out = next3_study(core, S, D, rank)
        if rank == 0:
            print(json.dumps(out), flush=True)
        return 0
    dev = torch.device(f"cuda:{local}")
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    skin = 0.5    # Verlet skin (A); rebuilds are gated on half-skin displacement

    def barrier():
        D.barrier(dev)

    def max_over_ranks(v):
        return D.max_over_ranks(v, dev)

    def timed(ctx_, st_, integ_, n):
        """ms per step of n steps through respa_step (max over ranks)."""
        barrier()
        e0.record(stream)
        core.respa_step(ctx_, st_, integ_, n)
        e1.record(stream)
        barrier()
        ctx_.sync()
        return max_over_ranks(e0.elapsed_time(e1)) / n

    def integ_of(spec, **kw):
        return core.integrator(spec.dt_outer, spec.n_inner, spec.temperature, spec.gamma_ps, skin=skin, **kw)

    def run_leg(ctx_, sy_, spec, v_seed, n, warm=3, sts=False):
        """ms per step of `n` steps of one system (HMR masses per `spec`)."""
        m_ = (core.masses_hmr(sy_.species, sy_.mol_id, sy_.element_masses(), spec.hmr_delta)
              if spec.hmr_delta else sy_.element_masses())
        d_ = core.DeviceSystem(sy_)
        st_ = core.MDState(d_, S.maxwell_boltzmann(m_, spec.temperature, v_seed), m_.astype(np.float32),
                           seeds=spec.seed, replica_ids=[D.replica_id(rank, 0)])
        ig = integ_of(spec, mode=core.L.MODE_STS if sts else core.L.MODE_RESPA)
        core.respa_step(ctx_, st_, ig, warm)
        ctx_.sync()
        ms = timed(ctx_, st_, ig, n)
        st_.release()
        return ms

    sy = W["system"]()
    cs, ns = W["cons"](), W["nc"]()    # split-bf16 MLP contractions on the tensor cores
    cb, nb = S.cons_weights(cs, W["w_seed"]), S.nc_weights(ns, W["w_seed"])
    ctx = core.Context(cons=(cs, cb), nc=(ns, nb), device=local)
    cs32 = dataclasses.replace(cs, bf16=False)
    ctx32 = core.Context(cons=(cs32, cb), device=local)     # plain FP32 single-time-step baseline

    # algorithmic work of the dominant kernels (active edges within the cutoffs)
    d0 = core.DeviceSystem(sy)
    e_cons = core.nbr_build(ctx, d0, cs.rc).n_pairs
    e_nc = core.nbr_build(ctx, d0, ns.rc).n_pairs
    del d0

    # ---------------------------------------------------------- DMTS-NC
    m_hmr = core.masses_hmr(sy.species, sy.mol_id, sy.element_masses(), I.hmr_delta)
    v0 = S.maxwell_boltzmann(m_hmr, I.temperature, W["rng_seed"])
    dsys = core.DeviceSystem(sy)
    st = core.MDState(dsys, v0, m_hmr.astype(np.float32), seeds=I.seed, replica_ids=[D.replica_id(rank, 0)],
                      thermo=True)
    integ = integ_of(I)
    core.respa_step(ctx, st, integ, args.warmup)
    ctx.sync()
    clocks = ClockSampler(local)
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
    ms_dmts = max_over_ranks(e0.elapsed_time(e1)) / args.steps
    # per-kernel CUDA events on every PROF_EVERY-th outer step of a second
    # run of the same length (those steps run without the graph replay)
    core.profile_enable(ctx, True, every=PROF_EVERY)
    n_prof = (args.steps + PROF_EVERY - 1) // PROF_EVERY
    core.respa_step(ctx, st, integ, args.steps)
    ctx.sync()
    prof = core.profile_read(ctx)
    core.profile_enable(ctx, False)
    thermo_end = st.thermo.cpu().numpy()[0].tolist()
    st.release()
    if args.main_only:
        if rank == 0:
            print(json.dumps({"workload": sy.name, "ms_per_step": ms_dmts,
                              "ns_per_day": ns_per_day(I.dt_outer, 1e3 / ms_dmts) * world, "gpu_launches": n_launches,
                              "kernels_ms_per_step": {k: v[1] / n_prof for k, v in prof.items()}}), flush=True)
        return 0

    # ------------------------------------- rewind guard, FFL thermostat
    # the same outer step under the rewind guard (saved frame and monitor
    # read every 50 outer steps, no disagreement), and with the Fast Forward
    # Langevin O-step
    n_side = max(10, args.steps // 2)
    side = {}
    for label, th in (("guarded", 0), ("ffl", 1)):
        dg = core.DeviceSystem(W["system"]())
        sg = core.MDState(dg, v0, m_hmr.astype(np.float32), seeds=I.seed, replica_ids=[D.replica_id(rank, 0)])
        ig = integ_of(I, thermostat=core.L.FFL if th else core.L.LANGEVIN)
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
    core.respa_step(ctx, sn, integ_of(I, barostat=True), 0)   # lists (with the piston's cell margin), forces
    ctx.sync()
    k_start = 0.5 * float((m_hmr[:, None] * v0 ** 2).sum()) / 4.184e-4
    p_start = (2 * k_start - float(sn.virial_cons[0].item())) / (3 * float(np.prod(sy.box))) / KCAL_A3_PER_ATM
    i_npt = integ_of(I, barostat=True, pressure_atm=p_start, tau_p_ps=2.0)
    core.respa_step(ctx, sn, i_npt, 2)
    ctx.sync()
    ms = timed(ctx, sn, i_npt, n_side)
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
    # single-time-step BAOAB at 1 fs, no HMR: with plain FP32 models (the
    # baseline the target is stated against) and with the same split-bf16
    # contractions as DMTS-NC (to separate precision from multiple time steps)
    sts = W["sts"]
    n_sts = max(10, args.steps // 2)
    ms_sts = run_leg(ctx32, W["system"](), sts, W["rng_seed"], n_sts, warm=args.warmup, sts=True)
    ms_sts_bf = run_leg(ctx, W["system"](), sts, W["rng_seed"], n_sts, warm=3, sts=True)

    # --------------------------------------------------------------- e2e
    # state held on the host (pinned): every step copies x, v in, runs one
    # outer step through the public API and reads x, v and the energy back
    d3 = core.DeviceSystem(W["system"]())
    st3 = core.MDState(d3, v0, m_hmr.astype(np.float32), seeds=I.seed, replica_ids=[D.replica_id(rank, 0)])
    hx = torch.from_numpy(sy.x.astype(np.float32)).pin_memory()
    hv = torch.from_numpy(v0.astype(np.float32)).pin_memory()
    he = torch.zeros(1, dtype=torch.float64).pin_memory()
    for _ in range(3):   # warm-up calls of one outer step, as timed (the first captures the call's graph)
        core.respa_step(ctx, st3, integ, 1)
    ctx.sync()
    n_e2e = max(5, args.steps // 4)
    barrier()
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

    # ---------------------------------- the other configurations (1, 2, 5)
    # each: DMTS-NC with its own models and the single-time-step baseline in
    # plain FP32; the 100,000-atom box also with FP32 DMTS-NC and bf16 STS
    others = {}
    for name in ("water_192", "water_12288", LARGE_WORKLOAD):
        Wo = S.WORKLOADS[name]
        syo = Wo["system"]()
        cso, nso = Wo["cons"](), Wo["nc"]()
        cbo, nbo = S.cons_weights(cso, Wo["w_seed"]), S.nc_weights(nso, Wo["w_seed"])
        ctxo = core.Context(cons=(cso, cbo), nc=(nso, nbo), device=local)
        ctxo32 = core.Context(cons=(dataclasses.replace(cso, bf16=False), cbo),
                              nc=(dataclasses.replace(nso, bf16=False), nbo), device=local)
        n_o = max(5, min(50, args.steps // 4)) if syo.n_atoms > 50000 else max(10, args.steps // 2)
        big = name == LARGE_WORKLOAD
        if big:
            core.profile_enable(ctxo, True)
        ms_d = run_leg(ctxo, syo, Wo["dmts"], Wo["rng_seed"], n_o)
        prof_o = core.profile_read(ctxo) if big else None
        if big:
            core.profile_enable(ctxo, False)
        ms_s = run_leg(ctxo32, syo, Wo["sts"], Wo["rng_seed"], 2 * n_o, sts=True)
        rec = {"n_atoms": syo.n_atoms, "precision": "split-bf16" if cso.bf16 else "fp32",
               "ns_per_day": ns_per_day(Wo["dmts"].dt_outer, 1e3 / ms_d) * world, "ms_per_step": ms_d,
               "sts_fp32_ns_per_day": ns_per_day(Wo["sts"].dt_outer, 1e3 / ms_s) * world,
               "sts_fp32_ms_per_step": ms_s, "steps": n_o}
        rec["speedup_vs_sts"] = rec["ns_per_day"] / rec["sts_fp32_ns_per_day"]
        if cso.bf16:
            ms_d32 = run_leg(ctxo32, syo, Wo["dmts"], Wo["rng_seed"], n_o)
            ms_sbf = run_leg(ctxo, syo, Wo["sts"], Wo["rng_seed"], 2 * n_o, sts=True)
            rec["fp32_ns_per_day"] = ns_per_day(Wo["dmts"].dt_outer, 1e3 / ms_d32) * world
            rec["sts_bf16_ns_per_day"] = ns_per_day(Wo["sts"].dt_outer, 1e3 / ms_sbf) * world
        if big:
            rec["kernels_ms_per_step"] = {k: v[1] / n_o for k, v in prof_o.items()}
            prof_large, n_large, n_at_large = prof_o, n_o, syo.n_atoms
        others[name] = rec
        del ctxo, ctxo32

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
    ms_sts_ns = ns_per_day(sts.dt_outer, 1e3 / ms_sts)
    serving = {
        "workload": f"{n_req} Poisson requests (200/s), 80-1600 atoms each, 50-2000 outer steps, open droplets",
        "p50_ms_per_outer_step": float(np.percentile(tk, 50)), "p99_ms_per_outer_step": float(np.percentile(tk, 99)),
        "ticks": int(sst["n_ticks"]), "wall_s": sst["wall_s"], "max_resident": int(sst["max_resident"]),
        "atom_outer_steps_per_s": sst["atom_outer_steps"] / sst["wall_s"] * world,
        "request_latency_s_p50": float(np.percentile(lat, 50)), "request_latency_s_p99": float(np.percentile(lat, 99)),
        "failed": int(sum(o["status"] != 0 for o in outs)),
        "kernel_roofline": serving_roofline(prof_serve, sst["atom_outer_steps"], I.n_inner, cs),
        "tick_ms_all": [round(float(t), 4) for t in tk],
        "tick_atoms_all": [int(a) for a in sst["tick_atoms"]],
        "tail": serving_tail(tk, sst["tick_atoms"]),
        "solvated_chain_23558_in_loop": {"ns_per_day": ns_per_day(I.dt_outer, 1e3 / ms_serve) * world,
                                         "ms_per_outer_step": ms_serve,
                                         "vs_sts": ns_per_day(I.dt_outer, 1e3 / ms_serve) / ms_sts_ns},
    }

    # ---------------------------------------------------------- roofline
    peaks = {}
    pk_path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(pk_path):
        peaks = json.load(open(pk_path))
    fp32_pk, fp32_src = fp32_peak_tflops(torch.cuda.get_device_properties(local), peaks)
    C = cs.C
    Lc = cs.L
    nl1 = cs.lmax + 1
    nlm = nl1 * nl1
    # the method's work per active edge and layer (each FMA 2 FLOP): the
    # radial contraction R_lc = sum_k W B_k (K (l_max+1) FMA per channel) and
    # the message into A_lm (one FMA per (l, m) and channel); the adjoint
    # with per-layer recomputation counts twice the forward
    flop_method = {"mp_fwd": 2 * (cs.K * nl1 + nlm) * C}
    flop_method["mp_bwd"] = 2 * flop_method["mp_fwd"]
    # what the kernels execute per active edge (each FMA 2 FLOP): forward
    # 36 FMA per channel; the adjoint forms each pair once, from its lower
    # atom: 99 FMA per channel (87 in layer 0, which has no sender-role
    # gradient), 30 per lane for the direction derivatives and 93 adds for
    # the lanes' sum of the pair force, and the lower atom's sender-role
    # term of the reverse edge takes 36 per channel (none in layer 0), so a
    # directed edge averages half of a pair; averaged over the L launches of
    # one evaluation
    flop_kernel = {"mp_fwd": 2 * 36 * C,
                   "mp_bwd": ((99 + 36) * C * (Lc - 1) + 87 * C) / Lc + 30 * 32 + 93 / 2}
    # a split-bf16 model with C = 128 runs the forward's radial contraction
    # on the tensor cores (three bf16 MMAs per product, K = 8): 12 FMA per
    # channel stay on the CUDA cores
    fwd_tc = cs.bf16 and C == 128 and cs.K == 8
    if fwd_tc:
        flop_kernel["mp_fwd"] = 2 * (nlm + nl1) * C
        flop_tensor_fwd = 2 * 3 * cs.K * nl1 * C

    def per_launch_s(pr, k):
        v = pr.get(k)
        return v[1] / v[0] * 1e-3 if v and v[0] else None

    ranked = sorted(((k, v) for k, v in prof.items() if k in flop_method), key=lambda kv: -kv[1][1])
    name = ranked[0][0] if ranked else "mp_bwd"
    pl = per_launch_s(prof, name)
    achieved = flop_method[name] * e_cons / pl / 1e12 if pl else None
    # node arrays once and the active-edge stream (4 B of column index per
    # active entry): forward reads s, x and writes A, q (+ its split-bf16
    # copy); the adjoint reads s, gA, g_s and x and writes g_s (+ copy) and F
    n_at = sy.n_atoms
    alg_bytes = {"mp_fwd": n_at * (4 * C + 12 + 4 * nlm * C + 8 * nl1 * C) + 4 * e_cons,
                 "mp_bwd": n_at * (4 * C + 4 * nlm * C + 12 + 12 + (Lc - 1) / Lc * (4 * C + 8 * C)) + 4 * e_cons}
    roof = {"kernel": name, "bound": "alu", "achieved": achieved, "peak": fp32_pk, "unit": "TFLOP/s",
            "frac": achieved / fp32_pk if achieved else None, "traffic": ncu_traffic(name),
            "work": f"{flop_method[name]} FLOP per active edge (the method's count) x {e_cons} edges per launch",
            "peak_source": fp32_src,
            "kernel_executed_tflops": flop_kernel[name] * e_cons / pl / 1e12 if pl else None,
            "algorithmic_bytes_per_launch": alg_bytes[name]}

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
        a = rate(flop_method[k] * e_cons, per_launch_s(prof, k), 1e12)
        kr[k] = {"row": "a2+a3" if k == "mp_fwd" else "a5", "bound": "alu", "tflops": a,
                 "frac_fp32_peak": a / fp32_pk if a else None,
                 "kernel_executed_tflops": rate(flop_kernel[k] * e_cons, per_launch_s(prof, k), 1e12)}
    if fwd_tc:
        kr["mp_fwd"]["bound"] = "latency (neighbour gathers)"
        kr["mp_fwd"]["radial_on_tensor_cores_tflops"] = rate(flop_tensor_fwd * e_cons, per_launch_s(prof, "mp_fwd"), 1e12)
        kr["mp_fwd"]["note"] = ("the method's count over the FP32 peak; the radial contraction runs on the tensor "
                                "cores (three bf16 MMAs per product), the messages on the CUDA cores")
    g = rate(gemm_flop_cons, t_gemm, 1e12)
    kr["gemm_tc"] = {"row": "a4", "bound": "tensor", "tflops": g, "frac_bf16_sustained": g / bf16_pk if g and bf16_pk else None,
                     "flop_per_step": gemm_flop_cons,
                     "note": "the model's FLOP; split-bf16 issues three bf16 MMAs per product"}
    g = rate(gemm_flop_nc * I.n_inner, t_ncg, 1e12)
    kr["nc_gemm_tc"] = {"row": "a4 (NC)", "bound": "tensor", "tflops": g,
                        "frac_bf16_sustained": g / bf16_pk if g and bf16_pk else None}
    nnl = ns.lmax + 1
    flop_nc_edge = 2 * (ns.K * nnl + nnl + nnl * nnl) * Cn
    a = rate(flop_nc_edge * e_nc, per_launch_s(prof, "nc_mp_fwd"), 1e12)
    kr["nc_mp_fwd"] = {"row": "a7 (NC layer: a2+a3 at NC sizes)", "bound": "alu", "tflops": a,
                       "frac_fp32_peak": a / fp32_pk if a else None, "flop_per_edge": flop_nc_edge}
    b = rate(nc_bytes, per_launch_s(prof, "nc_head"), 1e9)
    kr["nc_head"] = {"row": "a7", "bound": "hbm", "gbs": b, "frac_hbm": b / hbm if b and hbm else None,
                     "bytes_per_launch": nc_bytes}
    # average over the n_inner launches of an outer step (the one closing
    # launch of a long call is left out)
    ib = integ_bytes_per_outer_step(I.n_inner, False) / I.n_inner
    b = rate(ib * N, per_launch_s(prof, "integrate"), 1e9)
    kr["integrate"] = {"row": "a8", "bound": "hbm", "gbs": b, "frac_hbm": b / hbm if b and hbm else None,
                       "bytes_per_launch": ib * N}
    b = rate(ib * n_at_large, per_launch_s(prof_large, "integrate"), 1e9)
    kr["integrate_100k"] = {"row": "a8", "bound": "hbm", "gbs": b, "frac_hbm": b / hbm if b and hbm else None,
                            "bytes_per_launch": ib * n_at_large}
    shares = {k: {"launches": v[0], "ms_per_step": v[1] / n_prof,
                  "share": v[1] / max(sum(x[1] for x in prof.values()), 1e-9)} for k, v in prof.items()}

    val = ns_per_day(I.dt_outer, 1e3 / ms_dmts) * world
    sts_val = ns_per_day(sts.dt_outer, 1e3 / ms_sts) * world
    sts_bf_val = ns_per_day(sts.dt_outer, 1e3 / ms_sts_bf) * world
    e2e_val = ns_per_day(I.dt_outer, 1e3 / ms_e2e) * world
    cpu = None
    if rank == 0 and not args.no_cpu and world == 1:
        t_outer, _, desc = oracle_outer_step_seconds(sy, W, 0.6)
        ncpu, model = host_cpu()
        cpu = {"value": ns_per_day(I.dt_outer, 1.0 / t_outer), "unit": "ns/day", "cores": 1, "kind": "oracle",
               "sample": desc, "host_cpus": ncpu, "cpu_model": model}
        rate, p, wall, desc_all = oracle_all_cores(sy, W, 0.6)
        cpu["all_cores"] = {"value": ns_per_day(I.dt_outer, rate), "unit": "ns/day", "cores": p,
                            "kind": "oracle, one copy per core", "sample": desc_all, "wall_s": wall}
    pick = lambda d, *ks: {k: d[k] for k in ks}   # noqa: E731
    # the contract line: headline first, short; everything else in the detail file
    line = {
        "metric": "ns/day (DMTS-NC)", "value": val, "unit": "ns/day", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_dmts, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32+bf16" if cs.bf16 else "f32", "data": "synthetic",
        "config": {"workload": sy.name, "n_atoms": sy.n_atoms,
                   "integrator": f"DMTS-NC {I.dt_outer} fs / {I.n_inner} inner, HMR +{I.hmr_delta} Da on H "
                                 f"(the paper's HMR), HHF",
                   "precision": "split-bf16 tcgen05 MLPs, fp32 elsewhere, fp64 sums" if cs.bf16 else "fp32",
                   "l2": "inputs larger than L2", "parallelism": "replicas only"},
        "speedup_vs_sts": val / sts_val,
        "sts": {"fp32_ns_per_day": sts_val, "bf16_ns_per_day": sts_bf_val, "ms_per_step": ms_sts},
        "serving": {**pick(serving, "p50_ms_per_outer_step", "p99_ms_per_outer_step", "atom_outer_steps_per_s",
                           "failed"),
                    "atoms_at_p50_p99_tick": [serving["tail"]["atoms_at_p50_tick"], serving["tail"]["atoms_at_p99_tick"]]
                    if serving["tail"] else None,
                    "chain_in_loop_ns_per_day": serving["solvated_chain_23558_in_loop"]["ns_per_day"],
                    "chain_in_loop_vs_sts": serving["solvated_chain_23558_in_loop"]["vs_sts"]},
        "e2e": {"value": e2e_val, "unit": "ns/day", "h2d_bytes_per_step": bytes_in, "d2h_bytes_per_step": bytes_out},
        "atom_steps_per_s": sy.n_atoms * 1e3 / ms_dmts * world,
        "gpu_launches": n_launches,
        "clocks": ck,
        "roofline": pick(roof, "kernel", "bound", "achieved", "peak", "unit", "frac", "traffic"),
        "configs": {k: {"ns_per_day": round(v["ns_per_day"], 2), "vs_sts": round(v["speedup_vs_sts"], 2)}
                    for k, v in others.items()},
        "cpu_baseline": pick(cpu, "value", "unit", "cores", "kind", "sample") if cpu else None,
        "cpu_all_cores": pick(cpu["all_cores"], "value", "unit", "cores") if cpu else None,
    }
    detail = dict(line, roofline=roof, cpu_baseline=cpu, thermo_end={"K": thermo_end[0], "U_plus_K": thermo_end[1],
                                                                     "T": thermo_end[2]},
                  sts={"fp32": {"ns_per_day": sts_val, "ms_per_step": ms_sts},
                       "bf16": {"ns_per_day": sts_bf_val, "ms_per_step": ms_sts_bf},
                       "dt_fs": sts.dt_outer, "atom_steps_per_s": sy.n_atoms * 1e3 / ms_sts * world},
                  speedup_vs_sts_bf16=val / sts_bf_val, serving=serving, kernels=shares, kernel_roofline=kr,
                  rewind_guard=side["guarded"], ffl=side["ffl"], npt=side["npt"], distill=side["distill"],
                  configs=others, active_edges={"cons": e_cons, "nc": e_nc})
    if rank == 0:
        if args.detail:
            os.makedirs(os.path.dirname(os.path.abspath(args.detail)), exist_ok=True)
            with open(args.detail, "w") as f:
                json.dump(detail, f, indent=1)
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
