"""NEXT-3 on its own terms (Sec. 2, "Model training": the NC model is
distilled from the large model's forces; Sec. 3 checks the kinetic
temperature of DMTS-NC runs against (T/d) chi^2(d)): on-box distillation
lowers the held-out |F_L| = |F - F_S| several-fold, and DMTS-NC with the
distilled model samples kinetic temperatures whose distribution is
(T/d) chi^2(d), d = 3N."""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")
stats = pytest.importorskip("scipy.stats")

from paper_2602_14975_gb300 import core
from paper_2602_14975_gb300 import synth as S

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def distilled():
    """The 192-water configuration's models; the NC model distilled on
    frames 20 fs apart of a single-time-step run of the conservative model.
    Returns (context, system, held-out |F_L| RMS before, after)."""
    W = S.WORKLOADS["water_192"]
    sy = W["system"]()
    cs, ns = W["cons"](), W["nc"]()
    ctx = core.Context(cons=(cs, S.cons_weights(cs, W["w_seed"])), nc=(ns, S.nc_weights(ns, W["w_seed"])))
    m = sy.element_masses()
    d = core.DeviceSystem(sy)
    st = core.MDState(d, S.maxwell_boltzmann(m, 300.0, 5), m.astype(np.float32), seeds=17)
    ig = core.integrator(1.0, 1, 300.0, (20.0,) * 5, mode=core.L.MODE_STS, skin=0.5)
    core.respa_step(ctx, st, ig, 100)
    frames = []
    for _ in range(12):
        core.respa_step(ctx, st, ig, 20)
        frames.append(d.x.cpu().numpy().astype(np.float64))
    st.release()

    def batch(xs):
        db = core.DeviceSystem([S.System(sy.name, x, sy.species, sy.mol_id, sy.bonds, sy.bond_r0, sy.box)
                                for x in xs])
        _, T = core.energy_forces_cons(ctx, db, core.nbr_build(ctx, db, cs.rc + 0.5), with_prior=True)
        return db, core.nbr_build(ctx, db, ns.rc + 0.5), T

    train, hold = batch(frames[:10]), batch(frames[10:])

    def rms(b):
        loss, _ = core.nc_distill_step(ctx, b[0], b[1], b[2], lr=0.0)
        return math.sqrt(loss.sum().item() / (3 * b[0].n_atoms))

    before = rms(hold)
    n = 600
    for k in range(n):
        lr = 2e-3 * 0.5 * (1.0 + math.cos(math.pi * k / n))
        core.nc_distill_step(ctx, train[0], train[1], train[2], lr=lr, step=k + 1)
    return ctx, sy, before, rms(hold)


def test_distillation_lowers_held_out_fl_several_fold(distilled):
    _, _, before, after = distilled
    assert after <= before / 3.0, (before, after)


def test_dmts_nc_with_the_distilled_model_samples_chi2_temperatures(distilled):
    """32 replicas, 300 outer steps of Delta = 4 fs with n = 16 (delta =
    0.25 fs, where the O(delta^2) kinetic-energy deficit of BAOAB's
    end-of-step velocities for the O-H stretch is below 0.1 %), friction
    20/ps: after 100 outer steps, the replicas' kinetic temperatures every
    25 outer steps follow (T/d) chi^2(d), d = 3 N (Kolmogorov-Smirnov
    p > 1e-3), and their mean is within 4 standard errors of T."""
    ctx, sy, _, _ = distilled
    R = 32
    systems = [sy] * R
    d = core.DeviceSystem(systems)
    m = sy.element_masses()
    v = np.concatenate([S.maxwell_boltzmann(m, 300.0, 100 + r) for r in range(R)])
    st = core.MDState(d, v, np.tile(m, R).astype(np.float32), seeds=23, replica_ids=list(range(R)), thermo=True)
    ig = core.integrator(4.0, 16, 300.0, (20.0,) * 5, skin=0.5)
    core.respa_step(ctx, st, ig, 100)
    samples = []
    for _ in range(8):
        core.respa_step(ctx, st, ig, 25)
        samples.append(st.thermo.cpu().numpy()[:, 2].copy())
    st.release()
    T = np.concatenate(samples)
    dof = 3 * sy.n_atoms
    p = stats.kstest(T * dof / 300.0, stats.chi2(dof).cdf).pvalue
    assert p > 1e-3, (p, T.mean())
    assert abs(T.mean() - 300.0) <= 4.0 * 300.0 * math.sqrt(2.0 / dof) / math.sqrt(T.size), T.mean()
