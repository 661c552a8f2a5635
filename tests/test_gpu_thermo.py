"""GPU tests of the FP64 kinetic-energy, total-energy and temperature
reduction of respa_step (dmts_state.thermo / thermo_trace): against FP64
host sums over the same fp32 state, across call splits, batches and modes,
and a bounded, non-growing NVE energy error over 1,000 outer steps that
follows the oracle's trajectory."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle as O
from paper_2602_14975_gb300 import core
from paper_2602_14975_gb300 import synth as S

pytestmark = pytest.mark.gpu

CONV = 4.184e-4                   # (kcal/mol/A)/amu -> A/fs^2
KB = 8.314462618 / 4184.0         # kcal/mol/K
GAMMA = (20.0, 1.0, 1.0, 1.0, 1.0)


def _host_thermo(v, m, U):
    """(K, U + K, T) in FP64 from the fp32 state read back."""
    v = np.asarray(v, np.float64)
    m = np.asarray(m, np.float64)
    K = 0.5 * float((m[:, None] * v * v).sum()) / CONV
    return K, U + K, 2.0 * K / (3.0 * v.shape[0] * KB)


@pytest.fixture(scope="module")
def small():
    cs, ns = S.cons_spec(2, 64, 1), S.nc_spec(32, rc=3.5)
    return (cs, S.cons_weights(cs, 102)), (ns, S.nc_weights(ns, 102))


def _state(sy_list, seeds=7, vseeds=None, **kw):
    d = core.DeviceSystem(sy_list)
    vseeds = vseeds or [40 + k for k in range(len(sy_list))]
    ms = [O.hmr_masses(s.species, s.mol_id, s.element_masses(), 3.0) for s in sy_list]
    v = np.concatenate([S.maxwell_boltzmann(mk, 300.0, vs) for mk, vs in zip(ms, vseeds)])
    return d, core.MDState(d, v, np.concatenate(ms).astype(np.float32), seeds=seeds, **kw)


@pytest.mark.parametrize("mode", ["respa", "sts", "npt"])
def test_thermo_equals_host_fp64_sums(small, mode):
    """After a call, K equals an FP64 host sum of m v^2 / 2 over the fp32
    velocities read back (1e-12 relative: only the summation order
    differs), U + K and T follow from it, and the trace's last row is the
    call's value."""
    ctx = core.Context(cons=small[0], nc=small[1])
    sy = S.water_192()
    d, st = _state([sy], thermo=True, trace_rows=4, virial=(mode == "npt"), barostat=(mode == "npt"))
    integ = core.integrator(4.0 if mode != "sts" else 1.0, 4, 300.0, GAMMA, skin=0.5,
                            mode=core.L.MODE_STS if mode == "sts" else core.L.MODE_RESPA,
                            barostat=(mode == "npt"), pressure_atm=1.0, tau_p_ps=2.0)
    core.respa_step(ctx, st, integ, 3)
    ctx.sync()
    th = st.thermo.cpu().numpy()[0]
    K, Et, T = _host_thermo(st.v.cpu().numpy(), st.masses.cpu().numpy(), st.energy.cpu().numpy()[0])
    assert abs(th[0] - K) <= 1e-12 * K
    assert abs(th[1] - Et) <= 1e-12 * abs(Et) + 1e-12 * K
    assert abs(th[2] - T) <= 1e-12 * T
    assert 150.0 < th[2] < 450.0
    assert np.array_equal(st.thermo_trace.cpu().numpy()[2, 0], th)
    st.release()


@pytest.mark.parametrize("mode", ["respa", "sts", "npt"])
def test_trace_rows_equal_per_call_values(small, mode):
    """Row o of the trace (the velocities closed in the reduction's own
    arithmetic, before the integrator applies the pending kicks) equals,
    bit for bit, the end-of-call value of a run split into one-step calls."""
    ctx = core.Context(cons=small[0], nc=small[1])
    sy = S.water_192()
    integ = core.integrator(4.0 if mode != "sts" else 1.0, 4, 300.0, GAMMA, skin=0.5,
                            mode=core.L.MODE_STS if mode == "sts" else core.L.MODE_RESPA,
                            barostat=(mode == "npt"), pressure_atm=1.0, tau_p_ps=2.0)
    kw = dict(virial=(mode == "npt"), barostat=(mode == "npt"))
    d1, s1 = _state([sy], trace_rows=5, **kw)
    core.respa_step(ctx, s1, integ, 5)
    d2, s2 = _state([sy], thermo=True, **kw)
    rows = []
    for _ in range(5):
        core.respa_step(ctx, s2, integ, 1)
        rows.append(s2.thermo.cpu().numpy()[0].copy())
    ctx.sync()
    assert np.array_equal(s1.thermo_trace.cpu().numpy()[:, 0], np.array(rows))
    assert np.array_equal(d1.x.cpu().numpy(), d2.x.cpu().numpy())
    s1.release()
    s2.release()


def test_thermo_of_a_replica_does_not_depend_on_its_batch(small):
    ctx = core.Context(cons=small[0], nc=small[1])
    a = S.capped_molecule_in_droplet(40, seed=31)
    b = S.capped_molecule_in_droplet(25, seed=32)
    integ = core.integrator(10.0, 5, 300.0, GAMMA, skin=0.5)
    _, sa = _state([a], seeds=[9], vseeds=[50], thermo=True)
    core.respa_step(ctx, sa, integ, 4)
    _, sb = _state([b, a], seeds=[9, 9], vseeds=[51, 50], replica_ids=[0, 0], thermo=True)
    core.respa_step(ctx, sb, integ, 4)
    ctx.sync()
    assert np.array_equal(sa.thermo.cpu().numpy()[0], sb.thermo.cpu().numpy()[1])
    sa.release()
    sb.release()


def test_thermo_arguments_are_checked(small):
    ctx = core.Context(cons=small[0], nc=small[1])
    sy = S.water_192()
    _, st = _state([sy], trace_rows=2)
    with pytest.raises(core.L.DmtsError):
        core.respa_step(ctx, st, core.integrator(4.0, 4, 300.0, GAMMA, skin=0.5), 3)   # 3 > 2 rows
    st.release()


def test_nve_energy_bounded_and_follows_the_oracle():
    """gamma = 0 and a conservative fast force: both levels of Algorithm 1
    integrate the harmonic bonds alone (message-passing and NC outputs
    scaled by 0, Lennard-Jones and repulsion off), so the RESPA step is
    velocity Verlet at delta = 0.5 fs and U + K must stay bounded without
    drift (the oracle's NVE pin). Over 1,000 outer steps in ten calls the
    GPU's FP64 U + K per atom stays within 1e-2 kcal/mol of its start, the
    last five blocks' mean error is within 2e-3 of the first five's, and
    each block's U + K agrees with the oracle's trajectory within 1e-4
    kcal/mol per atom."""
    sy = S.water_192()
    cs, ns = S.cons_spec(1, 64, 0, scale=0.0), S.nc_spec(32, rc=3.5, scale=0.0)
    cb, nb = S.cons_weights(cs, 1), S.nc_weights(ns, 1)
    prior = (450.0, 0.0, 3.15, 5.0, 6.0, 0.0, 6.0)
    ctx = core.Context(cons=(cs, cb), nc=(ns, nb), prior=prior)
    m = sy.element_masses()
    v = S.maxwell_boltzmann(m, 300.0, 31)
    d = core.DeviceSystem(sy)
    st = core.MDState(d, v, m.astype(np.float32), seeds=1, thermo=True, trace_rows=100)
    integ = core.integrator(2.0, 4, 300.0, (0.0,) * 5, skin=0.5)
    ref = O.MDState(sy, v, m)
    ocs, ocb = S.cons_spec(1, 4, 0), S.cons_weights(S.cons_spec(1, 4, 0), 1)

    def oracle_etot():
        x = ref.x
        s2 = S.System(sy.name, x, sy.species, sy.mol_id, sy.bonds, sy.bond_r0, sy.box)
        eb, _ = O.prior(s2, terms=O.BONDS)
        return eb + 0.5 * (m[:, None] * ref.v ** 2).sum() / CONV

    core.respa_step(ctx, st, integ, 0)   # first call: no step, nothing reduced
    e_gpu, e_or, trace = [], [], []
    for blk in range(10):
        core.respa_step(ctx, st, integ, 100)
        O.respa_run(ref, sy, ocs, ocb, ocs, ocb, 2.0, 4, 300.0, np.zeros(5), 1, n_outer=100,
                    inner_mode=2, outer_mode=1)
        th = st.thermo.cpu().numpy()[0]
        e_gpu.append(th[1])
        e_or.append(oracle_etot())
        trace.append(st.thermo_trace.cpu().numpy()[:, 0, 1].copy())
    ctx.sync()
    e0 = _host_thermo(v.astype(np.float32), m.astype(np.float32), O.prior(sy, terms=O.BONDS)[0])[1]
    errs = (np.array(e_gpu) - e0) / sy.n_atoms
    assert np.isfinite(errs).all()
    assert np.abs(errs).max() < 1e-2, errs
    assert abs(errs[5:].mean() - errs[:5].mean()) < 2e-3, errs
    assert np.abs((np.array(e_gpu) - np.array(e_or)) / sy.n_atoms).max() < 1e-4
    # every outer step, not only the block ends
    assert np.abs((np.concatenate(trace) - e0) / sy.n_atoms).max() < 1e-2
    st.release()

