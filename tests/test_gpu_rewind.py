"""GPU tests of the rewind procedure (Sec. 2, "Preventing rare model
disagreements (Rewind procedure)") through the C ABI: disagreements are
injected on the host (a threshold, perturbed NC weights), never by faulting
the GPU."""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle as O
from paper_2602_14975_gb300 import core
from paper_2602_14975_gb300 import synth as S
from tests.helpers import TOL_POS

pytestmark = pytest.mark.gpu

DT, N_IN, T = 4.0, 4, 300.0
GAMMA = [1.0] * 5
CHUNK = 3


@pytest.fixture(scope="module")
def water():
    return S.water_192()


@pytest.fixture(scope="module")
def models():
    cs = S.cons_spec(2, 64, 1)
    ns = S.nc_spec(32, rc=3.5)
    return (cs, S.cons_weights(cs, 102)), (ns, S.nc_weights(ns, 102))


@pytest.fixture(scope="module")
def ctx(models):
    return core.Context(cons=models[0], nc=models[1])


def _state(water, seed=131):
    m = water.element_masses()
    v = S.maxwell_boltzmann(m, T, 103)
    d = core.DeviceSystem(water)
    return d, core.MDState(d, v, m.astype(np.float32), seeds=seed), m, v


def _snap(d, st):
    return d.x.cpu().numpy().copy(), st.v.cpu().numpy().copy(), int(st.step.cpu().numpy()[0])


def _integ():
    return core.integrator(DT, N_IN, T, GAMMA, skin=0.5)


def _sts_integ(dt):
    return core.integrator(dt, 1, T, GAMMA, mode=core.L.MODE_STS, skin=0.5)


def test_guard_without_disagreement_is_the_plain_run(ctx, water):
    d0, st0, _, _ = _state(water)
    core.respa_step(ctx, st0, _integ(), 10)
    ctx.sync()
    ref = _snap(d0, st0)
    st0.release()
    d1, st1, _, _ = _state(water)
    out = core.respa_guarded(ctx, st1, _integ(), 10, math.inf, CHUNK, 4, DT)
    ctx.sync()
    got = _snap(d1, st1)
    st1.release()
    assert out["n_rewinds"] == 0 and out["n_chunks"] == 4
    assert np.all(np.isfinite(out["chunk_max"])) and np.all(out["chunk_max"] > 0)
    assert np.array_equal(ref[0], got[0]) and np.array_equal(ref[1], got[1]) and ref[2] == got[2]


def test_rewind_mid_run_replays_sts_bit_for_bit(ctx, water):
    # chunk maxima of the undisturbed run decide a threshold that the run
    # first exceeds in chunk j; the guarded run must rewind there exactly
    # once and then equal "j chunks of Algorithm 1, then STS" bit for bit
    d0, st0, _, _ = _state(water)
    probe = core.respa_guarded(ctx, st0, _integ(), 8 * CHUNK, math.inf, CHUNK, 4, DT)
    st0.release()
    cm = probe["chunk_max"]
    j = next(k for k in range(1, len(cm)) if cm[k] > cm[:k].max())
    thr = 0.5 * (float(cm[:j].max()) + float(cm[j]))
    sts_steps, sts_dt = 4 * CHUNK, DT          # the STS segment spans one chunk
    d1, st1, _, _ = _state(water)
    out = core.respa_guarded(ctx, st1, _integ(), (j + 1) * CHUNK, thr, CHUNK, sts_steps, sts_dt)
    ctx.sync()
    got = _snap(d1, st1)
    st1.release()
    assert out["n_rewinds"] == 1 and out["rewind_at"][0] == j * CHUNK
    d2, st2, _, _ = _state(water)
    core.respa_step(ctx, st2, _integ(), j * CHUNK)
    core.respa_step(ctx, st2, _sts_integ(sts_dt), sts_steps)
    ctx.sync()
    ref = _snap(d2, st2)
    st2.release()
    assert np.array_equal(ref[0], got[0]) and np.array_equal(ref[1], got[1]) and ref[2] == got[2]


def test_perturbed_nc_weights_trigger_exactly_one_rewind(models, water):
    """A fast model that disagrees with the large one (its attention weights
    W_q, W_k scaled by 10, so every c_ijh by 100) drives |F - F_S| far above
    the undisturbed level: the first outer step is rewound, the
    single-time-step segment replaces it, and that segment follows the
    oracle's STS trajectory."""
    (cs, cb), (ns, nb_) = models
    ctx_ok = core.Context(cons=(cs, cb), nc=(ns, nb_))
    d0, st0, _, _ = _state(water)
    base = core.respa_guarded(ctx_ok, st0, _integ(), 1, math.inf, 1, 4, 1.0)["chunk_max"][0]
    st0.release()
    H = ns.K + ns.n_l
    bad = nb_.copy()
    bad[-2 * H * ns.n_c * ns.C:] *= 10.0
    ctx_bad = core.Context(cons=(cs, cb), nc=(ns, bad))
    d1, st1, m, v = _state(water)
    sts_steps, sts_dt = 4, 1.0                 # one outer step of 4 fs
    out = core.respa_guarded(ctx_bad, st1, _integ(), 1, 10.0 * base, 1, sts_steps, sts_dt)
    ctx_bad.sync()
    got = _snap(d1, st1)
    st1.release()
    assert out["n_rewinds"] == 1 and out["n_chunks"] == 1
    assert not (out["chunk_max"][0] <= 10.0 * base)
    ref = O.MDState(water, v.astype(np.float64), m.astype(np.float32).astype(np.float64))
    O.sts_run(ref, water, cs, cb, sts_dt, T, np.array(GAMMA), 131, sts_steps)
    assert np.abs(got[0] - ref.x).max() <= TOL_POS
    assert got[2] == sts_steps


def test_guard_rejects_bad_parameters(ctx, water):
    d, st, _, _ = _state(water)
    with pytest.raises(core.L.DmtsError):
        core.respa_guarded(ctx, st, _integ(), 6, 1.0, 0, 4, DT)          # no chunk
    with pytest.raises(core.L.DmtsError):
        core.respa_guarded(ctx, st, _integ(), 6, 1.0, 3, 3, 1.5)         # 4.5 fs: not whole outer steps
    with pytest.raises(core.L.DmtsError):
        core.respa_guarded(ctx, st, _sts_integ(1.0), 6, 1.0, 3, 4, DT)   # wraps RESPA only
    st.release()


def test_rewind_under_the_barostat_restores_box_and_piston(ctx, water):
    """With the barostat the saved frame holds the box and the piston state:
    a rewind returns to them, and the run equals "j chunks of Algorithm 1
    under the barostat, then STS (box fixed)" bit for bit, box included."""
    m = water.element_masses()
    v = S.maxwell_boltzmann(m, T, 103)
    d0 = core.DeviceSystem(water)
    s0 = core.MDState(d0, v, m.astype(np.float32), seeds=131, virial=True, barostat=True)
    core.respa_step(ctx, s0, core.integrator(DT, N_IN, T, GAMMA, skin=0.5, barostat=True), 0)
    ctx.sync()
    K = O.kinetic(v, m)
    c = -O.baro_force(10, 0.0, 0.0, np.ones(3), 1.0) / 3.0
    p_atm = (2 * K - float(s0.virial_cons[0].item())) / (3 * np.prod(water.box)) / c
    s0.release()

    def npt():
        return core.integrator(DT, N_IN, T, GAMMA, skin=0.5, barostat=True, pressure_atm=p_atm, tau_p_ps=0.2)

    def fresh():
        d = core.DeviceSystem(water)
        return d, core.MDState(d, v, m.astype(np.float32), seeds=131, virial=True, barostat=True)

    d1, s1 = fresh()
    probe = core.respa_guarded(ctx, s1, npt(), 6 * CHUNK, math.inf, CHUNK, 4, DT)
    s1.release()
    cm = probe["chunk_max"]
    j = next(k for k in range(1, len(cm)) if cm[k] > cm[:k].max())
    thr = 0.5 * (float(cm[:j].max()) + float(cm[j]))
    sts_steps, sts_dt = 4 * CHUNK, DT
    d2, s2 = fresh()
    out = core.respa_guarded(ctx, s2, npt(), (j + 1) * CHUNK, thr, CHUNK, sts_steps, sts_dt)
    ctx.sync()
    got = (d2.x.cpu().numpy().copy(), s2.v.cpu().numpy().copy(), d2.box.cpu().numpy().copy())
    s2.release()
    assert out["n_rewinds"] == 1 and out["rewind_at"][0] == j * CHUNK
    d3, s3 = fresh()
    core.respa_step(ctx, s3, npt(), j * CHUNK)
    core.respa_step(ctx, s3, _sts_integ(sts_dt), sts_steps)
    ctx.sync()
    ref = (d3.x.cpu().numpy().copy(), s3.v.cpu().numpy().copy(), d3.box.cpu().numpy().copy())
    s3.release()
    assert all(np.array_equal(a, b) for a, b in zip(ref, got))
    assert not np.array_equal(ref[2], water.box.astype(np.float32).reshape(ref[2].shape))   # the box moved
