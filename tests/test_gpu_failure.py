"""Failure detection on the GPU without a fault: a bounded device wait that
runs out reports DMTS_E_TIMEOUT through the sticky error word and leaves the
context usable."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle as O
from paper_2602_14975_gb300 import core
from paper_2602_14975_gb300 import synth as S

pytestmark = pytest.mark.gpu

GAMMA = (20.0, 1.0, 1.0, 1.0, 1.0)


@pytest.fixture(scope="module")
def small():
    cs, ns = S.cons_spec(2, 64, 1), S.nc_spec(32, rc=3.5)
    return (cs, S.cons_weights(cs, 102)), (ns, S.nc_weights(ns, 102))


def _state(sy):
    d = core.DeviceSystem([sy])
    m = O.hmr_masses(sy.species, sy.mol_id, sy.element_masses(), 3.0)
    v = S.maxwell_boltzmann(m, 300.0, 40)
    return d, core.MDState(d, v, m.astype(np.float32), seeds=7)


def test_bounded_wait_runs_out_and_the_context_stays_usable(small):
    """The library's mbarrier wait, given a 2 ms limit on a barrier nothing
    arrives on and no copy targets, gives up: dmts_sync reports
    DMTS_E_TIMEOUT once, then OK, and a following respa_step gives the same
    bits as on a fresh context."""
    import time
    ctx = core.Context(cons=small[0], nc=small[1])
    t0 = time.perf_counter()
    status = core.check_bounded_wait(ctx, 2000)
    dt = time.perf_counter() - t0
    assert status == core.L.E_TIMEOUT
    assert dt < 5.0
    assert ctx.lib.dmts_sync(ctx.handle, core._stream()) == core.L.OK
    sy = S.water_192()
    integ = core.integrator(4.0, 4, 300.0, GAMMA, skin=0.5)
    d1, s1 = _state(sy)
    core.respa_step(ctx, s1, integ, 2)
    ctx.sync()
    fresh = core.Context(cons=small[0], nc=small[1])
    d2, s2 = _state(sy)
    core.respa_step(fresh, s2, integ, 2)
    fresh.sync()
    assert np.array_equal(d1.x.cpu().numpy(), d2.x.cpu().numpy())
    s1.release()
    s2.release()
