"""GPU tests of the continuous-batching serving loop (run_replicas)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle as O
from paper_2602_14975_gb300 import core
from paper_2602_14975_gb300 import synth as S
from tests.helpers import TOL_POS

pytestmark = pytest.mark.gpu

GAMMA = (20.0, 1.0, 1.0, 1.0, 1.0)


@pytest.fixture(scope="module")
def models():
    cs = S.cons_spec(2, 64, 1)
    ns = S.nc_spec(32, rc=3.5)
    return (cs, S.cons_weights(cs, 402)), (ns, S.nc_weights(ns, 402))


@pytest.fixture(scope="module")
def ctx(models):
    return core.Context(cons=models[0], nc=models[1])


def _request(k, n_solute, n_outer, arrival=0.0):
    sy = S.capped_molecule_in_droplet(n_solute, seed=900 + k)
    m = O.hmr_masses(sy.species, sy.mol_id, sy.element_masses(), 3.0)
    v = S.maxwell_boltzmann(m, 300.0, 1000 + k)
    return core.ReplicaRequest(sy, v, m, n_outer, seed=403 * 10 ** 6 + k, replica_id=k, arrival_s=arrival)


def _integ():
    return core.integrator(10.0, 5, 300.0, GAMMA, skin=0.5)


def test_each_result_is_the_same_alone_and_in_the_mix(ctx):
    reqs = [_request(k, n, st) for k, (n, st) in enumerate([(20, 6), (45, 3), (33, 9), (20, 4), (60, 5)])]
    # three slots for five requests: admissions while others run, retirements, re-packs
    mix, stats = core.run_replicas(ctx, reqs, _integ(), max_slots=3)
    assert stats["n_ticks"] > max(r.n_outer for r in reqs)
    assert stats["max_resident"] == 3
    for k, r in enumerate(reqs):
        alone, _ = core.run_replicas(ctx, [r], _integ())
        assert mix[k]["status"] == 0 and alone[0]["status"] == 0
        assert np.abs(mix[k]["x"] - alone[0]["x"]).max() <= TOL_POS
        # replicas share no reduction: the results are in fact bit-identical
        assert np.array_equal(mix[k]["x"], alone[0]["x"])
        assert np.array_equal(mix[k]["v"], alone[0]["v"])
        assert mix[k]["energy"] == alone[0]["energy"]


def test_served_replica_matches_oracle(ctx, models):
    (cs, cb), (ns, nb) = models
    r = _request(7, 30, 4)
    out, _ = core.run_replicas(ctx, [_request(8, 25, 6), r, _request(9, 40, 2)], _integ(), max_slots=2)
    ref = O.MDState(r.system, r.v.astype(np.float64), r.masses.astype(np.float64))
    O.respa_run(ref, r.system, cs, cb, ns, nb, 10.0, 5, 300.0, np.array(GAMMA), r.seed, r.n_outer,
                replica=r.replica_id)
    assert np.abs(out[1]["x"] - ref.x).max() <= TOL_POS


def test_admission_respects_hbm_budget(ctx):
    reqs = [_request(20 + k, n, 3) for k, n in enumerate([40, 40, 40, 40])]
    fp = core.replica_footprint(ctx, reqs[0].x.shape[0])
    out, stats = core.run_replicas(ctx, reqs, _integ(), hbm_budget_bytes=2 * fp + fp // 2)
    assert stats["max_resident"] == 2
    assert all(o["status"] == 0 for o in out)
    # a request larger than the whole budget is refused, the others still run
    out, _ = core.run_replicas(ctx, reqs[:2], _integ(), hbm_budget_bytes=fp // 2)
    assert all(o["status"] == 2 for o in out)    # E_OOM


def test_poisson_arrivals_realtime(ctx):
    spec = S.serving_requests(n_req=8, seed=411, steps_lo=2, steps_hi=6, atoms_lo=20, atoms_hi=40)
    reqs = []
    for q in spec:
        sy = S.capped_molecule_in_droplet(q["n_solute"], seed=q["sys_seed"])
        m = O.hmr_masses(sy.species, sy.mol_id, sy.element_masses(), 3.0)
        v = S.maxwell_boltzmann(m, 300.0, q["sys_seed"] + 1)
        reqs.append(core.ReplicaRequest(sy, v, m, q["n_outer"], q["rng_seed"], q["id"], q["arrival_s"]))
    out, stats = core.run_replicas(ctx, reqs, _integ(), realtime=True)
    for o in out:
        assert o["status"] == 0
        assert o["t_admit_s"] >= o["t_arrival_s"] - 1e-9
        assert o["t_done_s"] >= o["t_admit_s"]
    assert stats["n_ticks"] >= max(q["n_outer"] for q in spec)
    assert np.all(stats["tick_ms"] > 0)


def test_zero_step_request_returns_its_input(ctx):
    r = _request(30, 20, 0)
    out, _ = core.run_replicas(ctx, [r], _integ())
    assert np.array_equal(out[0]["x"], r.x)


def test_alone_and_in_the_mix_at_serving_sizes():
    """The serving workload's model sizes (conservative L = 3, C = 128,
    l_max = 2, NC C = 64 at 4 Å, split-bf16 tensor-core contractions):
    packed batches whose 128-row contraction tiles span replica boundaries
    give each replica the same bits as a run alone."""
    cs, ns = S.cons_spec(3, 128, 2, bf16=True), S.nc_spec(64, rc=4.0, bf16=True)
    cx = core.Context(cons=(cs, S.cons_weights(cs, 402)), nc=(ns, S.nc_weights(ns, 402)))
    sizes = [(37, 4), (90, 3), (23, 6), (61, 2), (44, 5)]   # 148..360 atoms per replica
    reqs = [_request(40 + k, n, st) for k, (n, st) in enumerate(sizes)]
    assert any((sum(r.x.shape[0] for r in reqs[:j]) % 128) != 0 for j in range(1, 3))
    mix, stats = core.run_replicas(cx, reqs, _integ(), max_slots=3)
    assert stats["max_resident"] == 3
    for k, r in enumerate(reqs):
        alone, _ = core.run_replicas(cx, [r], _integ())
        assert mix[k]["status"] == 0 and alone[0]["status"] == 0
        assert np.array_equal(mix[k]["x"], alone[0]["x"])
        assert np.array_equal(mix[k]["v"], alone[0]["v"])
        assert mix[k]["energy"] == alone[0]["energy"]
