"""Parity on the two water boxes of the workload set besides the timed one:
12,288 atoms (49.7 Å box) and the 100,000-atom box (99.8 Å), each in the
launch configuration the benchmark runs it in (conservative L = 3, C = 128,
l_max = 2; NC C = 64, r_c = 4 Å). The oracle checks the whole 12,288-atom
energy; at 100,000 atoms it checks sampled outputs it can compute one by one
(the NC force of an atom from its local environment) and the adjoint is
checked against finite differences of the GPU energy, a property that holds
at any size."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle as O
from paper_2602_14975_gb300 import core
from paper_2602_14975_gb300 import synth as S
from tests.helpers import TOL_BF16_RMS, TOL_F32, cluster_around

pytestmark = pytest.mark.gpu

NAMES = ["water_12288", "water_100000"]
_SYS = {}


def _system(name):
    if name not in _SYS:
        _SYS[name] = S.WORKLOADS[name]["system"]()
    return _SYS[name]


def _weights(name):
    W = S.WORKLOADS[name]
    return S.cons_weights(W["cons"](), W["w_seed"]), S.nc_weights(W["nc"](), W["w_seed"])


def test_total_energy_water_12288():
    """U_MP + prior of the whole 12,288-atom box: fp32 contractions within
    1e-5 relative of the oracle, bf16 within 2e-3 relative."""
    name = "water_12288"
    sy = _system(name)
    cb, _ = _weights(name)
    d = core.DeviceSystem(sy)
    E_or = O.cons_energy(sy, S.cons_spec(3, 128, 2), cb) + O.prior(sy)[0]
    for bf16, tol in ((False, 1e-5), (True, 2e-3)):
        cs = S.cons_spec(3, 128, 2, bf16=bf16)
        ctx = core.Context(cons=(cs, cb))
        nb = core.nbr_build(ctx, d, cs.rc + 0.5)
        E, _ = core.energy_forces_cons(ctx, d, nb, with_prior=True, forces=False)
        assert abs(E.item() - E_or) <= tol * abs(E_or), (bf16, E.item(), E_or)


@pytest.mark.parametrize("name", NAMES)
@pytest.mark.parametrize("bf16", [False, True])
def test_nc_forces_sampled_atoms(name, bf16):
    """F_NC before mean subtraction on 16 sampled atoms against the oracle on
    each atom's 8.5 Å environment (one NC layer plus the head reach 2 r_c);
    the mean-subtracted force plus the reported net force over N is the
    force before subtraction, and the subtracted forces sum to zero. Bonds
    and repulsion are left out on both sides: the bars apply to the force
    the NC model produces."""
    sy = _system(name)
    _, nb_w = _weights(name)
    ns = S.nc_spec(64, rc=4.0, bf16=bf16)
    ctx = core.Context(nc=(ns, nb_w))
    d = core.DeviceSystem(sy)
    nb = core.nbr_build(ctx, d, ns.rc + 0.5)
    F, net = core.forces_nc(ctx, d, nb, with_bonds=False)
    F = F.cpu().numpy().astype(np.float64)
    pre = F + net.cpu().numpy()[0] / sy.n_atoms
    rng = np.random.default_rng(4040 + sy.n_atoms)
    sample = rng.choice(sy.n_atoms, 16, replace=False)
    ref = np.zeros((sample.size, 3))
    for k, i in enumerate(sample):
        sub, c = cluster_around(sy, int(i), 2 * ns.rc + 0.5)
        Fs, net_s = O.nc_forces(sub, ns, nb_w, with_bonds=False)
        ref[k] = Fs[c] + net_s / sub.n_atoms
    err = np.abs(pre[sample] - ref).max()
    if bf16:
        assert err <= TOL_BF16_RMS * np.sqrt((F ** 2).mean()), err
    else:
        assert err <= TOL_F32 * np.abs(ref).max(), err
    assert np.abs(F.sum(0)).max() <= 1e-5 * np.abs(F).sum()


def test_adjoint_forces_vs_finite_differences_100k():
    """Adjoint forces of U_MP (fp32 contractions) on 16 random atoms x 3
    directions of the 100,000-atom box against Richardson-extrapolated
    central differences of the GPU energy (steps h = 1e-2 Å and 2h, the steps
    taken in fp32 coordinates used): the rounding noise comes only from the
    atoms within L r_c of the moved one, as at any size."""
    name = "water_100000"
    sy = _system(name)
    cb, _ = _weights(name)
    cs = S.cons_spec(3, 128, 2)
    ctx = core.Context(cons=(cs, cb))
    d = core.DeviceSystem(sy)
    nb = core.nbr_build(ctx, d, cs.rc + 0.5)
    _, F = core.energy_forces_cons(ctx, d, nb, with_prior=False)
    F = F.cpu().numpy().astype(np.float64)
    rng = np.random.default_rng(5051)
    sample = rng.choice(sy.n_atoms, 16, replace=False)
    h = 1e-2
    x0 = d.x.clone()

    def quotient(i, a, step):
        xp, xm = x0[i, a] + step, x0[i, a] - step
        d.x[i, a] = xp
        Ep, _ = core.energy_forces_cons(ctx, d, nb, with_prior=False, forces=False)
        d.x[i, a] = xm
        Em, _ = core.energy_forces_cons(ctx, d, nb, with_prior=False, forces=False)
        d.x[i, a] = x0[i, a]
        return -(Ep.item() - Em.item()) / (float(xp.item()) - float(xm.item()))

    fd = np.zeros((sample.size, 3))
    for k, i in enumerate(sample):
        for a in range(3):
            fd[k, a] = (4.0 * quotient(i, a, h) - quotient(i, a, 2 * h)) / 3.0
    err = np.abs(fd - F[sample]).max()
    assert err <= 2e-3 * np.abs(F[sample]).max(), (err, np.abs(F[sample]).max())


def test_respa_100k_deterministic_and_moving():
    """Two outer steps of the 100,000-atom box in the benchmark's
    configuration (bf16 contractions, HMR, HHF), twice from the same state:
    bit-identical positions and velocities, finite, and the atoms moved.
    (The kinetic energy is no check here: the 0.05 Å jitter of the rigid
    starting geometry stores several kT in every O-H bond, which turns into
    kinetic energy within one vibration period.)"""
    name = "water_100000"
    W = S.WORKLOADS[name]
    sy = _system(name)
    cb, nb_w = _weights(name)
    ctx = core.Context(cons=(W["cons"](), cb), nc=(W["nc"](), nb_w))
    I = W["dmts"]
    m = core.masses_hmr(sy.species, sy.mol_id, sy.element_masses(), I.hmr_delta)
    v0 = S.maxwell_boltzmann(m, I.temperature, W["rng_seed"])
    out = []
    for _ in range(2):
        d = core.DeviceSystem(sy)
        st = core.MDState(d, v0, m.astype(np.float32), seeds=I.seed, replica_ids=[0])
        core.respa_step(ctx, st, core.integrator(I.dt_outer, I.n_inner, I.temperature, I.gamma_ps, skin=0.5), 2)
        ctx.sync()
        out.append((d.x.cpu().numpy().copy(), st.v.cpu().numpy().copy()))
        st.release()
    assert np.array_equal(out[0][0], out[1][0]) and np.array_equal(out[0][1], out[1][1])
    assert np.isfinite(out[0][0]).all() and np.isfinite(out[0][1]).all()
    assert np.abs(out[0][0] - sy.x.astype(np.float32)).max() > 1e-3
