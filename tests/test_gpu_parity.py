"""GPU parity of the CUDA path against the FP64 oracle, through the C ABI.

Neighbour sets and Philox words bit-exact; FP32 forces and energies within
1e-5 relative max-abs; positions within 1e-4 A after 10 outer steps.
"""
import ctypes as ct
import os
import subprocess

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle as O
from paper_2602_14975_gb300 import core
from paper_2602_14975_gb300 import synth as S
from tests.helpers import TOL_BF16_RMS, TOL_F32, TOL_POS, band_pairs, pair_set, rel_maxabs, with_x

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def water():
    return S.water_192()


@pytest.fixture(scope="module")
def models1():
    cs = S.cons_spec(2, 64, 1)
    ns = S.nc_spec(32, rc=3.5)
    return (cs, S.cons_weights(cs, 102)), (ns, S.nc_weights(ns, 102))


@pytest.fixture(scope="module")
def ctx1(models1):
    return core.Context(cons=models1[0], nc=models1[1])


# ------------------------------------------------------------- neighbours --

def _check_pairs(sys_list, nb, rcut):
    got = pair_set(nb.row_ptr.cpu().numpy(), nb.col.cpu().numpy())
    off = 0
    ref = set()
    band = set()
    for sy in sys_list:
        rp, col = O.nbr_brute(sy.x, sy.box, rcut)
        pr = pair_set(rp, col, off)
        ref |= pr
        local = {(i - off, j - off) for (i, j) in pr}
        band |= {(i + off, j + off) for (i, j) in band_pairs(sy, local, rcut)}
        off += sy.n_atoms
    diff = got ^ ref
    assert diff <= band, f"{len(diff - band)} pairs differ outside the cutoff band"
    # each row sorted ascending (canonical order)
    rp = nb.row_ptr.cpu().numpy()
    col = nb.col.cpu().numpy()
    for i in range(len(rp) - 1):
        row = col[rp[i]:rp[i + 1]]
        assert np.all(np.diff(row) > 0)


@pytest.mark.parametrize("rcut", [3.5, 4.5, 5.5])
def test_nbr_periodic_vs_brute_force(ctx1, water, rcut):
    d = core.DeviceSystem(water)
    nb = core.nbr_build(ctx1, d, rcut)
    _check_pairs([water], nb, rcut)


def test_nbr_batched_open_and_ragged(ctx1):
    systems = [S.capped_molecule_in_droplet(n, seed=40 + n) for n in (20, 37, 150, 23)]
    d = core.DeviceSystem(systems)
    nb = core.nbr_build(ctx1, d, 5.5)
    _check_pairs(systems, nb, 5.5)


@pytest.mark.parametrize("rcut", [5.5, 9.0])
def test_nbr_large_periodic_and_overflow_retry(ctx1, rcut):
    """rcut 5.5: each cell's ~450 candidates are staged in shared memory;
    rcut 9.0: ~2,600 candidates do not fit and the per-atom sweep takes
    over. Both start from a pair capacity of 1,000 (overflow, grow, retry)."""
    sy = S.water_12288()
    d = core.DeviceSystem(sy)
    nb = core.nbr_build(ctx1, d, rcut, capacity=1000)
    rp = nb.row_ptr.cpu().numpy()
    col = nb.col.cpu().numpy()
    rng = np.random.default_rng(0)
    for i in rng.choice(sy.n_atoms, 60, replace=False):
        dd = sy.x - sy.x[i]
        dd -= sy.box * np.rint(dd / sy.box)
        r2 = (dd ** 2).sum(1)
        ref = set(np.nonzero(r2 < rcut ** 2)[0]) - {i}
        row = col[rp[i]:rp[i + 1]]
        got = set(row.tolist())
        amb = set(np.nonzero(np.abs(r2 - rcut ** 2) < 1e-4)[0])
        assert (ref ^ got) <= amb
        assert np.all(np.diff(row) > 0)


def test_nbr_empty_replica_and_single_atom(ctx1):
    lone = S.System("lone", np.zeros((1, 3)), np.array([3], np.uint8), np.zeros(1, np.int32),
                    np.zeros((0, 2), np.int32), np.zeros(0), np.zeros(3))
    d = core.DeviceSystem([lone, S.capped_molecule_in_droplet(20, seed=3)])
    nb = core.nbr_build(ctx1, d, 5.5)
    rp = nb.row_ptr.cpu().numpy()
    assert rp[1] - rp[0] == 0
    # a system without atoms: no kernel runs, and its one row offset is 0
    none = S.System("none", np.zeros((0, 3)), np.zeros(0, np.uint8), np.zeros(0, np.int32),
                    np.zeros((0, 2), np.int32), np.zeros(0), np.zeros(3))
    d0 = core.DeviceSystem(none)
    for _ in range(2):
        nb0 = core.nbr_build(ctx1, d0, 5.5)
        assert nb0.n_pairs == 0 and nb0.row_ptr.cpu().tolist() == [0]


def _state_system(systems, x):
    """The systems with the state's current positions (batched order)."""
    out, off = [], 0
    for sy in systems:
        n = sy.n_atoms
        out.append(S.System(sy.name, x[off:off + n].astype(np.float64), sy.species, sy.mol_id, sy.bonds,
                            sy.bond_r0, sy.box))
        off += n
    return out


@pytest.mark.parametrize("which", ["periodic", "open_batch"])
def test_state_lists_vs_brute_force(ctx1, models1, water, which):
    """The lists the integrator builds and rebuilds on the device (cell sweep,
    rank-ordered slot rows, the NC list flagged in the same pass), read back
    through dmts_state_lists: right after the first build both equal the
    brute-force pair sets at r_c + skin (rows ascending); after 12 outer steps
    (rebuilds on the device) every pair within the model cutoff at the current
    positions is still listed and the rows stay ascending."""
    (cs, _), (ns, _) = models1
    systems = [water] if which == "periodic" else [S.capped_molecule_in_droplet(n, seed=60 + n) for n in (30, 18, 45)]
    m = np.concatenate([sy.element_masses() for sy in systems])
    v = S.maxwell_boltzmann(m, 300.0, 103)
    d = core.DeviceSystem(systems)
    st = core.MDState(d, v, m.astype(np.float32), seeds=181)
    integ = core.integrator(4.0, 4, 300.0, [1.0] * 5, skin=0.5)
    core.respa_step(ctx1, st, integ, 0)
    for which_list, rc in ((0, cs.rc), (1, ns.rc)):
        nb = st.lists(which_list)
        assert abs(nb.r_list - (rc + 0.5)) < 1e-6
        _check_pairs(systems, nb, rc + 0.5)
    core.respa_step(ctx1, st, integ, 12)
    ctx1.sync()
    now = _state_system(systems, d.x.cpu().numpy())
    for which_list, rc in ((0, cs.rc), (1, ns.rc)):
        nb = st.lists(which_list)
        rp, col = nb.row_ptr.cpu().numpy(), nb.col.cpu().numpy()
        for i in range(len(rp) - 1):
            assert np.all(np.diff(col[rp[i]:rp[i + 1]]) > 0)
        got = pair_set(rp, col)
        off = 0
        for sy in now:
            brp, bcol = O.nbr_brute(sy.x, sy.box, rc)
            assert pair_set(brp, bcol, off) <= got
            off += sy.n_atoms
    st.release()


# ------------------------------------------------------------ conservative --

def _gpu_cons(ctx, systems, rlist=5.5, with_prior=True):
    d = core.DeviceSystem(systems)
    nb = core.nbr_build(ctx, d, rlist)
    E, F = core.energy_forces_cons(ctx, d, nb, with_prior=with_prior)
    torch.cuda.synchronize()
    return E.cpu().numpy(), F.cpu().numpy()


def test_cons_energy_forces_fp32(ctx1, models1, water):
    (cs, cb), _ = models1
    E, F = _gpu_cons(ctx1, [water], with_prior=False)
    Eo, Fo = O.cons_energy_forces(water, cs, cb)
    assert abs(E[0] - Eo) <= TOL_F32 * abs(Eo)
    assert rel_maxabs(F, Fo) <= TOL_F32
    # with the prior
    E2, F2 = _gpu_cons(ctx1, [water], with_prior=True)
    Ep, Fp = O.prior(water)
    assert abs(E2[0] - (Eo + Ep)) <= TOL_F32 * abs(Eo + Ep)
    assert rel_maxabs(F2, Fo + Fp) <= TOL_F32


def test_cons_open_boundary_batch_equals_alone(ctx1, models1):
    (cs, cb), _ = models1
    systems = [S.capped_molecule_in_droplet(n, seed=90 + n) for n in (20, 61, 33)]
    E, F = _gpu_cons(ctx1, systems)
    off = 0
    for k, sy in enumerate(systems):
        Ea, Fa = _gpu_cons(ctx1, [sy])
        n = sy.n_atoms
        assert Ea[0] == E[k]                          # bit-exact: replicas share nothing
        assert np.array_equal(Fa, F[off:off + n])
        Eo, Fo = O.cons_energy_forces(sy, cs, cb)
        Ep, Fp = O.prior(sy)
        assert abs(E[k] - (Eo + Ep)) <= TOL_F32 * max(abs(Eo + Ep), 1.0)
        assert rel_maxabs(F[off:off + n], Fo + Fp) <= TOL_F32
        off += n


def test_cons_large_lmax2_c128(water):
    cs = S.cons_spec(3, 128, 2)
    cb = S.cons_weights(cs, 302)
    ctx = core.Context(cons=(cs, cb))
    E, F = _gpu_cons(ctx, [water], with_prior=False)
    Eo, Fo = O.cons_energy_forces(water, cs, cb)
    assert abs(E[0] - Eo) <= TOL_F32 * abs(Eo)
    assert rel_maxabs(F, Fo) <= TOL_F32


@pytest.mark.parametrize("L,C,lmax", [(2, 32, 0), (2, 32, 2), (3, 128, 1)])
def test_cons_other_shapes(water, L, C, lmax):
    """The adjoint's other instantiations against the oracle: one channel per
    lane (C = 32, scalar arithmetic), l_max = 0 (the pair force along n
    only) and l_max = 1 at C = 128."""
    cs = S.cons_spec(L, C, lmax)
    cb = S.cons_weights(cs, 311)
    ctx = core.Context(cons=(cs, cb))
    E, F = _gpu_cons(ctx, [water], with_prior=False)
    Eo, Fo = O.cons_energy_forces(water, cs, cb)
    assert abs(E[0] - Eo) <= TOL_F32 * abs(Eo)
    assert rel_maxabs(F, Fo) <= TOL_F32


def _net_within_rounding(F):
    """|sum_a F_a| against the bound sum_a ulp(F_a) / 2, per component."""
    F32 = np.asarray(F, dtype=np.float32)
    net = np.abs(F32.astype(np.float64).sum(axis=0))
    bound = 0.5 * np.spacing(np.abs(F32)).astype(np.float64).sum(axis=0)
    return net, bound


@pytest.mark.parametrize("which", ["water_fp32", "droplets_fp32", "water_bf16"])
def test_cons_forces_net_zero_to_rounding(ctx1, water, which):
    """Each pair's force (Sec. 2, F = -grad U, the adjoint of the message
    passing) enters its two atoms with opposite signs in 32.32 fixed point,
    so the fixed-point sums of a replica total exactly zero, and each atom's
    fp32 force is its sum rounded once: |sum_a F_a| <= sum_a ulp(F_a) / 2
    per component and replica. A sign, index or ownership slip in the pair
    terms breaks this by orders of magnitude (the forces are of order 1e-1,
    the bound of order 1e-6)."""
    if which == "water_bf16":
        cs = S.cons_spec(3, 128, 2, bf16=True)
        ctx = core.Context(cons=(cs, S.cons_weights(cs, 302)))
    else:
        ctx = ctx1
    systems = ([S.capped_molecule_in_droplet(n, seed=70 + n) for n in (20, 61, 33)]
               if which == "droplets_fp32" else [water])
    _, F = _gpu_cons(ctx, systems, with_prior=False)
    off = 0
    for sy in systems:
        Fr = F[off:off + sy.n_atoms]
        net, bound = _net_within_rounding(Fr)
        assert np.all(net <= bound), (net, bound)
        assert np.abs(Fr).max() > 1e3 * bound.max()   # the forces are not trivially zero
        off += sy.n_atoms


def test_cons_autograd_function(ctx1, models1, water):
    (cs, cb), _ = models1
    d = core.DeviceSystem(water)
    nb = core.nbr_build(ctx1, d, 5.5)
    x = d.x.clone().requires_grad_(True)
    E = core.ConsEnergy.apply(x, ctx1, d, nb, False)
    E.sum().backward()
    g = x.grad.cpu().numpy()
    _, Fo = O.cons_energy_forces(water, cs, cb)
    assert rel_maxabs(-g, Fo) <= TOL_F32


# ---------------------------------------------------------------- NC model --

def test_nc_forces_fp32(ctx1, models1, water):
    _, (ns, nb_) = models1
    d = core.DeviceSystem(water)
    nb = core.nbr_build(ctx1, d, 4.0)
    for with_bonds in (False, True):
        F, net = core.forces_nc(ctx1, d, nb, with_bonds=with_bonds)
        F = F.cpu().numpy()
        Fo, neto = O.nc_forces(water, ns, nb_, with_bonds=with_bonds)
        assert rel_maxabs(F, Fo) <= TOL_F32
        assert np.abs(F.astype(np.float64).sum(0)).max() <= 1e-5 * np.abs(Fo).max()
        # antisymmetric sum (Sec. 2, the NC force sums to zero): each pair term,
        # bond and repulsion enters its two atoms with opposite signs in exact
        # fixed-point sums, so the pre-subtraction net force is exactly zero
        assert np.array_equal(net.cpu().numpy(), np.zeros_like(net.cpu().numpy()))


def test_nc_open_boundary_batch(ctx1, models1):
    _, (ns, nb_) = models1
    systems = [S.capped_molecule_in_droplet(n, seed=70 + n) for n in (20, 45)]
    d = core.DeviceSystem(systems)
    nb = core.nbr_build(ctx1, d, 4.0)
    F, _ = core.forces_nc(ctx1, d, nb)
    F = F.cpu().numpy()
    off = 0
    for sy in systems:
        Fo, _ = O.nc_forces(sy, ns, nb_)
        assert rel_maxabs(F[off:off + sy.n_atoms], Fo) <= TOL_F32
        off += sy.n_atoms


def test_pair_once_kernels_on_a_degenerate_batch(ctx1, models1):
    """The kernels that form each pair once, from its lower atom (the
    adjoint of the message passing; the NC head, whose persistent warps take
    atoms from a work counter), on one batch of a lone atom (no pair), an
    isolated atom pair (one pair: the lower atom's warp forms both atoms'
    terms) and a droplet: every replica's forces against the oracle, the lone
    atom's exactly zero."""
    (cs, cb), (ns, nb_) = models1
    lone = S.System("lone", np.zeros((1, 3)), np.array([3], np.uint8), np.zeros(1, np.int32),
                    np.zeros((0, 2), np.int32), np.zeros(0), np.zeros(3))
    pair = S.System("pair", np.array([[0.0, 0.0, 0.0], [1.2, 0.3, -0.2]]), np.array([3, 0], np.uint8),
                    np.zeros(2, np.int32), np.zeros((0, 2), np.int32), np.zeros(0), np.zeros(3))
    systems = [lone, pair, S.capped_molecule_in_droplet(20, seed=5)]
    d = core.DeviceSystem(systems)
    nb = core.nbr_build(ctx1, d, 5.5)
    _, F = core.energy_forces_cons(ctx1, d, nb, with_prior=False)
    Fn, _ = core.forces_nc(ctx1, d, nb, with_bonds=False)
    F, Fn = F.cpu().numpy(), Fn.cpu().numpy()
    assert np.all(F[0] == 0.0) and np.all(Fn[0] == 0.0)
    off = 1
    for sy in systems[1:]:
        n = sy.n_atoms
        _, Fo = O.cons_energy_forces(sy, cs, cb)
        Fno, _ = O.nc_forces(sy, ns, nb_, with_bonds=False)
        assert rel_maxabs(F[off:off + n], Fo) <= TOL_F32
        assert rel_maxabs(Fn[off:off + n], Fno) <= TOL_F32
        off += n


def _virial_tol(sy, ns, nb_, with_bonds=True):
    # fp32 per-atom terms summed in fp64: 1e-5 of the sum of |F_i| times the
    # list radius bounds the rounding of sum_i w_i
    F, net = O.nc_forces(sy, ns, nb_, with_bonds=with_bonds)
    return 1e-5 * np.abs(F + net / sy.n_atoms).sum() * (ns.rc + 0.5)


def test_nc_virial_matches_oracle(ctx1, models1, water):
    """Virial proxy of the fast force (Sec. 2, virial term in NPT), periodic
    box and an open-boundary batch, with and without the analytic terms."""
    _, (ns, nb_) = models1
    d = core.DeviceSystem(water)
    nb = core.nbr_build(ctx1, d, 4.0)
    for with_bonds in (False, True):
        _, _, W = core.forces_nc(ctx1, d, nb, with_bonds=with_bonds, with_virial=True)
        _, _, Wo = O.nc_forces(water, ns, nb_, with_bonds=with_bonds, with_virial=True)
        assert abs(W.item() - Wo) <= _virial_tol(water, ns, nb_, with_bonds), (W.item(), Wo)
    systems = [S.capped_molecule_in_droplet(n, seed=80 + n) for n in (20, 45)]
    d = core.DeviceSystem(systems)
    nb = core.nbr_build(ctx1, d, 4.0)
    _, _, W = core.forces_nc(ctx1, d, nb, with_virial=True)
    for r, sy in enumerate(systems):
        _, _, Wo = O.nc_forces(sy, ns, nb_, with_virial=True)
        assert abs(W[r].item() - Wo) <= _virial_tol(sy, ns, nb_), (r, W[r].item(), Wo)


def test_respa_virial_average_matches_oracle(ctx1, models1, water):
    """The state's virial_nc after each outer step is the average over its
    inner steps of the fast force's virial proxy."""
    (cs, cb), (ns, nb_) = models1
    m, v = _md_setup(water)
    d = core.DeviceSystem(water)
    st = core.MDState(d, v, m.astype(np.float32), seeds=151, virial=True)
    core.respa_step(ctx1, st, core.integrator(4.0, 4, 300.0, [1.0] * 5, skin=0.5), 3)
    ctx1.sync()
    W = st.virial_nc.cpu().numpy()[0]
    st.release()
    ref = O.MDState(water, v, m.astype(np.float32).astype(np.float64))
    wav = ct.c_double(0.0)
    O.respa_run(ref, water, cs, cb, ns, nb_, 4.0, 4, 300.0, np.full(5, 1.0), 151, 3, virial_avg=wav)
    assert abs(W - wav.value) <= _virial_tol(water, ns, nb_), (W, wav.value)


def _cons_virial_scale(F, rlist):
    return 1e-5 * np.abs(F).sum() * rlist


def test_cons_virial_matches_oracle(ctx1, models1, water):
    """Virial of the full force -grad(U_MP + prior) in pair form (Sec. 2,
    virial term in NPT). Open droplets: equal to -sum_i F_i . q_i of the
    oracle's forces. Periodic water: equal to the oracle's dU(lambda q,
    lambda L)/dlambda by central differences."""
    (cs, cb), _ = models1
    systems = [S.capped_molecule_in_droplet(n, seed=90 + n) for n in (25, 40)]
    d = core.DeviceSystem(systems)
    nb = core.nbr_build(ctx1, d, 5.5)
    _, F, W = core.energy_forces_cons(ctx1, d, nb, with_prior=True, with_virial=True)
    for r, sy in enumerate(systems):
        _, Fo = O.cons_energy_forces(sy, cs, cb)
        _, Fp = O.prior(sy)
        Ft = Fo + Fp
        ref = -(Ft * sy.x).sum()
        assert abs(W[r].item() - ref) <= _cons_virial_scale(Ft, 5.5), (r, W[r].item(), ref)
    d = core.DeviceSystem(water)
    nb = core.nbr_build(ctx1, d, 5.5)
    _, F, W = core.energy_forces_cons(ctx1, d, nb, with_prior=True, with_virial=True)

    def energy(lam):
        sy = S.System(water.name, water.x * lam, water.species, water.mol_id, water.bonds, water.bond_r0,
                      water.box * lam)
        return O.cons_energy(sy, cs, cb) + O.prior(sy)[0]

    h = 1e-6
    fd = (energy(1 + h) - energy(1 - h)) / (2 * h)
    Ft = O.cons_energy_forces(water, cs, cb)[1] + O.prior(water)[1]
    assert abs(W.item() - fd) <= _cons_virial_scale(Ft, 5.5), (W.item(), fd)


def test_respa_keeps_the_last_full_force_virial(ctx1, water):
    m, v = _md_setup(water)
    d = core.DeviceSystem(water)
    st = core.MDState(d, v, m.astype(np.float32), seeds=161, virial=True)
    core.respa_step(ctx1, st, core.integrator(4.0, 4, 300.0, [1.0] * 5, skin=0.5), 2)
    ctx1.sync()
    Wst = st.virial_cons.cpu().numpy()[0]
    st.release()
    nb = core.nbr_build(ctx1, d, 5.5)
    _, _, W = core.energy_forces_cons(ctx1, d, nb, with_prior=True, with_virial=True)
    assert abs(W.item() - Wst) <= 1e-9 * abs(Wst)


def test_respa_virial_estimator(ctx1, models1, water):
    """Virial estimator of an outer step (Sec. 2, virial term in NPT): the
    full force's virial at the end of the outer step with the fast force's
    share there replaced by its inner-step average. GPU state against (i) its
    own parts, with W_NC(q_end) evaluated afresh at the final positions, and
    (ii) the oracle's trajectory: the average from its RESPA run, W_NC from
    its fast force at its final positions and the full force's virial from
    dU(lambda q, lambda L)/dlambda there by central differences."""
    (cs, cb), (ns, nb_) = models1
    m, v = _md_setup(water)
    d = core.DeviceSystem(water)
    st = core.MDState(d, v, m.astype(np.float32), seeds=171, virial=True)
    core.respa_step(ctx1, st, core.integrator(4.0, 4, 300.0, [1.0] * 5, skin=0.5), 2)
    ctx1.sync()
    est, cons, avg = (float(t.cpu().numpy()[0]) for t in (st.virial_est, st.virial_cons, st.virial_nc))
    st.release()
    nb = core.nbr_build(ctx1, d, 4.0)
    _, _, Wl = core.forces_nc(ctx1, d, nb, with_virial=True)
    tol = _virial_tol(water, ns, nb_)
    assert abs(est - (cons - Wl.item() + avg)) <= tol, (est, cons, Wl.item(), avg)
    assert avg != Wl.item()   # the correction is not empty

    ref = O.MDState(water, v, m.astype(np.float32).astype(np.float64))
    wav = ct.c_double(0.0)
    O.respa_run(ref, water, cs, cb, ns, nb_, 4.0, 4, 300.0, np.full(5, 1.0), 171, 2, virial_avg=wav)
    end = S.System(water.name, ref.x.copy(), water.species, water.mol_id, water.bonds, water.bond_r0, water.box)
    _, _, Wl_o = O.nc_forces(end, ns, nb_, with_virial=True)

    def energy(lam):
        sy = S.System(end.name, end.x * lam, end.species, end.mol_id, end.bonds, end.bond_r0, end.box * lam)
        return O.cons_energy(sy, cs, cb) + O.prior(sy)[0]

    h = 1e-6
    cons_o = (energy(1 + h) - energy(1 - h)) / (2 * h)
    est_o = cons_o - Wl_o + wav.value
    Ft = O.cons_energy_forces(end, cs, cb)[1] + O.prior(end)[1]
    assert abs(est - est_o) <= _cons_virial_scale(Ft, 5.5) + tol, (est, est_o)


def test_virial_estimator_needs_its_parts(ctx1, water):
    m, v = _md_setup(water)
    d = core.DeviceSystem(water)
    st = core.MDState(d, v, m.astype(np.float32), seeds=171, virial=True)
    st.c.virial_nc = None
    with pytest.raises(core.L.DmtsError):
        core.respa_step(ctx1, st, core.integrator(4.0, 4, 300.0, [1.0] * 5, skin=0.5), 1)
    st.release()


def _npt_start(water, models1):
    """Initial kinetic energy, full-force virial (oracle) and the pressure in
    atm at which the piston force starts near zero."""
    (cs, cb), _ = models1
    m, v = _md_setup(water)

    def energy(lam):
        sy = S.System(water.name, water.x * lam, water.species, water.mol_id, water.bonds, water.bond_r0,
                      water.box * lam)
        return O.cons_energy(sy, cs, cb) + O.prior(sy)[0]

    h = 1e-6
    W = (energy(1 + h) - energy(1 - h)) / (2 * h)
    K = O.kinetic(v, m)
    c = -O.baro_force(10, 0.0, 0.0, np.ones(3), 1.0) / 3.0
    return m, v, (2 * K - W) / (3 * np.prod(water.box)) / c


def test_npt_matches_oracle(ctx1, models1, water):
    """Algorithm 1 with the barostat (piston on ln V / 3 driven by the virial
    estimator, MTK coupling in every A half-step): 10 outer steps against the
    oracle's trajectory, positions within the 10-step tolerance, box and
    piston momentum close, and the box moved."""
    (cs, cb), (ns, nb_) = models1
    m, v, p_atm = _npt_start(water, models1)
    tau = 0.2
    d = core.DeviceSystem(water)
    st = core.MDState(d, v, m.astype(np.float32), seeds=191, virial=True, barostat=True)
    integ = core.integrator(4.0, 4, 300.0, [1.0] * 5, skin=0.5, barostat=True, pressure_atm=p_atm, tau_p_ps=tau)
    core.respa_step(ctx1, st, integ, 6)
    core.respa_step(ctx1, st, integ, 4)      # state (piston, box) carried across calls
    ctx1.sync()
    x = d.x.cpu().numpy()
    box = d.box.cpu().numpy().reshape(-1)
    baro = st.baro.cpu().numpy()[0]
    st.release()
    ref = O.MDState(water, v, m.astype(np.float32).astype(np.float64))
    rbox, rbaro = np.array(water.box, np.float64), np.zeros(3)
    O.respa_run(ref, water, cs, cb, ns, nb_, 4.0, 4, 300.0, np.full(5, 1.0), 191, 10,
                barostat=(p_atm, tau, rbox, rbaro))
    assert np.abs(x - ref.x).max() <= TOL_POS, np.abs(x - ref.x).max()
    assert np.abs(box / rbox - 1.0).max() <= 1e-6, (box, rbox)
    assert abs(box[0] / water.box[0] - 1.0) > 1e-6      # the piston moved the box
    assert abs(baro[0] - rbaro[0]) <= 1e-3 * abs(rbaro[0]) + 1e-2, (baro, rbaro)
    assert baro[2] == 1.0


def test_npt_needs_its_arrays(ctx1, water):
    m, v = _md_setup(water)
    d = core.DeviceSystem(water)
    st = core.MDState(d, v, m.astype(np.float32), seeds=191, virial=True)    # no piston state
    with pytest.raises(core.L.DmtsError):
        core.respa_step(ctx1, st, core.integrator(4.0, 4, 300.0, [1.0] * 5, skin=0.5, barostat=True), 1)
    st.release()


def _nc_offsets(ns):
    """Offsets of the NC blob's W_rad, W1, b1, W2, b2, U and W_qk."""
    S_, C, K = ns.n_species, ns.C, ns.K
    o_wr = S_ * C
    o_w1 = o_wr + 2 * K * C
    o_b1 = o_w1 + 2 * C * C
    o_w2 = o_b1 + C
    o_b2 = o_w2 + C * C
    o_u = o_b2 + C
    o_qk = o_u + ns.n_l * C
    return {"Wrad": (o_wr, 2 * K * C), "W1": (o_w1, 2 * C * C), "b1": (o_b1, C), "W2": (o_w2, C * C),
            "b2": (o_b2, C), "U": (o_u, ns.n_l * C), "Wqk": (o_qk, 2 * (K + ns.n_l) * ns.n_c * C)}


def test_distill_gradient_matches_oracle(models1, water):
    """On-box distillation of the NC model: the loss L = sum_i |F_S,i - T_i|^2
    (F_S the fast force with bonds and repulsion, mean subtracted) and its
    gradient with respect to the q/k projection, the MLP, the radial weights
    and the tensor-head mix (the adjoint of the mean subtraction, of the NC
    head with respect to its q/k rows and V, of the contractions and the SiLU
    MLP, and of the message-passing layer with respect to its weights) against
    the oracle's loss and central differences of it; the species embedding,
    not fitted, gets zero."""
    (cs, cb), (ns, nb_) = models1
    ctx = core.Context(cons=(cs, cb), nc=(ns, nb_))      # its own context: training changes the weights
    T = O.cons_energy_forces(water, cs, cb)[1] + O.prior(water)[1]
    d = core.DeviceSystem(water)
    nb = core.nbr_build(ctx, d, 4.0)
    loss, grad = core.nc_distill_step(ctx, d, nb, T.astype(np.float32), lr=0.0, with_grad=True)
    loss, grad = loss.item(), grad.cpu().numpy()
    assert grad.size == nb_.size

    def L_oracle(blob):
        F, _ = O.nc_forces(water, ns, blob)
        return float(((F - T.astype(np.float32).astype(np.float64)) ** 2).sum())

    L0 = L_oracle(nb_)
    assert abs(loss - L0) <= 1e-4 * L0, (loss, L0)
    offs = _nc_offsets(ns)
    fitted = np.zeros(nb_.size, bool)
    for o, n in offs.values():
        fitted[o:o + n] = True
    assert not np.any(grad[~fitted])
    rng = np.random.default_rng(44)
    h = 1e-3
    for name, (o, n) in offs.items():
        gmax = np.abs(grad[o:o + n]).max()
        assert gmax > 0, name
        for k in o + rng.choice(n, 4, replace=False):
            bp, bm = nb_.copy(), nb_.copy()
            bp[k] += h
            bm[k] -= h
            fd = (L_oracle(bp) - L_oracle(bm)) / (2 * h)
            assert abs(grad[k] - fd) <= 2e-3 * gmax + 1e-6 * L0, (name, k, grad[k], fd)
    # fitting W_qk alone leaves the MLP's gradient at zero
    _, gq = core.nc_distill_step(ctx, d, nb, T.astype(np.float32), lr=0.0, params=core.L.FIT_QK, with_grad=True)
    gq = gq.cpu().numpy()
    o, n = offs["W1"]
    assert not np.any(gq[o:o + n])
    o, n = offs["Wqk"]
    assert np.allclose(gq[o:o + n], grad[o:o + n], rtol=1e-6, atol=1e-9)


def test_distill_adam_lowers_the_loss(models1, water):
    (cs, cb), (ns, nb_) = models1
    ctx = core.Context(cons=(cs, cb), nc=(ns, nb_))
    T = (O.cons_energy_forces(water, cs, cb)[1] + O.prior(water)[1]).astype(np.float32)
    d = core.DeviceSystem(water)
    nb = core.nbr_build(ctx, d, 4.0)
    losses = []
    for step in range(1, 41):
        loss, _ = core.nc_distill_step(ctx, d, nb, T, lr=2e-3, step=step)
        losses.append(loss.item())
    final, _ = core.nc_distill_step(ctx, d, nb, T, lr=0.0)
    assert final.item() < 0.8 * losses[0], (losses[0], final.item())


# ------------------------------------------------------------------ Philox --

def test_philox_words_bit_exact(ctx1):
    seed, rep, step = 0x0123456789ABCDEF, 5, (3 << 32) + 17
    w = core.philox_words(ctx1, seed, rep, step, 100, 64).cpu().numpy().view(np.uint32).reshape(-1, 4)
    for i in range(64):
        assert list(w[i]) == list(O.noise_words(seed, rep, step, 100 + i))


def test_philox_vs_curand(ctx1, tmp_path):
    so = tmp_path / "libcurandprobe.so"
    subprocess.check_call(["nvcc", "-gencode", "arch=compute_103a,code=sm_103a", "-shared",
                           "-Xcompiler", "-fPIC", "-o", str(so), os.path.join(HERE, "probes", "curand_philox.cu")])
    lib = ct.CDLL(str(so))
    lib.curand_words.argtypes = [ct.c_uint64, ct.c_uint32, ct.c_uint64, ct.c_uint32, ct.c_int, ct.c_void_p]
    ref = np.zeros(4 * 256, np.uint32)
    seed, rep, step = 987654321987, 3, 42
    assert lib.curand_words(seed, rep, step, 0, 256, ref.ctypes.data) == 0
    w = core.philox_words(ctx1, seed, rep, step, 0, 256).cpu().numpy().view(np.uint32)
    assert np.array_equal(w, ref)


def test_gaussians_match_oracle(ctx1):
    g = core.gaussians(ctx1, 103, 0, 7, 0, 500).cpu().numpy().reshape(-1, 3)
    ref = np.array([O.gauss3(103, 0, 7, i) for i in range(500)])
    assert np.abs(g - ref).max() <= 1e-5 * max(1.0, np.abs(ref).max())


# --------------------------------------------------------------- integrator --

def _md_setup(water, hmr=0.0):
    m = water.element_masses()
    if hmr:
        m = O.hmr_masses(water.species, water.mol_id, m, hmr)
    v = S.maxwell_boltzmann(m, 300.0, 103)
    return m, v


@pytest.mark.parametrize("gamma", [1.0, 0.0])
def test_respa_positions_after_10_outer_steps(ctx1, models1, water, gamma):
    (cs, cb), (ns, nb_) = models1
    m, v = _md_setup(water)
    d = core.DeviceSystem(water)
    st = core.MDState(d, v, m.astype(np.float32), seeds=103)
    integ = core.integrator(4.0, 4, 300.0, [gamma] * 5, skin=0.5)
    core.respa_step(ctx1, st, integ, 10)
    ctx1.sync()
    xg = d.x.cpu().numpy()
    ref = O.MDState(water, v, m.astype(np.float32).astype(np.float64))
    O.respa_run(ref, water, cs, cb, ns, nb_, 4.0, 4, 300.0, np.full(5, gamma), 103, 10)
    assert np.abs(xg - ref.x).max() <= TOL_POS
    assert int(st.step.cpu().numpy()[0]) == 40
    st.release()


def test_respa_ffl_positions_after_10_outer_steps(ctx1, models1, water):
    """Fast Forward Langevin O-step (HHF frictions) against the oracle, and
    the direction rule it follows: with plain Langevin the same run differs."""
    (cs, cb), (ns, nb_) = models1
    m, v = _md_setup(water)
    gam = [20.0, 1.0, 1.0, 1.0, 1.0]
    out = {}
    for th in (core.L.LANGEVIN, core.L.FFL):
        d = core.DeviceSystem(water)
        st = core.MDState(d, v, m.astype(np.float32), seeds=113)
        integ = core.integrator(4.0, 4, 300.0, gam, skin=0.5, thermostat=th)
        core.respa_step(ctx1, st, integ, 10)
        ctx1.sync()
        out[th] = d.x.cpu().numpy()
        st.release()
    ref = O.MDState(water, v, m.astype(np.float32).astype(np.float64))
    O.respa_run(ref, water, cs, cb, ns, nb_, 4.0, 4, 300.0, np.array(gam), 113, 10, thermostat=O.FFL)
    assert np.abs(out[core.L.FFL] - ref.x).max() <= TOL_POS
    assert np.abs(out[core.L.FFL] - out[core.L.LANGEVIN]).max() > 10 * TOL_POS


def test_bad_thermostat_is_rejected(ctx1, water):
    m, v = _md_setup(water)
    d = core.DeviceSystem(water)
    st = core.MDState(d, v, m.astype(np.float32), seeds=1)
    integ = core.integrator(4.0, 4, 300.0, [1.0] * 5, skin=0.5, thermostat=7)
    with pytest.raises(core.L.DmtsError):
        core.respa_step(ctx1, st, integ, 1)
    st.release()


@pytest.mark.parametrize("mode", ["respa", "sts"])
def test_respa_split_calls_equal_single_call(ctx1, water, mode):
    """A call of three or more outer steps replays the second one's CUDA
    graph for the rest; calls of one or two run every launch directly. The
    trajectories agree bit for bit, with and without the graph, and with the
    step counters (Philox keys) advanced inside the graph."""
    m, v = _md_setup(water)
    out = []
    for split in ((6,), (2, 3, 1), (1,) * 6):
        d = core.DeviceSystem(water)
        st = core.MDState(d, v, m.astype(np.float32), seeds=7)
        integ = core.integrator(4.0 if mode == "respa" else 1.0, 4, 300.0, [1.0] * 5, skin=0.5,
                                mode=core.L.MODE_RESPA if mode == "respa" else core.L.MODE_STS)
        for k in split:
            core.respa_step(ctx1, st, integ, k)
        ctx1.sync()
        out.append((d.x.cpu().numpy(), st.v.cpu().numpy(), st.step.cpu().numpy()))
        st.release()
    for o in out[1:]:
        assert np.array_equal(out[0][0], o[0])
        assert np.array_equal(out[0][1], o[1])
        assert np.array_equal(out[0][2], o[2])


def test_cached_call_graph_follows_parameter_changes(ctx1, water):
    """Calls of one outer step replay a graph the state keeps; a call with
    other integrator parameters (here the temperature) is captured anew.
    The trajectory equals the same calls run without any graph (the
    profiler, when on, keeps every launch direct)."""
    m, v = _md_setup(water)
    temps = (300.0, 300.0, 310.0, 310.0, 300.0, 300.0)
    out = []
    for direct in (False, True):
        d = core.DeviceSystem(water)
        st = core.MDState(d, v, m.astype(np.float32), seeds=5)
        if direct:
            core.profile_enable(ctx1, True)
        for T in temps:
            core.respa_step(ctx1, st, core.integrator(4.0, 4, T, [1.0] * 5, skin=0.5), 1)
        ctx1.sync()
        if direct:
            core.profile_enable(ctx1, False)
        out.append((d.x.cpu().numpy(), st.v.cpu().numpy()))
        st.release()
    assert np.array_equal(out[0][0], out[1][0])
    assert np.array_equal(out[0][1], out[1][1])


def test_cached_call_graphs_of_two_states_sharing_a_context(ctx1, water):
    """Two states of the same size but different species order (the water
    box and its atoms in reverse order) alternate one-step calls on one
    context: each replays its own cached graph, which computes its own
    species embedding (the context's workspace holds the other state's by
    then). Positions equal those of the same calls without graphs."""
    n = water.n_atoms
    rev = S.System(water.name + "_rev", water.x[::-1].copy(), water.species[::-1].copy(),
                   water.mol_id[::-1].copy(), (n - 1 - water.bonds).astype(np.int32), water.bond_r0.copy(),
                   water.box)
    out = []
    for direct in (False, True):
        states = []
        for sy in (water, rev):
            m, v = _md_setup(sy)
            d = core.DeviceSystem(sy)
            states.append((d, core.MDState(d, v, m.astype(np.float32), seeds=3)))
        if direct:
            core.profile_enable(ctx1, True)
        integ = core.integrator(4.0, 4, 300.0, [1.0] * 5, skin=0.5)
        for _ in range(3):
            for _, st in states:
                core.respa_step(ctx1, st, integ, 1)
        ctx1.sync()
        if direct:
            core.profile_enable(ctx1, False)
        out.append([d.x.cpu().numpy() for d, _ in states])
        for _, st in states:
            st.release()
    for a, b in zip(out[0], out[1]):
        assert np.array_equal(a, b)


def test_sts_positions_after_10_steps(ctx1, models1, water):
    (cs, cb), _ = models1
    m, v = _md_setup(water)
    d = core.DeviceSystem(water)
    st = core.MDState(d, v, m.astype(np.float32), seeds=11)
    integ = core.integrator(1.0, 1, 300.0, [1.0] * 5, mode=1, skin=0.5)
    core.respa_step(ctx1, st, integ, 10)
    ctx1.sync()
    ref = O.MDState(water, v, m.astype(np.float32).astype(np.float64))
    O.sts_run(ref, water, cs, cb, 1.0, 300.0, np.ones(5), 11, 10)
    assert np.abs(d.x.cpu().numpy() - ref.x).max() <= TOL_POS
    st.release()


def test_respa_hmr_hhf_replicas_batch(ctx1, models1):
    (cs, cb), (ns, nb_) = models1
    systems = [S.capped_molecule_in_droplet(n, seed=20 + n) for n in (20, 30)]
    ms, vs = [], []
    for sy in systems:
        m = O.hmr_masses(sy.species, sy.mol_id, sy.element_masses(), 3.0)
        ms.append(m)
        vs.append(S.maxwell_boltzmann(m, 300.0, 5))
    d = core.DeviceSystem(systems)
    st = core.MDState(d, np.concatenate(vs), np.concatenate(ms).astype(np.float32), seeds=[11, 12],
                      replica_ids=[4, 9])
    gam = (20.0, 1.0, 1.0, 1.0, 1.0)
    integ = core.integrator(10.0, 5, 300.0, gam, skin=0.5)
    core.respa_step(ctx1, st, integ, 10)
    ctx1.sync()
    xg = d.x.cpu().numpy()
    off = 0
    for k, sy in enumerate(systems):
        ref = O.MDState(sy, vs[k], ms[k].astype(np.float32).astype(np.float64))
        O.respa_run(ref, sy, cs, cb, ns, nb_, 10.0, 5, 300.0, np.array(gam), [11, 12][k], 10,
                    replica=[4, 9][k])
        assert np.abs(xg[off:off + sy.n_atoms] - ref.x).max() <= TOL_POS
        off += sy.n_atoms
    st.release()


def test_nonfinite_positions_are_reported(ctx1, water):
    m, v = _md_setup(water)
    x = water.x.copy()
    x[5, 0] = np.nan
    sy = with_x(water, x)
    d = core.DeviceSystem(sy)
    st = core.MDState(d, v, m.astype(np.float32), seeds=1)
    integ = core.integrator(4.0, 4, 300.0, [1.0] * 5, skin=0.5)
    from paper_2602_14975_gb300 import _lib as L
    with pytest.raises(L.DmtsError) as ei:
        core.respa_step(ctx1, st, integ, 2)
        ctx1.sync()
    assert ei.value.status in (L.E_NONFINITE, L.E_NBR_OVERFLOW, L.E_INVALID)
    st.release()
    ctx1.sync()   # the sticky word is cleared: the context stays usable


# ------------------------------------------------------- bf16 tensor cores --

def _rms(F):
    return float(np.sqrt((np.asarray(F, np.float64) ** 2).mean()))


@pytest.mark.parametrize("which", ["water", "chain"])
def test_bf16_tensor_core_path(which):
    """MLP contractions on the tensor cores with split-bf16 operands (the
    precision of the timed workload; conservative L = 3, C = 128, l_max = 2,
    NC C = 64): the message-passing force alone (no prior) and the NC force
    alone (no bonds, no repulsion), i.e. the forces the contractions
    produce, each within 2e-3 of its own RMS (max-abs) against the oracle;
    the message-passing energy within 2e-3 relative; and the total force
    (message passing + prior) within 2e-3 of its RMS."""
    sy = S.water_192() if which == "water" else S.solvated_chain(n_chain=300, n_water=900, box_len=31.0, seed=9)
    cs = S.cons_spec(3, 128, 2, bf16=True)
    ns = S.nc_spec(64, rc=4.0, bf16=True)
    cb, nb_ = S.cons_weights(cs, 302), S.nc_weights(ns, 302)
    ctx = core.Context(cons=(cs, cb), nc=(ns, nb_))
    d = core.DeviceSystem(sy)
    nb = core.nbr_build(ctx, d, 5.5)
    Eo, Fo = O.cons_energy_forces(sy, cs, cb)
    E, F = core.energy_forces_cons(ctx, d, nb, with_prior=False)
    E, F = E.cpu().numpy(), F.cpu().numpy()
    assert np.abs(F - Fo).max() <= TOL_BF16_RMS * _rms(Fo), (np.abs(F - Fo).max() / _rms(Fo))
    assert abs(E[0] - Eo) <= TOL_BF16_RMS * abs(Eo)
    Ep, Fp = O.prior(sy)
    Et, Ft = core.energy_forces_cons(ctx, d, nb, with_prior=True)
    assert np.abs(Ft.cpu().numpy() - (Fo + Fp)).max() <= TOL_BF16_RMS * _rms(Fo + Fp)
    assert abs(Et.item() - (Eo + Ep)) <= TOL_BF16_RMS * abs(Eo + Ep)
    Fno, neto = O.nc_forces(sy, ns, nb_, with_bonds=False)
    Fn, net = core.forces_nc(ctx, d, nb, with_bonds=False)
    Fn = Fn.cpu().numpy()
    assert np.abs(Fn - Fno).max() <= TOL_BF16_RMS * _rms(Fno), (np.abs(Fn - Fno).max() / _rms(Fno))
    # the fp32 SIMT contractions reach the fp32 bar on the same weights
    cs32, ns32 = S.cons_spec(3, 128, 2), S.nc_spec(64, rc=4.0)
    ctx32 = core.Context(cons=(cs32, cb), nc=(ns32, nb_))
    _, F32 = core.energy_forces_cons(ctx32, d, nb, with_prior=False)
    assert np.abs(F32.cpu().numpy() - Fo).max() <= TOL_F32 * np.abs(Fo).max()


def test_tensor_core_forward_layer_over_several_passes():
    """The forward layer's tensor-core kernel tests a row's candidates 96 at
    a time and contracts the active ones 32 at a time: with a 7.5 A list
    (about 180 candidates per row, two passes, chunks cut at pass
    boundaries) the message-passing force meets the split-bf16 bar against
    the oracle, and differs from the 5.5 A list's only by the order of the
    forward's fp32 sums (relative 1e-7) carried through the split-bf16
    contractions, whose lo parts resolve 2^-16: within 2e-4 of the RMS."""
    sy = S.solvated_chain(n_chain=300, n_water=900, box_len=31.0, seed=9)
    cs = S.cons_spec(3, 128, 2, bf16=True)
    cb = S.cons_weights(cs, 302)
    ctx = core.Context(cons=(cs, cb))
    d = core.DeviceSystem(sy)
    _, Fo = O.cons_energy_forces(sy, cs, cb)
    out = []
    for r_list in (5.5, 7.5):
        nb = core.nbr_build(ctx, d, r_list)
        if r_list == 7.5:
            rp = nb.row_ptr.cpu().numpy()
            assert np.diff(rp).max() > 96   # rows of two or more passes
        _, F = core.energy_forces_cons(ctx, d, nb, with_prior=False)
        out.append(F.cpu().numpy())
    for F in out:
        assert np.abs(F - Fo).max() <= TOL_BF16_RMS * _rms(Fo), (np.abs(F - Fo).max() / _rms(Fo))
    assert np.abs(out[0] - out[1]).max() <= 2e-4 * _rms(Fo), np.abs(out[0] - out[1]).max() / _rms(Fo)


def test_bf16_plain_is_coarser():
    """DMTS_BF16_PLAIN (one bf16 rounding per operand, hi*hi products only)
    runs the same kernels with a third of the tensor-core work: its
    message-passing force is off by a few per cent of that force's RMS
    (bf16 rounding through three layers and the adjoint), and the split
    pairs of DMTS_BF16 cut that error by more than an order of magnitude."""
    sy = S.water_192()
    cb = S.cons_weights(S.cons_spec(3, 128, 2), 302)
    Eo, Fo = O.cons_energy_forces(sy, S.cons_spec(3, 128, 2), cb)
    d = core.DeviceSystem(sy)
    err = {}
    for plain in (False, True):
        cs = S.cons_spec(3, 128, 2, bf16=True, bf16_plain=plain)
        ctx = core.Context(cons=(cs, cb))
        nb = core.nbr_build(ctx, d, 5.5)
        _, F = core.energy_forces_cons(ctx, d, nb, with_prior=False)
        err[plain] = np.abs(F.cpu().numpy() - Fo).max() / _rms(Fo)
    assert err[True] <= 1e-1
    assert err[False] <= TOL_BF16_RMS
    assert err[False] * 10 <= err[True], err


@pytest.mark.parametrize("M,N,K", [(128, 128, 64), (23558, 128, 384), (1000, 384, 128), (300, 160, 64),
                                   (4099, 64, 128), (129, 16, 64), (1, 128, 64), (92, 160, 64), (127, 64, 128)])
def test_tcgen05_contraction_exact_products(M, N, K):
    """The tensor-core contraction against an FP64 product of the same bf16
    values: only the fp32 accumulation order differs."""
    cs = S.cons_spec(1, 64, 0)
    ctx = core.Context(cons=(cs, S.cons_weights(cs, 1)))
    g = torch.Generator().manual_seed(M * 7 + N)
    a = torch.randn(M, K, generator=g).to(torch.bfloat16)
    w = torch.randn(N, K, generator=g).to(torch.bfloat16)
    out = core.contract_bf16(ctx, a.cuda(), w.cuda()).cpu().double()
    ref = a.double() @ w.double().T
    scale = (a.double().abs() @ w.double().abs().T)
    assert ((out - ref).abs() / scale).max().item() <= 1e-6 * K ** 0.5


def _split(x):
    hi = x.to(torch.bfloat16)
    lo = (x - hi.float()).to(torch.bfloat16)
    return hi, lo


@pytest.mark.parametrize("M,N,K", [(128, 128, 64), (23558, 128, 384), (1000, 384, 128), (300, 160, 64),
                                   (4099, 64, 128), (37, 128, 384)])
def test_tcgen05_split_contraction(M, N, K):
    """Split-bf16 contraction: against an FP64 evaluation of
    a_hi w_hi + a_lo w_hi + a_hi w_lo of the same bf16 values (only the fp32
    accumulation order differs), and against the FP64 product of the fp32
    operands within the 2^-16-level error that the dropped lo*lo term and
    the rounding of the lo parts leave."""
    cs = S.cons_spec(1, 64, 0)
    ctx = core.Context(cons=(cs, S.cons_weights(cs, 1)))
    g = torch.Generator().manual_seed(M * 11 + N)
    a = torch.randn(M, K, generator=g)
    w = torch.randn(N, K, generator=g)
    ah, al = _split(a)
    wh, wl = _split(w)
    a2 = torch.cat([ah, al], 1).contiguous()
    w2 = torch.cat([wh, wl], 1).contiguous()
    out = core.contract_bf16(ctx, a2.cuda(), w2.cuda(), split=True).cpu().double()
    ref3 = ah.double() @ wh.double().T + al.double() @ wh.double().T + ah.double() @ wl.double().T
    scale = (a.double().abs() @ w.double().abs().T)
    assert ((out - ref3).abs() / scale).max().item() <= 1e-6 * K ** 0.5
    exact = a.double() @ w.double().T
    assert ((out - exact).abs() / scale).max().item() <= 4.0 * 2.0 ** -16
