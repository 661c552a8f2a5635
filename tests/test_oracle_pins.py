"""Pins of the FP64 oracle against facts it does not compute itself.

Each test checks the oracle against something the paper or mathematics fixes:
published known-answer vectors, closed forms, invariances, library routines
(scipy, numpy) and textbook special cases. No GPU.
"""
import copy
import math
import os

import numpy as np
import pytest
from scipy import integrate, special
from scipy.spatial import cKDTree
from scipy.spatial.transform import Rotation

import oracle as O
from paper_2602_14975_gb300 import synth as S

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _copy_sys(sy, x=None):
    s2 = copy.deepcopy(sy)
    if x is not None:
        s2.x = np.array(x, dtype=np.float64)
    return s2


@pytest.fixture(scope="module")
def water():
    return S.water_192()


@pytest.fixture(scope="module")
def cluster():
    # open-boundary small molecule in a droplet (80 atoms)
    return S.capped_molecule_in_droplet(20, seed=7)


@pytest.fixture(scope="module")
def cons1():
    spec = S.cons_spec(2, 16, 2)
    return spec, S.cons_weights(spec, 11)


@pytest.fixture(scope="module")
def nc1():
    spec = S.nc_spec(16, rc=3.5)
    return spec, S.nc_weights(spec, 12)


# ------------------------------------------------------------------ Philox --

def test_philox_known_answer_vectors():
    rows = [l.split() for l in open(os.path.join(GOLDEN, "philox4x32_10_kat.txt"))
            if l.strip() and not l.startswith("#")]
    assert len(rows) == 3
    for r in rows:
        v = [int(t, 16) for t in r]
        out = O.philox4x32_10(v[0:4], v[4:6])
        assert list(out) == v[6:10]


def test_noise_counter_layout():
    # counter = (atom, replica, step_lo, step_hi), key = (seed_lo, seed_hi)
    seed, rep, step, atom = 0x1234567890ABCDEF, 7, (5 << 32) + 3, 11
    w = O.noise_words(seed, rep, step, atom)
    ref = O.philox4x32_10([atom, rep, 3, 5], [0x90ABCDEF, 0x12345678])
    assert list(w) == list(ref)


def test_gaussian_moments():
    # Box-Muller of uniform (w + 1/2) 2^-32: mean 0, variance 1, no correlation
    g = np.array([O.gauss3(103, 0, s, a) for s in range(200) for a in range(150)])
    n = g.shape[0]
    assert np.all(np.abs(g.mean(0)) < 5.0 / math.sqrt(n))
    assert np.all(np.abs(g.var(0) - 1.0) < 5.0 * math.sqrt(2.0 / n))
    c = np.corrcoef(g.T)
    assert np.all(np.abs(c[np.triu_indices(3, 1)]) < 5.0 / math.sqrt(n))
    # Kolmogorov-Smirnov against the standard normal (scipy)
    from scipy import stats
    for a in range(3):
        assert stats.kstest(g[:, a], "norm").pvalue > 1e-3


# --------------------------------------------------- radial basis, cutoff --

def test_bessel_closed_form_and_orthonormality():
    rc = 5.0
    # B_1(rc/2) = sqrt(2/rc) * sin(pi/2) / (rc/2)
    assert abs(O.bessel(1, rc / 2, rc) - math.sqrt(2 / rc) * 2 / rc) < 1e-15
    # spherical Bessel j0 zeros: int_0^rc B_k B_l r^2 dr = delta_kl
    for k in range(1, 9):
        for l in range(k, 9):
            val, _ = integrate.quad(lambda r: O.bessel(k, r, rc) * O.bessel(l, r, rc) * r * r,
                                    0, rc, limit=200)
            assert abs(val - (1.0 if k == l else 0.0)) < 1e-9
    # B_k(r) = sqrt(2/rc) (k pi/rc) j0(k pi r/rc) with scipy's spherical j0
    for k in (1, 3, 8):
        for r in (0.3, 1.7, 4.9):
            ref = math.sqrt(2 / rc) * (k * math.pi / rc) * special.spherical_jn(0, k * math.pi * r / rc)
            assert abs(O.bessel(k, r, rc) - ref) < 1e-13
            dref = math.sqrt(2 / rc) * (k * math.pi / rc) ** 2 * special.spherical_jn(
                0, k * math.pi * r / rc, derivative=True)
            assert abs(O.dbessel(k, r, rc) - dref) < 1e-12


@pytest.mark.parametrize("p", [5, 6, 8])
def test_envelope_smooth_cutoff(p):
    assert O.envelope(0.0, p) == 1.0
    assert O.envelope(1.0, p) == 0.0
    assert O.envelope(1.2, p) == 0.0
    h = 1e-5
    # value, first and second derivative vanish at u = 1 (C2 cutoff)
    assert abs(O.envelope(1 - h, p)) < 1e-12
    assert abs(O.denvelope(1 - h, p)) < 1e-7
    h2 = 1e-6
    d2 = (O.denvelope(1 - h2, p) - O.denvelope(1 - 2 * h2, p)) / h2
    assert abs(d2) < 2e-3
    us = np.linspace(0, 1, 101)
    vals = np.array([O.envelope(u, p) for u in us])
    assert np.all(np.diff(vals) <= 1e-15)           # monotone decreasing
    for u in (0.1, 0.5, 0.93):                       # derivative vs central difference
        fd = (O.envelope(u + 1e-6, p) - O.envelope(u - 1e-6, p)) / 2e-6
        assert abs(O.denvelope(u, p) - fd) < 1e-6


# ------------------------------------------------------ spherical harmonics --

def test_sph_norm_and_addition_theorem():
    rng = np.random.default_rng(0)
    v = rng.normal(size=(50, 3))
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    Y = np.array([O.sph(n) for n in v])
    sl = [slice(0, 1), slice(1, 4), slice(4, 9)]
    for l in range(3):
        assert np.allclose((Y[:, sl[l]] ** 2).sum(1), 2 * l + 1, atol=1e-13)
    # component normalisation: sum_m Y_lm(n) Y_lm(n') = (2l+1) P_l(n.n')
    for a in range(10):
        for b in range(10):
            cosg = float(v[a] @ v[b])
            for l in range(3):
                lhs = float(Y[a, sl[l]] @ Y[b, sl[l]])
                assert abs(lhs - (2 * l + 1) * special.eval_legendre(l, cosg)) < 1e-12


# ------------------------------------------------------------ neighbours --

def test_neighbour_list_vs_kdtree(water):
    rcut = 5.5
    rp, col = O.nbr_brute(water.x, water.box, rcut)
    tree = cKDTree(np.mod(water.x, water.box), boxsize=water.box)
    pairs = tree.query_pairs(rcut, output_type="ndarray")
    ref = set(map(tuple, pairs)) | set(map(tuple, pairs[:, ::-1]))
    got = {(i, int(j)) for i in range(water.n_atoms) for j in col[rp[i]:rp[i + 1]]}
    # scipy uses <= r; exclude pairs in a 1e-9 band at the cutoff
    d = lambda i, j: np.linalg.norm((water.x[j] - water.x[i]) - water.box * np.rint(
        (water.x[j] - water.x[i]) / water.box))
    band = {p for p in ref ^ got if abs(d(*p) - rcut) < 1e-9}
    assert (ref ^ got) == band
    # symmetric rows, no self pairs
    assert all((j, i) in got for (i, j) in got)
    assert all(i != j for (i, j) in got)


def test_neighbour_list_open_boundary(cluster):
    rp, col = O.nbr_brute(cluster.x, cluster.box, 5.0)
    tree = cKDTree(cluster.x)
    ref = tree.query_pairs(5.0)
    assert 2 * len(ref) == len(col)


# -------------------------------------------------------- conservative U --

def _rotate(sy, R, center):
    return _copy_sys(sy, (sy.x - center) @ R.T + center)


def test_cons_rotation_translation_permutation(cluster, cons1):
    spec, blob = cons1
    E0, F0 = O.cons_energy_forces(cluster, spec, blob)
    assert abs(E0) > 1e-3
    R = Rotation.random(random_state=3).as_matrix()
    c = cluster.x.mean(0)
    E1, F1 = O.cons_energy_forces(_rotate(cluster, R, c), spec, blob)
    assert abs(E1 - E0) < 1e-11 * abs(E0)
    assert np.abs(F1 - F0 @ R.T).max() < 1e-10 * np.abs(F0).max()
    E2 = O.cons_energy(_copy_sys(cluster, cluster.x + np.array([3.1, -7.2, 0.4])), spec, blob)
    assert abs(E2 - E0) < 1e-11 * abs(E0)
    perm = np.random.default_rng(1).permutation(cluster.n_atoms)
    s3 = _copy_sys(cluster, cluster.x[perm])
    s3.species = cluster.species[perm]
    E3, F3 = O.cons_energy_forces(s3, spec, blob)
    assert abs(E3 - E0) < 1e-11 * abs(E0)
    assert np.abs(F3 - F0[perm]).max() < 1e-11 * np.abs(F0).max()
    # net force vanishes (translation invariance)
    assert np.abs(F0.sum(0)).max() < 1e-12 * np.abs(F0).max() * cluster.n_atoms


def test_cons_periodic_cubic_symmetry(water):
    spec = S.cons_spec(2, 16, 2)
    blob = S.cons_weights(spec, 13)
    E0 = O.cons_energy(water, spec, blob)
    L = water.box[0]
    for M in (np.array([[0, -1, 0], [1, 0, 0], [0, 0, 1]]),       # 90 deg about z
              np.array([[0, 1, 0], [1, 0, 0], [0, 0, 1]]),        # x <-> y mirror
              -np.eye(3)):                                         # inversion
        E1 = O.cons_energy(_copy_sys(water, np.mod(water.x @ M.T, L)), spec, blob)
        assert abs(E1 - E0) < 1e-11 * abs(E0)


def test_cons_forces_finite_difference(water):
    spec = S.cons_spec(2, 16, 2)
    blob = S.cons_weights(spec, 14)
    E, F = O.cons_energy_forces(water, spec, blob)
    rng = np.random.default_rng(5)

    def cd(i, a, h):
        xp = water.x.copy(); xp[i, a] += h
        xm = water.x.copy(); xm[i, a] -= h
        return -(O.cons_energy(_copy_sys(water, xp), spec, blob)
                 - O.cons_energy(_copy_sys(water, xm), spec, blob)) / (2 * h)

    for i in rng.choice(water.n_atoms, 12, replace=False):
        for a in range(3):
            # central differences at h = 1e-4 A (truncation ~ h^2) and a
            # Richardson extrapolation of h = 1e-3, 5e-4 (truncation ~ h^4)
            assert abs(F[i, a] - cd(i, a, 1e-4)) < 1e-6 * np.abs(F).max()
            rich = (4 * cd(i, a, 5e-4) - cd(i, a, 1e-3)) / 3
            assert abs(F[i, a] - rich) < 1e-9 * np.abs(F).max()


def _silu(v):
    return v / (1 + np.exp(-v))


def _cons_parts(spec, blob):
    C, K, nl1, Sx = spec.C, spec.K, spec.lmax + 1, spec.n_species
    o = 0
    def take(n, shape):
        nonlocal o
        a = blob[o:o + n].reshape(shape)
        o += n
        return a
    emb = take(Sx * C, (Sx, C))
    layers = []
    for _ in range(spec.L):
        layers.append(dict(wrad=take(nl1 * K * C, (nl1, K, C)), w1=take(C * nl1 * C, (C, nl1 * C)),
                           b1=take(C, (C,)), w2=take(C * C, (C, C)), b2=take(C, (C,))))
    wr = take(C * C, (C, C)); br = take(C, (C,)); wo = take(C, (C,))
    assert o == blob.shape[0]
    return emb, layers, wr, br, wo


def test_cons_isolated_atoms_closed_form():
    # atoms farther apart than rc: no messages, so s^L = emb + sum_t (W2 silu(b1) + b2)
    spec = S.cons_spec(3, 8, 2)
    blob = S.cons_weights(spec, 15).copy()
    rng = np.random.default_rng(2)
    emb, layers, wr, br, wo = _cons_parts(spec, blob)
    for ly in layers:          # non-zero biases so that every term is exercised
        ly["b1"][:] = rng.normal(size=ly["b1"].shape)
        ly["b2"][:] = rng.normal(size=ly["b2"].shape)
    br[:] = rng.normal(size=br.shape)
    sp = np.array([0, 1, 2, 3, 4, 3], np.uint8)
    x = np.arange(6)[:, None] * np.array([6.0, 0.0, 0.0])
    sy = S.System("iso", x, sp, np.arange(6, dtype=np.int32), np.zeros((0, 2), np.int32),
                  np.zeros(0), np.zeros(3))
    E, F = O.cons_energy_forces(sy, spec, blob)
    s = emb[sp].copy()
    for ly in layers:
        s = s + _silu(ly["b1"]) @ ly["w2"].T + ly["b2"]
    ref = spec.scale * (_silu(s @ wr.T + br) @ wo).sum()
    assert abs(E - ref) < 1e-13 * max(1.0, abs(ref))
    assert np.abs(F).max() == 0.0


def test_cons_two_atom_closed_form():
    # for two atoms, q_i[l,c] = (nu R_lc(r) s_j[c])^2 (2l+1) whatever the direction
    spec = S.cons_spec(2, 8, 2)
    blob = S.cons_weights(spec, 16)
    emb, layers, wr, br, wo = _cons_parts(spec, blob)
    r = 2.3
    d = np.array([0.3, -0.8, 0.5]); d /= np.linalg.norm(d)
    x = np.stack([np.zeros(3), r * d])
    sp = np.array([3, 1], np.uint8)
    sy = S.System("pair", x, sp, np.arange(2, dtype=np.int32), np.zeros((0, 2), np.int32),
                  np.zeros(0), np.zeros(3))
    E = O.cons_energy(sy, spec, blob)
    fc = O.envelope(r / spec.rc, spec.p)
    B = np.array([O.bessel(k + 1, r, spec.rc) for k in range(spec.K)])
    s = emb[sp].copy()
    for ly in layers:
        R = fc * np.einsum("lkc,k->lc", ly["wrad"], B)                 # [l, c]
        deg = np.array([1, 3, 5])[:, None]
        q = np.stack([(spec.nu * R * s[1]) ** 2 * deg, (spec.nu * R * s[0]) ** 2 * deg])
        q = q.reshape(2, -1)                                            # l-major
        h = q @ ly["w1"].T + ly["b1"]
        s = s + _silu(h) @ ly["w2"].T + ly["b2"]
    ref = spec.scale * (_silu(s @ wr.T + br) @ wo).sum()
    assert abs(E - ref) < 1e-12 * abs(ref)


# ----------------------------------------------------------------- prior --

def test_prior_pins():
    sp = np.array([3, 3, 1, 0], np.uint8)   # two O (different molecules), C, H
    sig = O.PRIOR[2]
    for r, expect in ((sig, 0.0),
                      (2 ** (1 / 6) * sig, -O.PRIOR[1] * O.envelope(2 ** (1 / 6) * sig / 5.0, 6))):
        x = np.array([[0, 0, 0], [r, 0, 0], [0, 30, 0], [1.09, 30, 0]], np.float64)
        sy = S.System("p", x, sp, np.array([0, 1, 2, 2], np.int32),
                      np.array([[2, 3]], np.int32), np.array([1.09]), np.zeros(3))
        E, F = O.prior(sy, terms=O.LJ)
        assert abs(E - expect) < 1e-12
    # bond energy zero at its rest length for the rigid water template
    w = S.water_box(8, 20.0, 3, jitter=0.0)
    Eb, _ = O.prior(w, terms=O.BONDS)
    assert Eb < 1e-8          # float32 rounding of coordinates only
    # gradient by central differences (bonds + LJ)
    w = S.water_192()
    E, F = O.prior(w)
    h = 1e-5
    for i in (0, 5, 77):
        for a in range(3):
            xp = w.x.copy(); xp[i, a] += h
            xm = w.x.copy(); xm[i, a] -= h
            fd = -(O.prior(_copy_sys(w, xp))[0] - O.prior(_copy_sys(w, xm))[0]) / (2 * h)
            assert abs(F[i, a] - fd) < 1e-6 * max(1.0, abs(fd))


def test_screened_repulsion_pins():
    # ZBL universal screening: phi(0) = 1 (coefficients sum to one), so the
    # pair energy tends to the bare Coulomb repulsion k_e Z_i Z_j / r as r -> 0
    assert abs(O.zbl_phi(0.0) - 1.0) < 1e-12
    assert O.zbl_phi(5.0) < O.zbl_phi(1.0) < O.zbl_phi(0.5)
    Z = [1, 6, 7, 8, 16]
    for si, sj in ((0, 0), (3, 3), (1, 4)):
        r = 1e-5
        e, _ = O.rep_pair(si, sj, r)
        assert abs(e * r / (332.0637133 * Z[si] * Z[sj]) - 1.0) < 1e-3
        # vanishes with zero slope at the switch radius
        rc = O.PRIOR[5]
        assert O.rep_pair(si, sj, rc)[0] == 0.0
        assert abs(O.rep_pair(si, sj, rc - 1e-4)[1]) < 1e-5
        # dE/dr by central differences
        for r in (0.7, 1.6, 2.9):
            fd = (O.rep_pair(si, sj, r + 1e-6)[0] - O.rep_pair(si, sj, r - 1e-6)[0]) / 2e-6
            assert abs(O.rep_pair(si, sj, r)[1] - fd) < 1e-6 * max(1.0, abs(fd))
    # screening length a = 0.8854 a_0 / (Z_i^0.23 + Z_j^0.23): E(r) Z-scaling
    r = 0.8
    a_hh = 0.8854 * 0.529177210903 / 2.0
    assert abs(O.rep_pair(0, 0, r)[0] / O.envelope(r / O.PRIOR[5], O.PRIOR[6])
               - 332.0637133 / r * O.zbl_phi(r / a_hh)) < 1e-9
    # a bonded pair feels only its bond
    x = np.array([[0, 0, 0], [1.2, 0, 0]], float)
    sy = S.System("b", x, np.array([3, 0], np.uint8), np.zeros(2, np.int32),
                  np.array([[0, 1]], np.int32), np.array([0.9572]), np.zeros(3))
    E, _ = O.prior(sy)
    assert abs(E - 0.5 * 450.0 * (1.2 - 0.9572) ** 2) < 1e-10
    # an unbonded pair feels the repulsion
    sy.bonds = np.zeros((0, 2), np.int32)
    sy.bond_r0 = np.zeros(0)
    E, _ = O.prior(sy)
    assert abs(E - O.rep_pair(3, 0, 1.2)[0]) < 1e-10


# ---------------------------------------------------------------- NC model --

def test_nc_zero_net_force_and_equivariance(cluster, nc1):
    spec, blob = nc1
    F, net = O.nc_forces(cluster, spec, blob, with_bonds=False)
    rms = np.sqrt((F ** 2).mean())
    assert rms > 1e-4
    # antisymmetric sum cancels exactly before the mean subtraction
    assert np.abs(net).max() <= 1e-10 * rms * cluster.n_atoms
    assert np.abs(F.sum(0)).max() <= 1e-12 * rms * cluster.n_atoms
    R = Rotation.random(random_state=9).as_matrix()
    F1, _ = O.nc_forces(_rotate(cluster, R, cluster.x.mean(0)), spec, blob, with_bonds=False)
    assert np.abs(F1 - F @ R.T).max() < 1e-10 * np.abs(F).max()
    F2, _ = O.nc_forces(_copy_sys(cluster, cluster.x + 2.5), spec, blob, with_bonds=False)
    assert np.abs(F2 - F).max() < 1e-11 * np.abs(F).max()
    perm = np.random.default_rng(4).permutation(cluster.n_atoms)
    s3 = _copy_sys(cluster, cluster.x[perm]); s3.species = cluster.species[perm]
    F3, _ = O.nc_forces(s3, spec, blob, with_bonds=False)
    assert np.abs(F3 - F[perm]).max() < 1e-11 * np.abs(F).max()
    # with bonds: still zero net force before subtraction
    Fb, netb = O.nc_forces(cluster, spec, blob, with_bonds=True)
    assert np.abs(netb).max() <= 1e-10 * np.sqrt((Fb ** 2).mean()) * cluster.n_atoms


def _nc_parts(spec, blob):
    C, K, Sx, H = spec.C, spec.K, spec.n_species, spec.K + spec.n_l
    o = 0
    def take(n, shape):
        nonlocal o
        a = blob[o:o + n].reshape(shape)
        o += n
        return a
    p = dict(emb=take(Sx * C, (Sx, C)), wrad=take(2 * K * C, (2, K, C)),
             w1=take(C * 2 * C, (C, 2 * C)), b1=take(C, (C,)), w2=take(C * C, (C, C)),
             b2=take(C, (C,)), U=take(spec.n_l * C, (spec.n_l, C)),
             Wq=take(H * spec.n_c * C, (H, spec.n_c, C)), Wk=take(H * spec.n_c * C, (H, spec.n_c, C)))
    assert o == blob.shape[0]
    return p


def test_nc_two_atom_closed_form(nc1):
    # W1 = W2 = 0: x_i = emb[sp_i]; two atoms: V_ih = nu sqrt3 sum_c U_hc R_1c s_j[c] n_ij
    spec, blob0 = nc1
    blob = blob0.copy()
    p = _nc_parts(spec, blob)
    p["w1"][:] = 0.0
    p["w2"][:] = 0.0
    r = 2.1
    n = np.array([0.2, 0.9, -0.3]); n /= np.linalg.norm(n)
    sp = np.array([1, 3], np.uint8)
    sy = S.System("pair", np.stack([np.zeros(3), r * n]), sp, np.array([0, 1], np.int32),
                  np.zeros((0, 2), np.int32), np.zeros(0), np.zeros(3))
    F, net = O.nc_forces(sy, spec, blob, with_bonds=False)
    K, nl = spec.K, spec.n_l
    fc = O.envelope(r / spec.rc, spec.p)
    B = np.array([O.bessel(k + 1, r, spec.rc) for k in range(K)])
    xs = p["emb"][sp]
    R1 = fc * p["wrad"][1].T @ B                        # R_{l=1,c}
    q = np.einsum("hkc,ic->ihk", p["Wq"], xs)
    k_ = np.einsum("hkc,ic->ihk", p["Wk"], xs)
    c01 = np.einsum("hk,hk->h", q[0], k_[1]) / math.sqrt(spec.n_c)
    c10 = np.einsum("hk,hk->h", q[1], k_[0]) / math.sqrt(spec.n_c)
    v0 = spec.nu * math.sqrt(3) * (p["U"] @ (R1 * xs[1]))   # V_0h = v0[h] * n
    v1 = spec.nu * math.sqrt(3) * (p["U"] @ (R1 * xs[0]))   # V_1h = v1[h] * (-n)
    S01, S10 = c01[:K] @ B, c10[:K] @ B
    F01 = S01 * (1 + c01[K:] @ v0) * fc                  # along +n
    F10 = -S10 * (1 + c10[K:] @ v1) * fc                 # along +n (F_10 points along -n)
    ref0 = spec.scale * (F01 - F10) * n
    assert np.abs(F[0] - ref0).max() < 1e-13 * max(1e-3, np.abs(ref0).max())
    assert np.abs(F[1] + ref0).max() < 1e-13 * max(1e-3, np.abs(ref0).max())


def test_nc_cutoff_continuity(nc1):
    spec, blob = nc1
    for r in (spec.rc - 1e-4, spec.rc + 1e-4):
        sy = S.System("pair", np.array([[0, 0, 0], [r, 0, 0]], float), np.array([3, 1], np.uint8),
                      np.array([0, 1], np.int32), np.zeros((0, 2), np.int32), np.zeros(0), np.zeros(3))
        F, _ = O.nc_forces(sy, spec, blob, with_bonds=False)
        assert np.abs(F).max() < 1e-9


# ------------------------------------------------------- masses, friction --

def test_hmr_preserves_molecule_mass():
    sy = S.solvated_chain(n_chain=60, n_water=200, box_len=20.0, seed=3)
    m0 = sy.element_masses()
    m1 = O.hmr_masses(sy.species, sy.mol_id, m0, 3.0)
    for mol in np.unique(sy.mol_id):
        sel = sy.mol_id == mol
        assert abs(m1[sel].sum() - m0[sel].sum()) < 1e-10
    assert np.allclose(m1[sy.species == S.SP_H], 1.008 + 3.0)
    w = sy.mol_id > 0
    assert np.allclose(m1[w & (sy.species == S.SP_O)], 15.999 - 6.0)
    assert np.all(m1 > 0)
    # the deficit is spread over a molecule's heavy atoms in proportion to
    # their masses (Sec. 2 "Hydrogen Mass Repartitioning" fixes only the
    # per-molecule total): one common factor per molecule
    heavy = sy.species != S.SP_H
    for mol in np.unique(sy.mol_id):
        sel = (sy.mol_id == mol) & heavy
        r = m1[sel] / m0[sel]
        n_h = int(((sy.mol_id == mol) & ~heavy).sum())
        assert np.allclose(r, 1.0 - 3.0 * n_h / m0[sel].sum(), rtol=0, atol=1e-13)


def test_ostep_fluctuation_dissipation():
    # stationarity of N(0, kT/m) under v <- c1 v + c2 sqrt(1/m) G
    kT = 8.314462618 / 4184.0 * 300.0 * 4.184e-4
    c1, c2 = O.gamma_table(np.array([20.0, 1.0, 0.0, 1e6, 1.0]), 2.0, 300.0)
    for s in range(5):
        assert abs(c1[s] ** 2 * kT + c2[s] ** 2 - kT) < 1e-15
    assert c1[2] == 1.0 and c2[2] == 0.0
    assert abs(c1[0] - math.exp(-20e-3 * 2.0)) < 1e-15


# ------------------------------------------------------------ integrators --

def _vv(sy, x, v, m, dt, nsteps, spec, blob):
    """Textbook velocity Verlet with the full force -grad(U_MP + prior)."""
    conv = 4.184e-4
    def force(xx):
        s2 = _copy_sys(sy, xx)
        _, F1 = O.cons_energy_forces(s2, spec, blob)
        _, F2 = O.prior(s2)
        return F1 + F2
    F = force(x)
    for _ in range(nsteps):
        v = v + dt / 2 * conv * F / m[:, None]
        x = x + dt * v
        F = force(x)
        v = v + dt / 2 * conv * F / m[:, None]
    return x, v


@pytest.fixture(scope="module")
def small_md():
    sy = S.water_box(8, 7.0, 21, name="w24")
    cs = S.cons_spec(1, 8, 1, rc=3.4)
    cb = S.cons_weights(cs, 22)
    ns = S.nc_spec(8, rc=3.0)
    nb = S.nc_weights(ns, 23)
    m = sy.element_masses()
    v = S.maxwell_boltzmann(m, 300.0, 24)
    return sy, cs, cb, ns, nb, m, v


def test_respa_collapses_to_velocity_verlet(small_md):
    sy, cs, cb, ns, nb, m, v = small_md
    # F_S = -grad U and gamma = 0: Algorithm 1 is n velocity-Verlet steps of delta
    st = O.MDState(sy, v, m)
    O.respa_run(st, sy, cs, cb, ns, nb, 2.0, 4, 300.0, np.zeros(5), 1, n_outer=3, inner_mode=1)
    xr, vr = _vv(sy, sy.x.copy(), v.copy(), m, 0.5, 12, cs, cb)
    assert np.abs(st.x - xr).max() < 1e-12 * np.abs(xr).max()
    assert np.abs(st.v - vr).max() < 1e-12 * np.abs(vr).max()
    # n = 1, gamma = 0: velocity Verlet with step Delta whatever F_S is
    st = O.MDState(sy, v, m)
    O.respa_run(st, sy, cs, cb, ns, nb, 0.5, 1, 300.0, np.zeros(5), 1, n_outer=4, inner_mode=0)
    xr, vr = _vv(sy, sy.x.copy(), v.copy(), m, 0.5, 4, cs, cb)
    assert np.abs(st.x - xr).max() < 1e-10
    assert np.abs(st.v - vr).max() < 1e-10 * np.abs(vr).max()


def test_sts_collapses_to_velocity_verlet_and_reverses(small_md):
    # single-time-step BAOAB (the baseline of Sec. 3) at gamma = 0 is
    # velocity Verlet with the full force, and is time reversible
    sy, cs, cb, ns, nb, m, v = small_md
    st = O.MDState(sy, v, m)
    O.sts_run(st, sy, cs, cb, 0.5, 300.0, np.zeros(5), 1, 6)
    xr, vr = _vv(sy, sy.x.copy(), v.copy(), m, 0.5, 6, cs, cb)
    assert np.abs(st.x - xr).max() < 1e-12 * np.abs(xr).max()
    assert np.abs(st.v - vr).max() < 1e-12 * np.abs(vr).max()
    x1 = st.x.copy()
    st.v = -st.v
    O.sts_run(st, sy, cs, cb, 0.5, 300.0, np.zeros(5), 1, 6)
    assert np.abs(x1 - sy.x).max() > 1e-3
    assert np.abs(st.x - sy.x).max() < 1e-10


def test_sts_free_particle_temperature():
    # the O-step of single-time-step BAOAB thermalises free particles: mean
    # temperature 300 K and (T/d) chi^2_d statistics of the samples
    from scipy import stats
    n = 400
    sy = _free_gas(n, 3)
    cs, cb = S.cons_spec(1, 4, 0), S.cons_weights(S.cons_spec(1, 4, 0), 1)
    m = sy.element_masses()
    st = O.MDState(sy, np.zeros((n, 3)), m)
    conv, kB = 4.184e-4, 8.314462618 / 4184.0
    Ts = []
    for _ in range(60):
        O.sts_run(st, sy, cs, cb, 2.0, 300.0, np.full(5, 20.0), 9, 50, outer_mode=1)
        Ts.append((m[:, None] * st.v ** 2).sum() / conv / (3 * n * kB))
    Ts = np.array(Ts[10:])
    d = 3 * n
    assert abs(Ts.mean() - 300.0) < 10 * 300.0 * math.sqrt(2.0 / d) / math.sqrt(len(Ts))
    assert stats.kstest(Ts * d / 300.0, stats.chi2(d).cdf).pvalue > 1e-3


def test_sts_equals_respa_with_one_inner_step_of_the_full_force(small_md):
    # Algorithm 1 with n = 1 and F_S = F (inner_mode 1) is BAOAB with step
    # Delta: the two oracle paths draw the same noise and agree to rounding
    sy, cs, cb, ns, nb, m, v = small_md
    a = O.MDState(sy, v, m)
    O.sts_run(a, sy, cs, cb, 1.0, 300.0, np.full(5, 5.0), 17, 5)
    b = O.MDState(sy, v, m)
    O.respa_run(b, sy, cs, cb, ns, nb, 1.0, 1, 300.0, np.full(5, 5.0), 17, n_outer=5, inner_mode=1)
    assert np.abs(a.x - b.x).max() < 1e-10
    assert np.abs(a.v - b.v).max() < 1e-10 * np.abs(b.v).max()


def test_respa_time_reversible(small_md):
    sy, cs, cb, ns, nb, m, v = small_md
    st = O.MDState(sy, v, m)
    x0 = st.x.copy()
    O.respa_run(st, sy, cs, cb, ns, nb, 2.0, 4, 300.0, np.zeros(5), 1, n_outer=5)
    assert np.abs(st.x - x0).max() > 1e-2
    st.v = -st.v
    O.respa_run(st, sy, cs, cb, ns, nb, 2.0, 4, 300.0, np.zeros(5), 1, n_outer=5)
    assert np.abs(st.x - x0).max() < 1e-10


def test_nve_energy_drift_bounded():
    # gamma = 0, F_S = F = -grad E_bond: bounded, non-growing energy error
    sy = S.water_192()
    cs, cb = S.cons_spec(1, 4, 0), S.cons_weights(S.cons_spec(1, 4, 0), 1)
    m = sy.element_masses()
    v = S.maxwell_boltzmann(m, 300.0, 31)
    st = O.MDState(sy, v, m)
    conv = 4.184e-4
    def etot():
        eb, _ = O.prior(_copy_sys(sy, st.x), terms=O.BONDS)
        return eb + 0.5 * (m[:, None] * st.v ** 2).sum() / conv
    e0 = etot()
    errs = []
    for blk in range(10):
        O.respa_run(st, sy, cs, cb, cs, cb, 2.0, 4, 300.0, np.zeros(5), 1, n_outer=100,
                    inner_mode=2, outer_mode=1)
        errs.append(etot() - e0)
    errs = np.array(errs) / sy.n_atoms
    # velocity Verlet at omega*delta ~ 0.2 for O-H: O(1e-3) kcal/mol/atom
    # shadow-energy fluctuation, no secular drift
    assert np.abs(errs).max() < 1e-2
    assert abs(errs[5:].mean() - errs[:5].mean()) < 2e-3


def test_free_particle_temperature():
    # free particles under Langevin reach <T> = 300 K, (T/d) chi^2_d statistics
    from scipy import stats
    n = 400
    sy = S.System("gas", np.random.default_rng(0).uniform(0, 1000, (n, 3)),
                  np.full(n, S.SP_O, np.uint8), np.arange(n, dtype=np.int32),
                  np.zeros((0, 2), np.int32), np.zeros(0), np.zeros(3))
    cs, cb = S.cons_spec(1, 4, 0), S.cons_weights(S.cons_spec(1, 4, 0), 1)
    m = sy.element_masses()
    st = O.MDState(sy, np.zeros((n, 3)), m)
    conv, kB = 4.184e-4, 8.314462618 / 4184.0
    Ts = []
    for _ in range(60):
        O.respa_run(st, sy, cs, cb, cs, cb, 10.0, 5, 300.0, np.full(5, 20.0), 1, n_outer=20,
                    inner_mode=2, outer_mode=1)
        ke = 0.5 * (m[:, None] * st.v ** 2).sum() / conv
        Ts.append(2 * ke / (3 * n * kB))
    Ts = np.array(Ts[10:])
    d = 3 * n
    assert abs(Ts.mean() - 300.0) < 5 * 300.0 * math.sqrt(2.0 / d) / math.sqrt(len(Ts)) * 2
    assert stats.kstest(Ts * d / 300.0, stats.chi2(d).cdf).pvalue > 1e-3


def _free_gas(n, seed=0):
    return S.System("gas", np.random.default_rng(seed).uniform(0, 1000, (n, 3)),
                    np.full(n, S.SP_O, np.uint8), np.arange(n, dtype=np.int32),
                    np.zeros((0, 2), np.int32), np.zeros(0), np.zeros(3))


def test_ffl_keeps_each_direction():
    # Fast Forward Langevin (Sec. 2, the FFL update): the O-step replaces an
    # atom's speed, never its direction; plain Langevin turns the velocities
    n = 200
    sy = _free_gas(n, 1)
    cs, cb = S.cons_spec(1, 4, 0), S.cons_weights(S.cons_spec(1, 4, 0), 1)
    m = sy.element_masses()
    v0 = S.maxwell_boltzmann(m, 300.0, 5)
    out = {}
    for th in (O.LANGEVIN, O.FFL):
        st = O.MDState(sy, v0.copy(), m)
        O.sts_run(st, sy, cs, cb, 2.0, 300.0, np.full(5, 20.0), 7, 3, outer_mode=1, thermostat=th)
        out[th] = st.v.copy()
    cos = (out[O.FFL] * v0).sum(1) / (np.linalg.norm(out[O.FFL], axis=1) * np.linalg.norm(v0, axis=1))
    assert np.all(cos > 1.0 - 1e-12)
    cos_l = (out[O.LANGEVIN] * v0).sum(1) / (np.linalg.norm(out[O.LANGEVIN], axis=1) * np.linalg.norm(v0, axis=1))
    assert cos_l.min() < 0.99
    # the speeds were redrawn: not all equal to the old ones
    assert np.abs(np.linalg.norm(out[O.FFL], axis=1) - np.linalg.norm(v0, axis=1)).max() > 1e-3


def test_ffl_from_rest_equals_langevin():
    # an atom at rest has no direction: it takes the Langevin velocity
    n = 50
    sy = _free_gas(n, 2)
    cs, cb = S.cons_spec(1, 4, 0), S.cons_weights(S.cons_spec(1, 4, 0), 1)
    m = sy.element_masses()
    res = []
    for th in (O.LANGEVIN, O.FFL):
        st = O.MDState(sy, np.zeros((n, 3)), m)
        O.sts_run(st, sy, cs, cb, 2.0, 300.0, np.full(5, 20.0), 9, 1, outer_mode=1, thermostat=th)
        res.append(st.v.copy())
    assert np.array_equal(res[0], res[1])


def test_ffl_free_particle_temperature():
    # FFL leaves the canonical distribution invariant: free particles reach
    # <T> = 300 K with the (T/d) chi^2_d statistics of the Langevin case
    from scipy import stats
    n = 400
    sy = _free_gas(n, 0)
    cs, cb = S.cons_spec(1, 4, 0), S.cons_weights(S.cons_spec(1, 4, 0), 1)
    m = sy.element_masses()
    st = O.MDState(sy, np.zeros((n, 3)), m)
    conv, kB = 4.184e-4, 8.314462618 / 4184.0
    Ts = []
    for _ in range(60):
        O.respa_run(st, sy, cs, cb, cs, cb, 10.0, 5, 300.0, np.full(5, 20.0), 1, n_outer=20,
                    inner_mode=2, outer_mode=1, thermostat=O.FFL)
        ke = 0.5 * (m[:, None] * st.v ** 2).sum() / conv
        Ts.append(2 * ke / (3 * n * kB))
    Ts = np.array(Ts[10:])
    d = 3 * n
    assert abs(Ts.mean() - 300.0) < 5 * 300.0 * math.sqrt(2.0 / d) / math.sqrt(len(Ts)) * 2
    assert stats.kstest(Ts * d / 300.0, stats.chi2(d).cdf).pvalue > 1e-3


# ------------------------------------------------------------ NPT virial --

def test_nc_virial_pair_form_is_minus_sum_of_F_dot_q():
    # Sec. 2 "Computation of the virial term in NPT": with symmetric
    # neighbour lists and antisymmetric pair terms, -sum_i F_i . q_i equals
    # sum_i sum_j (F_ij + F_pair,ij / 2) . r_ij; in an open droplet q_i are
    # the plain coordinates, so both sides can be evaluated
    sy = S.capped_molecule_in_droplet(30, seed=5)
    ns = S.nc_spec(32, rc=3.5)
    nb = S.nc_weights(ns, 7)
    F, net, W = O.nc_forces(sy, ns, nb, with_virial=True)
    F_pre = F + net / sy.n_atoms
    direct = -(F_pre * sy.x).sum()
    assert abs(W - direct) <= 1e-10 * abs(direct)
    # and without the analytic fast terms
    F0, net0, W0 = O.nc_forces(sy, ns, nb, with_bonds=False, with_virial=True)
    assert abs(W0 + ((F0 + net0 / sy.n_atoms) * sy.x).sum()) <= 1e-10 * abs(W0)


def test_prior_virial_is_the_scaling_derivative_of_the_energy():
    # for any potential, d U(lambda q, lambda L) / d lambda at lambda = 1 is
    # sum_i grad_i U . q_i = -sum_i F_i . q_i; central difference of the
    # energy against the pair form, periodic (box scaled too) and open
    for sy in (S.water_192(), S.capped_molecule_in_droplet(25, seed=3)):
        for terms in (O.BONDS, O.LJ, O.REP, O.BONDS | O.LJ | O.REP):
            W = O.prior_virial(sy, terms)
            h = 1e-6
            Ep, _ = O.prior(_scaled(sy, 1 + h), terms=terms)
            Em, _ = O.prior(_scaled(sy, 1 - h), terms=terms)
            fd = (Ep - Em) / (2 * h)
            assert abs(fd - W) <= 1e-6 * max(1.0, abs(W)), (terms, fd, W)


def _scaled(sy, lam):
    return S.System(sy.name, sy.x * lam, sy.species, sy.mol_id, sy.bonds, sy.bond_r0, sy.box * lam)


def test_nc_virial_is_translation_invariant_under_pbc():
    sy = S.water_192()
    ns = S.nc_spec(32, rc=3.5)
    nb = S.nc_weights(ns, 7)
    _, _, W = O.nc_forces(sy, ns, nb, with_virial=True)
    shifted = S.System(sy.name, sy.x + np.array([3.7, -11.2, 5.05]), sy.species, sy.mol_id, sy.bonds,
                       sy.bond_r0, sy.box)
    _, _, W2 = O.nc_forces(shifted, ns, nb, with_virial=True)
    assert abs(W2 - W) <= 1e-9 * abs(W)


# --------------------------------------------------------------- barostat --

def test_baro_drift_is_the_exact_flow():
    # the piston's A half-step: x(h) solves dx/dt = v + b x with v fixed
    # (checked against an RK4 integration), velocities scale by e^(-a h),
    # the box by e^(b h); two half-steps equal one step when a = 0
    rng = np.random.default_rng(12)
    x0, v0 = rng.normal(0, 5, (7, 3)), rng.normal(0, 0.01, (7, 3))
    h, b, a = 2.0, 3e-5, 4e-5
    x, v, box = x0.copy(), v0.copy(), np.array([20.0, 21.0, 22.0])
    O.baro_drift(x, v, box, h, b, a)
    sol = integrate.solve_ivp(lambda t, y: (v0.reshape(-1) + b * y), (0, h), x0.reshape(-1), method="RK45",
                              rtol=1e-12, atol=1e-12)
    assert np.abs(x - sol.y[:, -1].reshape(-1, 3)).max() < 1e-9
    assert np.allclose(v, v0 * math.exp(-a * h), rtol=1e-14, atol=0)
    assert np.allclose(box, np.array([20.0, 21.0, 22.0]) * math.exp(b * h), rtol=1e-14, atol=0)
    x1, v1, b1 = x0.copy(), v0.copy(), np.ones(3)
    O.baro_drift(x1, v1, b1, h, b, 0.0)
    x2, v2, b2 = x0.copy(), v0.copy(), np.ones(3)
    O.baro_drift(x2, v2, b2, h / 2, b, 0.0)
    O.baro_drift(x2, v2, b2, h / 2, b, 0.0)
    assert np.abs(x1 - x2).max() < 1e-12 and np.allclose(b1, b2, rtol=1e-14)
    # b = 0 is the plain drift
    x3, v3, b3 = x0.copy(), v0.copy(), np.ones(3)
    O.baro_drift(x3, v3, b3, h, 0.0, 0.0)
    assert np.allclose(x3, x0 + h * v0, rtol=0, atol=1e-14)


def test_baro_pressure_units_and_force():
    # 1 kcal/mol/A^3 = 68,568.4 atm (SI-derived tabulated value); the piston
    # force is (1 + 3/N_f) 2K - W - 3 V P
    c = -O.baro_force(10, 0.0, 0.0, np.ones(3), 1.0) / 3.0
    assert abs(c * 68568.4 - 1.0) < 1e-5
    n, K, W, box, P = 30, 40.0, -12.5, np.array([10.0, 11.0, 12.0]), 250.0
    assert math.isclose(O.baro_force(n, K, W, box, P), (1 + 1.0 / n) * 2 * K - W - 3 * 1320.0 * P * c, rel_tol=1e-13)
    kB = 8.314462618 / 4184.0
    assert math.isclose(O.baro_mass(n, 300.0, 2000.0), (3 * n + 3) * kB * 300.0 * 2000.0 ** 2, rel_tol=1e-13)


def test_kinetic_energy_units_and_equipartition():
    # 1 amu A^2 / fs^2 = 1e-3 kg/mol x 1e10 m^2/s^2 = 1e7 J/mol = 1e7 / 4184
    # kcal/mol (CODATA amu x N_A = 1e-3 kg/mol to 4e-10); a Maxwell-Boltzmann
    # sample at T holds 3/2 N kT on average (relative spread sqrt(2 / 3N))
    m = np.array([2.0, 16.0])
    v = np.array([[1.0, 2.0, 2.0], [0.0, 0.0, 0.5]])
    amu_na = 1.66053906660e-27 * 6.02214076e23
    e_unit = amu_na * 1e10 / 4184.0
    assert math.isclose(O.kinetic(v, m), (0.5 * 2.0 * 9.0 + 0.5 * 16.0 * 0.25) * e_unit, rel_tol=1e-8)
    n, T = 30000, 300.0
    mm = np.where(np.arange(n) % 3 == 0, 15.999, 1.008)
    vv = S.maxwell_boltzmann(mm, T, 11)
    kB = 8.314462618 / 4184.0
    assert abs(O.kinetic(vv, mm) / (1.5 * n * kB * T) - 1.0) < 5.0 * math.sqrt(2.0 / (3 * n))


def test_baro_ideal_gas_volume_distribution():
    # an ideal gas (no forces) under the piston samples the isothermal-
    # isobaric volume density V^N exp(-P V / kT): <V> = (N + 1) kT / P and
    # var(V) / <V>^2 = 1 / (N + 1)
    n = 64
    sy = _free_gas(n, 0)
    sy.box = np.full(3, 10.0)
    cs, cb = S.cons_spec(1, 4, 0), S.cons_weights(S.cons_spec(1, 4, 0), 1)
    m = sy.element_masses()
    kB, T = 8.314462618 / 4184.0, 300.0
    v = S.maxwell_boltzmann(m, T, 5)
    st = O.MDState(sy, v, m)
    c = -O.baro_force(10, 0.0, 0.0, np.ones(3), 1.0) / 3.0    # kcal/mol/A^3 per atm
    v_target = 1000.0
    p_atm = (n + 1) * kB * T / v_target / c
    box = np.full(3, 10.0)
    baro = np.zeros(3)
    vols = []
    for _ in range(400):
        O.respa_run(st, sy, cs, cb, cs, cb, 4.0, 2, T, np.full(5, 5.0), 3, n_outer=20,
                    inner_mode=2, outer_mode=1, barostat=(p_atm, 0.2, box, baro))
        vols.append(float(np.prod(box)))
    vols = np.array(vols[40:])
    rel_sd = 1.0 / math.sqrt(n + 1)
    n_eff = len(vols) / 4.0          # samples 80 fs apart, correlation ~ tau_P = 200 fs
    assert abs(vols.mean() / v_target - 1.0) < 4 * rel_sd / math.sqrt(n_eff)
    assert abs(vols.var() / vols.mean() ** 2 * (n + 1) - 1.0) < 0.35
