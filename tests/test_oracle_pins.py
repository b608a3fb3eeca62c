"""Pins of the FP64 oracle against what the paper and mathematics fix (CPU only).

Each test checks the oracle against something other than itself: published values,
closed forms, brute force, or invariants, chosen so that a dropped term, a wrong sign
or index, or a transposed operand fails at least one of them.
"""
import math
import os

import numpy as np
import pytest

import oracle
from paper_1904_08756_gb300 import synth

S = 1 << 20
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# --------------------------------------------------------------------------------------
# Philox4x32-10 (Salmon et al., SC'11) against its published known-answer vectors
# --------------------------------------------------------------------------------------

def test_philox_known_answers():
    rows = [l.split() for l in open(os.path.join(GOLDEN, "philox4x32_10_kat.txt"))
            if l.strip() and not l.startswith("#")]
    assert len(rows) == 3
    for r in rows:
        w = [int(x, 16) for x in r]
        out = oracle.philox(w[0:4], w[4:6])
        assert [int(x) for x in out] == w[6:10]


# --------------------------------------------------------------------------------------
# Constants
# --------------------------------------------------------------------------------------

def test_physical_constants():
    # e^2 N_A / (4 pi eps0) = 1389.35458 kJ A / mol / e^2 (= 138.935458 kJ nm / mol / e^2)
    assert abs(oracle.coulomb_constant() - 1389.35458) < 2e-5
    # R = 8.314462618 J / mol / K
    assert abs(oracle.gas_constant() - 8.314462618e-3) < 1e-12


# --------------------------------------------------------------------------------------
# Minimum image, exact squared distance, bins
# --------------------------------------------------------------------------------------

def test_min_image_is_the_nearest_image():
    rng = np.random.default_rng(5)
    for L in (7, 8, 21810381, 104857250):
        for dx in list(rng.integers(-L + 1, L, 300)) + [L // 2, -(L // 2), (L + 1) // 2, 0,
                                                       L - 1, -L + 1]:
            m = oracle.min_image(int(dx), L)
            assert (m - dx) % L == 0
            cands = [abs(dx + k * L) for k in (-2, -1, 0, 1, 2)]
            assert abs(m) == min(cands)
            assert -L < 2 * m <= L


def test_bin_index_is_floor_of_r_over_dr():
    """k satisfies (k dr)^2 <= r^2 < ((k+1) dr)^2, checked in exact integers."""
    rng = np.random.default_rng(6)
    for p, q in ((3, 100), (2, 100), (1, 10), (7, 3)):
        d2s = list(rng.integers(0, 3 * (60 * S) ** 2, 400)) + [0, 1, 3 * (1 << 52)]
        for d2 in d2s:
            d2 = int(d2)
            k = oracle.bin_index(d2, p, q)
            # r / dr = sqrt(d2) q / (p S):  k <= that < k+1  <=>  (k p S)^2 <= d2 q^2 < ((k+1) p S)^2
            assert (k * p * S) ** 2 <= d2 * q * q < ((k + 1) * p * S) ** 2


def test_two_atoms_on_a_bin_edge():
    """r = 0.75 A is exactly the lower edge of bin 25 for 0.03 A bins."""
    edge = 786432                          # 0.75 * 2^20
    assert oracle.bin_index(edge * edge, 3, 100) == 25
    assert oracle.bin_index(edge * edge - 1, 3, 100) == 24


def _r3(n):
    """Number of integer vectors with squared length n (brute force)."""
    m = int(math.isqrt(n)) + 1
    return sum(1 for a in range(-m, m + 1) for b in range(-m, m + 1) for c in range(-m, m + 1)
               if a * a + b * b + c * c == n)


def test_simple_cubic_shell_counts():
    """Shell counts of a simple-cubic lattice (spacing 1 A): N r3(n) / 2 unordered pairs
    at r = sqrt(n) A for r < L/2, r3 the number of integer vectors of squared length n."""
    n_side = 8
    sysl = synth.lattice_box(n_side, S, n_bins=80, bin_p=1, bin_q=20)   # 0.05 A bins, 4 A
    box = oracle.Box(sysl)
    H = box.histogram()[0]
    N = sysl.n_atoms
    expect = np.zeros(80, np.uint64)
    for n in range(1, 16):
        expect[int(math.floor(math.sqrt(n) * 20 + 1e-9))] += N * _r3(n) // 2
    assert np.array_equal(H, expect)


def test_histogram_counts_every_pair_once():
    s = synth.uniform_gas(300, 12.0, seed=3, n_types=3)
    s.bin_p, s.bin_q, s.n_bins = 1, 1, 11      # 1 A bins up to 11 A > sqrt(3) * 6
    box = oracle.Box(s)
    H = box.histogram()
    counts = np.bincount(s.type)
    for a in range(3):
        for b in range(a, 3):
            P = counts[a] * (counts[a] - 1) // 2 if a == b else counts[a] * counts[b]
            assert int(H[oracle.pair_index(a, b, 3)].sum()) == P


def test_histogram_brute_force_tiny():
    """Against a direct Python evaluation of every pair with exact integers."""
    s = synth.uniform_gas(40, 6.0, seed=9, n_types=2)
    s.bin_p, s.bin_q, s.n_bins = 1, 4, 16
    box = oracle.Box(s)
    H = box.histogram()
    L = s.L_fx
    E = np.zeros_like(H)
    for i in range(s.n_atoms):
        for j in range(i + 1, s.n_atoms):
            d2 = 0
            for c in range(3):
                d = int(s.xyz[i, c]) - int(s.xyz[j, c])
                d = min(abs(d), L - abs(d))
                d2 += d * d
            k = math.isqrt(d2 * 16 // (S * S))   # (r / 0.25)^2 = 16 d2 / S^2
            if k < 16:
                a, b = sorted((int(s.type[i]), int(s.type[j])))
                E[{(0, 0): 0, (0, 1): 1, (1, 1): 2}[(a, b)], k] += 1
    assert np.array_equal(H, E)


def test_histogram_translation_and_permutation_invariance(small_water):
    s = small_water
    box = oracle.Box(s)
    H = box.histogram()
    rng = np.random.default_rng(1)
    shift = rng.integers(0, s.L_fx, 3)
    xyz2 = ((s.xyz.astype(np.int64) + shift) % s.L_fx).astype(np.int32)
    H2 = oracle.Box(s, xyz=xyz2).histogram()
    assert np.array_equal(H, H2)
    perm = rng.permutation(s.n_atoms)
    s3 = synth.System(**{**s.__dict__, "xyz": s.xyz[perm], "type": s.type[perm]})
    H3 = oracle.Box(s3).histogram()
    assert np.array_equal(H, H3)


def test_histogram_omp_equals_serial(small_water):
    box = oracle.Box(small_water)
    assert np.array_equal(box.histogram(), box.histogram(threads=4))


def test_ideal_gas_g_tends_to_one():
    """Uniform random atoms: g_ab(r) -> 1 within counting noise (reading c7 normalisation)."""
    s = synth.uniform_gas(3000, 30.0, seed=11, n_types=2)
    s.bin_p, s.bin_q, s.n_bins = 1, 2, 28      # 0.5 A bins to 14 A
    box = oracle.Box(s)
    H = box.histogram(threads=4)
    g = box.normalize_g(H)
    for p in range(3):
        sel = slice(4, 28)                     # beyond 2 A
        n = H[p, sel].astype(np.float64)
        err = np.abs(g[p, sel] - 1.0) * np.sqrt(n)
        assert np.all(err < 5.0), (p, err.max())
        assert abs(g[p, sel].mean() - 1.0) < 3.0 / math.sqrt(n.sum()) * 3


# --------------------------------------------------------------------------------------
# Pair energies
# --------------------------------------------------------------------------------------

def _two_type_system(sig=(3.0, 2.0), eps=(0.5, 0.2), q=(1.0, -0.5), ep=False):
    s = synth.uniform_gas(2, 20.0, seed=0, n_types=2)
    s.sigma, s.eps, s.q = list(sig), list(eps), list(q)
    s.bin_p, s.bin_q, s.n_bins = 1, 10, 100
    return s


def test_lj_zero_and_minimum():
    s = _two_type_system(q=(0.0, 0.0))
    box = oracle.Box(s)
    # sigma_00 = 3 A exactly on the grid -> LJ = 0
    assert abs(box.pair_energy(0, 0, (3 * S) ** 2)) < 1e-14
    # Lorentz-Berthelot: sigma_01 = 2.5 A, eps_01 = sqrt(0.1) -> LJ(sigma_01) = 0
    assert abs(box.pair_energy(0, 1, (5 * S // 2) ** 2)) < 1e-14
    # minimum -eps at r = 2^(1/6) sigma
    rmin = 2 ** (1 / 6) * 3.0
    d = int(round(rmin * S))
    assert abs(box.pair_energy(0, 0, d * d) + 0.5) < 1e-9
    assert abs(box.pair_energy(0, 1, int(round(2 ** (1 / 6) * 2.5 * S)) ** 2)
               + math.sqrt(0.1)) < 1e-9
    # r = 2 sigma: 4 eps (2^-12 - 2^-6)
    assert abs(box.pair_energy(0, 0, (6 * S) ** 2) - 4 * 0.5 * (2.0 ** -12 - 2.0 ** -6)) < 1e-15


def test_coulomb_value_and_cutoff_step():
    s = _two_type_system(eps=(0.0, 0.0))
    box = oracle.Box(s)
    ke = oracle.coulomb_constant()
    assert abs(box.pair_energy(0, 1, (4 * S) ** 2) - ke * 1.0 * -0.5 / 4.0) < 1e-12
    rc = 9 * S
    assert abs(box.pair_energy(0, 0, rc * rc - 1) - ke / 9.0) < 1e-9
    assert box.pair_energy(0, 0, rc * rc) == 0.0


def test_ep_table_lookup_is_binwise():
    s = _two_type_system(eps=(0.0, 0.0), q=(0.0, 0.0))
    ep = np.arange(3 * 100, dtype=np.float64).reshape(3, 100) * 0.01
    box = oracle.Box(s, ep=ep)
    # r = 2.05 A -> bin 20 of 0.1 A bins; pair (0,1) -> index 1
    assert box.pair_energy(0, 1, int(2.05 * S) ** 2) == ep[1, 20]
    assert box.pair_energy(1, 1, int(0.55 * S) ** 2) == ep[2, 5]
    assert box.pair_energy(0, 0, (10 * S) ** 2) == 0.0          # beyond the table


def test_lj_cutoff_step():
    """Truncated Lennard-Jones: the uncut value one grid unit inside r_lj, exactly zero at
    r_lj (the exact integer test d^2 < llround(r_lj S)^2), so the step at the cutoff is
    LJ(r_lj); zero r_lj means no cutoff."""
    s = _two_type_system(q=(0.0, 0.0))
    uncut = oracle.Box(s)
    s.r_lj = 5.0
    cut = oracle.Box(s)
    rl = 5 * S
    lj5 = 4 * 0.5 * ((3 / 5) ** 12 - (3 / 5) ** 6)
    assert cut.pair_energy(0, 0, rl * rl - 1) == uncut.pair_energy(0, 0, rl * rl - 1)
    assert abs(cut.pair_energy(0, 0, rl * rl - 1) - lj5) < 1e-12
    assert cut.pair_energy(0, 0, rl * rl) == 0.0
    assert abs(uncut.pair_energy(0, 0, rl * rl) - lj5) < 1e-15
    assert cut.pair_energy(0, 1, (4 * S) ** 2) == uncut.pair_energy(0, 1, (4 * S) ** 2)
    # Coulomb and the cutoff of LJ are independent
    s.q = [1.0, -0.5]
    both = oracle.Box(s)
    ke = oracle.coulomb_constant()
    assert abs(both.pair_energy(0, 0, (6 * S) ** 2) - ke / 6.0) < 1e-12


@pytest.mark.parametrize("which", ["water", "silica"])
def test_delta_u_with_lj_cutoff_equals_total_energy_difference(which):
    """With LJ cut at 4 A (boxes of 10-12 A, so pairs on both sides of the cutoff), dU of a
    move equals the difference of brute-force total energies, and a cutoff beyond every
    minimum-image distance (L sqrt(3)/2) gives the uncut dU exactly."""
    if which == "water":
        s = synth.water_box(40, seed=23, L_A=10.0)
    else:
        s = synth.silica_box(60, seed=24, n_bins=300, bin_p=2, bin_q=100)
    s.r_lj = 4.0
    box = oracle.Box(s)
    s2 = synth.System(**{**s.__dict__, "r_lj": s.L * 0.87})
    far = oracle.Box(s2)
    s3 = synth.System(**{**s.__dict__, "r_lj": 0.0})
    uncut = oracle.Box(s3)
    moved = 0
    for t in range(16):
        mol, trial, u = box.propose(11, t)
        dU, C = box.delta_u(mol, trial)
        U0 = box.total_energy()
        saved = box.xyz.copy()
        box.apply(mol, trial)
        U1 = box.total_energy()
        box.xyz[:] = saved
        assert abs(dU - (U1 - U0)) <= 1e-9 * max(1.0, abs(U0)), (t, dU, U1 - U0)
        assert far.delta_u(mol, trial)[0] == uncut.delta_u(mol, trial)[0]
        moved += dU != uncut.delta_u(mol, trial)[0]
    assert moved > 0               # the cutoff changes some dU


# --------------------------------------------------------------------------------------
# Moves and dU
# --------------------------------------------------------------------------------------

def test_delta_u_equals_total_energy_difference():
    s = synth.water_box(40, seed=21, L_A=10.0)
    box = oracle.Box(s)
    for t in range(12):
        mol, trial, u = box.propose(7, t)
        dU, C = box.delta_u(mol, trial)
        U0 = box.total_energy()
        saved = box.xyz.copy()
        box.apply(mol, trial)
        U1 = box.total_energy()
        box.xyz[:] = saved
        assert abs(dU - (U1 - U0)) <= 1e-9 * max(1.0, abs(U0)), (t, dU, U1 - U0)
        assert C >= abs(dU)


def test_delta_u_with_ep_equals_total_energy_difference():
    s = synth.silica_box(60, seed=22, n_bins=300, bin_p=2, bin_q=100)
    rng = np.random.default_rng(3)
    ep = rng.normal(size=(3, 300))
    box = oracle.Box(s, ep=ep)
    for t in range(12):
        mol, trial, u = box.propose(9, t)
        dU, _ = box.delta_u(mol, trial)
        U0 = box.total_energy()
        saved = box.xyz.copy()
        box.apply(mol, trial)
        U1 = box.total_energy()
        box.xyz[:] = saved
        assert abs(dU - (U1 - U0)) <= 1e-9 * max(1.0, abs(U0))


def test_delta_u_translation_invariance(small_water):
    s = small_water
    box = oracle.Box(s)
    shift = np.array([123456789 % s.L_fx, 777, s.L_fx - 5])
    box2 = oracle.Box(s, xyz=((s.xyz.astype(np.int64) + shift) % s.L_fx).astype(np.int32))
    for t in range(5):
        m1, tr1, u1 = box.propose(3, t)
        m2, tr2, u2 = box2.propose(3, t)
        assert m1 == m2 and u1 == u2
        assert np.array_equal((tr1.astype(np.int64) + shift) % s.L_fx, tr2)
        assert box.delta_u(m1, tr1)[0] == box2.delta_u(m2, tr2)[0]


def test_proposal_geometry(small_water):
    """Rotation keeps intramolecular distances (to grid rounding), the rotation angle is
    at most 5 degrees, and the shift of the centre is at most 0.1 A per axis."""
    s = small_water
    box = oracle.Box(s)
    L = s.L_fx
    M = round(0.1 * S)
    for t in range(200):
        mol, trial, u = box.propose(11, t)
        assert 0 <= mol < s.n_mol and 0.0 <= u < 1.0
        old = s.xyz[3 * mol:3 * mol + 3].astype(np.int64)
        new = trial.astype(np.int64)

        def unwrap(x):
            d = x - x[0]
            d = np.where(2 * d > L, d - L, np.where(2 * d <= -L, d + L, d))
            return d
        uo, un = unwrap(old), unwrap(new)
        for a in range(3):
            for b in range(a + 1, 3):
                do = np.sqrt(((uo[a] - uo[b]) ** 2).sum())
                dn = np.sqrt(((un[a] - un[b]) ** 2).sum())
                assert abs(do - dn) <= 2.0
        co, cn = uo.mean(0), un.mean(0)
        shift = (new[0] - old[0] + cn - co)
        shift = np.where(2 * shift > L, shift - L, np.where(2 * shift <= -L, shift + L, shift))
        assert np.all(np.abs(shift) <= M + 2)
        # rotation angle from the O->H vectors
        vo = (uo[1] - co) / np.linalg.norm(uo[1] - co)
        vn = (un[1] - cn) / np.linalg.norm(un[1] - cn)
        assert math.degrees(math.acos(min(1.0, float(vo @ vn)))) <= 5.0 + 1e-3


def test_zero_potential_accepts_everything():
    s = synth.uniform_gas(50, 10.0, seed=4)
    box = oracle.Box(s)
    att, acc, sdu = box.mc_sweep(500, seed=1)
    assert att == 500 and acc == 500 and sdu == 0.0


def test_metropolis_rule():
    T = 298.0
    kT = oracle.gas_constant() * T
    assert oracle.accept(-1.0, 0.999, T) and oracle.accept(0.0, 0.999, T)
    assert oracle.accept(kT, math.exp(-1.0) - 1e-12, T)
    assert not oracle.accept(kT, math.exp(-1.0) + 1e-12, T)
    assert not oracle.accept(float("nan"), 0.0, T)
    assert not oracle.accept(float("inf"), 0.0, T)


def test_two_atom_boltzmann_distribution():
    """Two LJ atoms in a periodic box sampled by Metropolis: the separation density is
    proportional to r^2 exp(-u(r)/kT) for r < L/2 (chi^2 test over bins)."""
    s = synth.uniform_gas(2, 12.0, seed=2, n_types=1)
    s.sigma, s.eps, s.q = [3.0], [2.5], [0.0]
    s.max_translation = 2.0
    s.temperature = 300.0
    box = oracle.Box(s)
    L = s.L_fx
    edges = np.linspace(2.6, 6.0, 18)
    counts = np.zeros(len(edges) - 1)
    for blk in range(400):
        box.mc_sweep(500, seed=5, move0=blk * 500)
        d = box.xyz[0].astype(np.int64) - box.xyz[1].astype(np.int64)
        d = np.where(2 * d > L, d - L, np.where(2 * d <= -L, d + L, d))
        r = math.sqrt(float((d * d).sum())) / S
        k = np.searchsorted(edges, r) - 1
        if 0 <= k < len(counts):
            counts[k] += 1
    kT = oracle.gas_constant() * 300.0
    r = np.linspace(edges[0], edges[-1], 20001)
    u = 4 * 2.5 * ((3.0 / r) ** 12 - (3.0 / r) ** 6)
    dens = r * r * np.exp(-u / kT)
    expect = np.array([np.trapezoid(dens[(r >= a) & (r <= b)], r[(r >= a) & (r <= b)])
                       for a, b in zip(edges[:-1], edges[1:])])
    expect *= counts.sum() / expect.sum()
    chi2 = float(((counts - expect) ** 2 / np.maximum(expect, 1)).sum())
    assert chi2 < 60.0, (chi2, counts, expect)


# --------------------------------------------------------------------------------------
# Eq. (1): S(Q)
# --------------------------------------------------------------------------------------

def test_sq_flat_background_when_g_is_one(small_water):
    box = oracle.Box(small_water)
    g = np.ones((3, small_water.n_bins))
    Sp, St = oracle.sq_of_box(box, g)
    W, flat = oracle.eq1_weights(small_water)
    assert np.all(Sp == 0.0)
    assert np.all(St == flat)
    c = oracle.concentrations(small_water)
    b = np.asarray(small_water.b) / 10
    assert abs(flat - (c * b * b).sum()) < 1e-15


def test_eq1_weight_identity(small_water):
    """sum_{a<=b} (2 - delta_ab) c_a c_b b_a b_b = (sum_a c_a b_a)^2."""
    for s in (small_water, synth.silica_box(30, seed=1), synth.uniform_gas(30, 9.0, 1, 4)):
        W, flat = oracle.eq1_weights(s)
        c = oracle.concentrations(s)
        b = np.asarray(s.b) / 10
        assert abs(W.sum() - (c * b).sum() ** 2) < 1e-14


def test_poisson_basis_peak_and_closed_form_transform():
    """p_n peaks at r = n s with height 1 (Fig. 1), and the closed-form transform agrees
    with numerical quadrature of 4 pi rho int r^2 p_n sin(Qr)/(Qr) dr."""
    from scipy import integrate
    s_, rho = 0.5, 0.1
    for n in (1, 2, 5, 12, 20):
        r = np.linspace(0.01, 40, 400001)
        p = oracle.poisson_p(n, s_, r)
        assert abs(r[np.argmax(p)] - n * s_) < 1e-3
        assert abs(p.max() - 1.0) < 1e-6
        for Q in (0.3, 1.7, 6.0, 25.0):
            f = lambda x: 4 * math.pi * rho * x * x * oracle.poisson_p(n, s_, np.array([x]))[0] \
                * math.sin(Q * x) / (Q * x)
            num, _ = integrate.quad(f, 0, 80 + 4 * n * s_, limit=2000, epsabs=1e-13)
            cf = oracle.poisson_F(n, s_, np.array([Q]), rho)[0]
            assert abs(num - cf) < 1e-8 * max(1.0, abs(cf)), (n, Q, num, cf)


def test_sq_discrete_transform_matches_closed_form():
    """orc_sq on g - 1 = p_n(r) reproduces the closed-form transform within the
    midpoint-rule error O(dr^2), pinning the sign, scaling and sinc kernel of Eq. 1."""
    s_, rho, n = 0.5, 0.1, 6
    dr, n_bins = 0.005, 4000                          # 20 A, tail of p_6 ~ e^-34
    r = (np.arange(n_bins) + 0.5) * dr
    g = (1.0 + oracle.poisson_p(n, s_, r))[None, :]
    Q = np.array([0.5, 1.0, 3.0, 8.0, 20.0])
    Sp, St = oracle.sq(g, dr, Q, np.array([4 * math.pi * rho]), 1, np.array([0.25]))
    cf = oracle.poisson_F(n, s_, Q, rho)
    assert np.all(np.abs(Sp[0] - cf) < 2e-5 * np.abs(cf).max())
    assert np.all(np.abs(St[0] - 0.25 - cf) < 2e-5 * np.abs(cf).max())


def test_sq_high_q_limit(small_water):
    """S(Q) -> flat background at large Q for a smooth g (here the ideal-gas g)."""
    s = synth.uniform_gas(2000, 26.0, seed=12, n_types=2)
    s.bin_p, s.bin_q, s.n_bins = 1, 10, 120
    box = oracle.Box(s)
    g = box.normalize_g(box.histogram(threads=4))
    Sp, St = oracle.sq_of_box(box, g, Q=np.array([80.0, 120.0]))
    W, flat = oracle.eq1_weights(s)
    assert np.all(np.abs(St - flat) < 0.02)


# --------------------------------------------------------------------------------------
# Empirical potential fit
# --------------------------------------------------------------------------------------

def test_ep_fit_recovers_coefficients_and_table():
    rng = np.random.default_rng(8)
    Q = 0.3 + np.arange(2000) * (39.7 / 1999)
    F = oracle.ep_basis_matrix(20, 0.5, Q, 0.1)
    C_true = rng.normal(size=(3, 20))
    dSp = C_true @ F.T
    C_fit = oracle.ep_fit(dSp, F)
    assert np.abs(C_fit - C_true).max() < 1e-6 * np.abs(C_true).max()
    tab = oracle.ep_table(C_true, 0.5, 600, 0.02, alpha=1.0, kT=2.5)
    r = (np.arange(600) + 0.5) * 0.02
    direct = -2.5 * sum(C_true[:, n - 1:n] * oracle.poisson_p(n, 0.5, r)[None, :]
                        for n in range(1, 21))
    assert np.allclose(tab, direct, rtol=0, atol=1e-12)


def test_pair_resolve_inverts_square_weights():
    rng = np.random.default_rng(2)
    w = rng.uniform(0.1, 1.0, (3, 3))
    dSp = rng.normal(size=(3, 50))
    assert np.allclose(oracle.pair_resolve(w @ dSp, w), dSp, atol=1e-10)


# --------------------------------------------------------------------------------------
# Smeared histogram and its adjoint
# --------------------------------------------------------------------------------------

def test_smeared_weights_conserve_counts_and_reduce_to_histogram():
    s = synth.uniform_gas(400, 14.0, seed=13, n_types=2)
    s.bin_p, s.bin_q, s.n_bins = 1, 20, 130           # 0.05 A bins to 6.5 A
    box = oracle.Box(s)
    H = box.histogram().astype(np.float64)
    Ht_tiny = box.smeared_hist(1e-7)
    assert np.abs(Ht_tiny - H).max() <= 2.0             # only pairs within 5e-7 A of an edge
    Ht = box.smeared_hist(0.05)
    # pairs well inside [5 sigma, r_max - 5 sigma] keep their unit mass
    inner = slice(10, 120)
    assert abs(Ht[:, inner].sum() - H[:, inner].sum()) < 0.02 * H[:, inner].sum() ** 0.5 + 3


def test_smeared_gradient_matches_finite_differences():
    s = synth.water_box(30, seed=31, L_A=9.0, n_bins=100, bin_p=5, bin_q=100)
    box = oracle.Box(s)
    rng = np.random.default_rng(4)
    lam = rng.normal(size=(3, 100))
    # sigma = 0.047 keeps the rigid O-H (1.0 A) and H-H distances away from the kinks of
    # the +-5 sigma truncation (bin edge +- 5 sigma), where one-sided derivatives differ
    # by phi(5) lambda / sigma and a central difference straddling one is off by half that.
    sigma = 0.047
    grad = box.smeared_grad(sigma, lam)
    h = 105                                            # ~1.0014e-4 A
    # tolerance relative to the scale of the gradient: components that nearly cancel
    # still carry the O(h^2) and truncation-kink errors of the difference quotient
    tol = 1e-5 * np.abs(grad).max()
    for i in rng.choice(s.n_atoms, 12, replace=False):
        for c in range(3):
            xp = box.xyz.copy(); xp[i, c] = (xp[i, c] + h) % s.L_fx
            xm = box.xyz.copy(); xm[i, c] = (xm[i, c] - h) % s.L_fx
            fp = (lam * oracle.Box(s, xyz=xp).smeared_hist(sigma)).sum()
            fm = (lam * oracle.Box(s, xyz=xm).smeared_hist(sigma)).sum()
            fd = (fp - fm) / (2 * h / S)
            assert abs(fd - grad[i, c]) <= tol, (i, c, fd, grad[i, c])


def test_chi2_gradients_match_finite_differences():
    s = synth.water_box(30, seed=32, L_A=9.0, n_bins=100, bin_p=5, bin_q=100)
    s.Q = 0.5 + np.arange(60) * 0.25
    box = oracle.Box(s)
    rng = np.random.default_rng(5)
    target = rng.normal(size=60) * 0.05
    C_ = rng.normal(size=(3, 4)) * 0.01
    sigma = 0.047                                      # away from truncation kinks
    chi2, dC, gx, _, _ = oracle.chi2_and_grads(box, sigma, s.Q, target, C_, 0.5)
    eps = 1e-6
    for p in range(3):
        for n in range(4):
            Cp = C_.copy(); Cp[p, n] += eps
            Cm = C_.copy(); Cm[p, n] -= eps
            fp = oracle.chi2_and_grads(box, sigma, s.Q, target, Cp, 0.5)[0]
            fm = oracle.chi2_and_grads(box, sigma, s.Q, target, Cm, 0.5)[0]
            assert abs((fp - fm) / (2 * eps) - dC[p, n]) < 1e-6 * max(1.0, abs(dC[p, n]))
    h = 105
    tol = 1e-5 * np.abs(gx).max()
    for i in (0, 7, 44):
        for c in range(3):
            xp = box.xyz.copy(); xp[i, c] = (xp[i, c] + h) % s.L_fx
            xm = box.xyz.copy(); xm[i, c] = (xm[i, c] - h) % s.L_fx
            fp = oracle.chi2_and_grads(oracle.Box(s, xyz=xp), sigma, s.Q, target, C_, 0.5)[0]
            fm = oracle.chi2_and_grads(oracle.Box(s, xyz=xm), sigma, s.Q, target, C_, 0.5)[0]
            fd = (fp - fm) / (2 * h / S)
            assert abs(fd - gx[i, c]) <= tol, (i, c, fd, gx[i, c])


def test_rotation_matrix_against_scipy():
    """The fixed-point rotation matrix of the move (quaternion (1, v)/|(1, v)|) equals the
    rotation SciPy builds from the same quaternion, to the 2^-30 rounding."""
    import ctypes as C
    Rotation = pytest.importorskip("scipy.spatial.transform").Rotation
    L = oracle.lib()
    L.orc_rotation_fixed.argtypes = [C.c_double, C.c_double, C.c_double, C.POINTER(C.c_int32)]
    rng = np.random.default_rng(17)
    for _ in range(200):
        v = rng.uniform(-0.3, 0.3, 3)
        Rq = np.zeros(9, np.int32)
        L.orc_rotation_fixed(v[0], v[1], v[2], Rq.ctypes.data_as(C.POINTER(C.c_int32)))
        ref = Rotation.from_quat([v[0], v[1], v[2], 1.0]).as_matrix()   # scalar-last
        assert np.abs(Rq.reshape(3, 3) / 2.0 ** 30 - ref).max() <= 2.0 ** -30 + 1e-15


# --------------------------------------------------------------------------------------
# flexible molecules (Sec. 3.1: springs between every two atoms; three kinds of moves)
# --------------------------------------------------------------------------------------

def _one_molecule(xyz_A, k=2000.0, L_A=20.0):
    """A single flexible water molecule (O, H, H) at the given positions (A)."""
    s = synth.flexible_water_box(1, seed=0, L_A=L_A, k_spring=k)
    s.xyz = np.rint(np.asarray(xyz_A) * S).astype(np.int32) % s.L_fx
    return s


def test_intra_energy_scales_quadratically():
    """Scaling the reference geometry by lambda about O scales every distance: the spring
    energy is (lambda - 1)^2 k (d_OH^2 + d_OH^2 + d_HH^2), zero at lambda = 1."""
    g = synth.water_geometry_A() + 5.0
    d_hh = 2.0 * 0.8164904309201172
    for lam in (1.0, 1.01, 0.97, 1.05):
        xyz = g[0] + lam * (g - g[0])
        box = oracle.Box(_one_molecule(xyz))
        expect = (lam - 1.0) ** 2 * 2000.0 * (1.0 + 1.0 + d_hh * d_hh)
        assert abs(box.total_energy() - expect) <= 1e-3 * max(expect, 1e-3), (lam, box.total_energy(), expect)


def test_flexible_delta_u_equals_total_energy_difference():
    s = synth.flexible_water_box(60, seed=3, L_A=12.0)
    box = oracle.Box(s)
    for t in range(60):
        mol, trial, u = box.propose(7, t)
        dU, C = box.delta_u(mol, trial)
        U0 = box.total_energy()
        saved = box.xyz.copy()
        box.apply(mol, trial)
        U1 = box.total_energy()
        box.xyz[:] = saved
        assert abs(dU - (U1 - U0)) <= 1e-9 * max(1.0, abs(U0)), (t, dU, U1 - U0)
        assert C >= abs(dU) - 1e-12


def test_flexible_move_kinds():
    """Each move is one of: all atoms shifted by one vector, a rotation (every atom moves,
    the centre stays within grid rounding), or exactly one atom shifted; the three kinds
    occur about equally often."""
    s = synth.flexible_water_box(50, seed=4, L_A=12.0)
    box = oracle.Box(s)
    L = s.L_fx
    seen = {"translate": 0, "rotate": 0, "atom": 0}
    for t in range(1500):
        mol, trial, u = box.propose(13, t)
        old = s.xyz[3 * mol:3 * mol + 3].astype(np.int64)
        d = trial.astype(np.int64) - old
        d = np.where(2 * d > L, d - L, np.where(2 * d <= -L, d + L, d))
        moved = (d != 0).any(axis=1)
        if moved.sum() <= 1:
            seen["atom"] += 1
            assert np.abs(d).max() <= round(0.1 * S)
        elif (d == d[0]).all():
            seen["translate"] += 1
        else:
            seen["rotate"] += 1
            assert np.abs(d.mean(axis=0)).max() <= 2
    for k, v in seen.items():
        assert abs(v - 500) < 4 * math.sqrt(1500 * (1 / 3) * (2 / 3)), seen


def test_spring_boltzmann_distribution():
    """One flexible two-atom molecule (no non-bonded terms) sampled by Metropolis: the bond
    length density is proportional to r^2 exp(-k (r - d)^2 / kT) (chi^2 test over bins)."""
    k = 200.0
    base = synth.flexible_water_box(1, seed=0, L_A=30.0, k_spring=k)
    s = synth.System(**{**base.__dict__,
                        "xyz": (np.rint(np.array([[5.0, 5.0, 5.0], [6.0, 5.0, 5.0]]) * S)).astype(np.int32),
                        "type": np.array([0, 1], np.int32), "mol_start": np.array([0, 2], np.int64),
                        "q": [0.0, 0.0], "eps": [0.0, 0.0], "temperature": 300.0})
    box = oracle.Box(s)
    L = s.L_fx
    edges = np.linspace(0.75, 1.25, 16)
    counts = np.zeros(len(edges) - 1)
    for blk in range(600):
        box.mc_sweep(60, seed=9, move0=blk * 60)
        d = box.xyz[1].astype(np.int64) - box.xyz[0].astype(np.int64)
        d = np.where(2 * d > L, d - L, np.where(2 * d <= -L, d + L, d))
        r = math.sqrt(float((d * d).sum())) / S
        j = np.searchsorted(edges, r) - 1
        if 0 <= j < len(counts):
            counts[j] += 1
    kT = oracle.gas_constant() * 300.0
    r = np.linspace(edges[0], edges[-1], 20001)
    dens = r * r * np.exp(-k * (r - 1.0) ** 2 / kT)
    expect = np.array([np.trapezoid(dens[(r >= a) & (r <= b)], r[(r >= a) & (r <= b)])
                       for a, b in zip(edges[:-1], edges[1:])])
    expect *= counts.sum() / expect.sum()
    chi2 = float(((counts - expect) ** 2 / np.maximum(expect, 1)).sum())
    assert chi2 < 50.0, (chi2, counts, expect)


# --------------------------------------------------------------------------------------
# Pair resolution with gamma > 0 (reading c16), the smeared g~ normalisation and the
# chi^2 value of the differentiable form (reading c15)
# --------------------------------------------------------------------------------------

@pytest.mark.parametrize("n_data,P", [(1, 3), (2, 3), (3, 6), (5, 3)])
def test_pair_resolve_with_gamma_solves_the_regularised_normal_equations(n_data, P):
    """The pseudo-inverse of [w; gamma I] applied to [dS; 0] minimises
    ||w x - dS||^2 + gamma^2 ||x||^2, so x solves (w^T w + gamma^2 I) x = w^T dS. A wrong
    right-hand side of the stacked rows or gamma in place of gamma^2 fails this."""
    rng = np.random.default_rng(10 * n_data + P)
    w = rng.uniform(0.05, 1.0, (n_data, P))
    dS = rng.normal(size=(n_data, 40))
    for gamma in (0.3, 1.0, 2.5):
        x = oracle.pair_resolve(dS, w, gamma)
        assert x.shape == (P, 40)
        lhs = (w.T @ w + gamma * gamma * np.eye(P)) @ x
        assert np.allclose(lhs, w.T @ dS, rtol=0, atol=1e-12 * np.abs(w.T @ dS).max())


def test_pair_resolve_with_gamma_scalar_closed_form_and_small_gamma_limit():
    # one dataset, one pair: x = w dS / (w^2 + gamma^2)
    dS = np.array([[0.7, -1.3, 2.0]])
    for wv, gamma in ((0.4, 1.0), (2.0, 0.5)):
        x = oracle.pair_resolve(dS, np.array([[wv]]), gamma)
        assert np.allclose(x, wv * dS / (wv * wv + gamma * gamma), rtol=1e-14, atol=0)
    # square, well-conditioned w: gamma -> 0 approaches the exact inverse
    rng = np.random.default_rng(3)
    w = np.eye(3) + rng.uniform(-0.2, 0.2, (3, 3))
    dSp = rng.normal(size=(3, 20))
    for gamma, tol in ((1e-2, 1e-3), (1e-4, 1e-7)):
        x = oracle.pair_resolve(w @ dSp, w, gamma)
        assert np.abs(x - dSp).max() < tol * np.abs(dSp).max()


def test_smeared_g_of_integer_counts_equals_normalize_g(small_water):
    """g~ applies the normalisation of g (reading c7) to real-valued counts: on an integer
    histogram it equals the C oracle's g (P_aa = N_a (N_a - 1) / 2 there), and the factor it
    returns is the one that multiplies the counts."""
    ob = oracle.Box(small_water)
    H = ob.histogram()
    g_ref = ob.normalize_g(H)
    g, fac = oracle.smeared_g(ob, H.astype(np.float64))
    assert np.allclose(g, g_ref, rtol=1e-12, atol=0)   # rounding order of the shell volume
    assert np.allclose(g, H * fac, rtol=1e-15, atol=0)


def test_chi2_value_against_eq1_and_the_ep_image():
    """The chi^2 value: with C = 0 and the target equal to the Eq. (1) S~ of g~ (orc_sq on
    the smeared g~), chi^2 = 0; one planted coefficient C_pn adds the image W_p C_pn F_n(Q),
    so chi^2 = (W_p C_pn)^2 sum_Q F_n(Q)^2 (F_n the closed-form Poisson transform)."""
    s = synth.water_box(30, seed=33, L_A=9.0, n_bins=100, bin_p=5, bin_q=100)
    Q = 0.5 + np.arange(60) * 0.25
    box = oracle.Box(s)
    sigma = 0.05
    W, flat = oracle.eq1_weights(s)
    rho = oracle.number_density(s)
    g, _ = oracle.smeared_g(box, box.smeared_hist(sigma))
    _, St = oracle.sq(g, s.dr, Q, 4.0 * math.pi * rho * W, 3, np.array([flat]))
    C0 = np.zeros((3, 4))
    chi2, dC, _, S_t, _ = oracle.chi2_and_grads(box, sigma, Q, St[0], C0, 0.5)
    assert np.array_equal(S_t, St[0])
    assert chi2 < 1e-24 and np.abs(dC).max() < 1e-12
    for p, n, c in ((0, 1, 0.3), (2, 3, -0.05), (1, 4, 1.2)):
        Cp = C0.copy()
        Cp[p, n - 1] = c
        chi2p = oracle.chi2_and_grads(box, sigma, Q, St[0], Cp, 0.5)[0]
        Fn = oracle.poisson_F(n, 0.5, Q, rho)
        assert abs(chi2p - (W[p] * c) ** 2 * (Fn * Fn).sum()) <= 1e-12 * chi2p


# --------------------------------------------------------------------------------------
# The refinement loop (Sec. 2.2 items III-VI, Eq. 2)
# --------------------------------------------------------------------------------------

def _lj_target(amp=1.5, r0=4.5, width=0.4, n_conf=8):
    """S(Q) of a Lennard-Jones liquid whose O(1 kT) potential has a planted repulsive bump
    amp exp(-((r - r0)/width)^2), equilibrated and averaged over n_conf configurations on the
    oracle; returns (target S, the bump table, Eq. (1) weights, flat)."""
    s = synth.lj_fluid(10, seed=52)
    r = (np.arange(s.n_bins) + 0.5) * s.dr
    bump = np.zeros((1, s.n_bins))
    bump[0] = amp * np.exp(-((r - r0) / width) ** 2)
    o = oracle.Box(s, ep=bump)
    o.mc_sweep(20000, seed=52)
    H = None
    for k in range(n_conf):
        o.mc_sweep(2000, seed=52, move0=20000 + 2000 * k)
        h = o.histogram()
        H = h if H is None else H + h
    W, flat = oracle.eq1_weights(s)
    rho = oracle.number_density(s)
    _, St = oracle.sq(o.normalize_g(H, n_conf), s.dr, s.Q, 4.0 * math.pi * rho * W, 1, np.array([flat]))
    return St[0], bump, W, flat


def test_refine_loop_learns_a_planted_potential():
    """The loop in the paper's order (moves, histogram, Eq. (1), Delta S = target - S, Poisson
    fit, U_EP += -alpha kT sum C p_n) against a target simulated with a planted repulsive bump:
    chi^2 falls to under half its first value within six passes and the learned potential is
    repulsive where the bump is. A wrong sign of the update (reading c13) or of Delta S makes
    chi^2 grow instead."""
    target, bump, W, flat = _lj_target()
    s = synth.lj_fluid(10, seed=51)
    ob = oracle.Box(s)
    ob.mc_sweep(20000, seed=51)
    chi = []
    for it in range(6):
        r = oracle.refine_pass(ob, target[None, :], W[None, :], np.array([flat]), s.Q, 20, 0.5, 0.0, 1.0,
                               moves=4000, seed=9, move0=10**6 + 4000 * it)
        chi.append(r["chi2"])
    k = int(4.5 / s.dr)
    assert chi[-1] < 0.5 * chi[0], chi
    assert r["ep"][0][k] > 0.3 * bump[0][k], r["ep"][0][k]
