"""Pins of the FP64 oracle to things other than itself (CPU only).

Each test checks the oracle against a fact that the paper or the mathematics
fixes: published known-answer vectors of the generator, a library matrix
exponential, the closed-form unmonitored evolution, a brute-force many-body
state vector driven by the same draws, and exact invariants.
"""
import os

import numpy as np
import pytest
import scipy.linalg

from oracle import lattice, observables, philox, trajectory
from oracle.trajectory import HOMODYNE, PROJECTIVE, Params
from tests import brute

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------- generator

def test_philox_known_answers():
    rows = [l.split() for l in open(os.path.join(GOLDEN, "philox4x32_10_kat.txt"))
            if l.strip() and not l.startswith("#")]
    assert len(rows) == 3
    for r in rows:
        v = [int(x, 16) for x in r]
        out = philox.philox4x32_10(v[0:4], v[4:6])
        assert [int(o) for o in out] == v[6:10]


def test_uniform53_is_the_53_bit_grid():
    """u = k 2^-53 with k the 27 high bits of the first word over the 26 high bits of the
    second: every value on the 53-bit grid of [0, 1) is reachable, 0 and 1 - 2^-53 at the ends,
    and the low bits of the words do not matter."""
    top = np.uint64(0xFFFFFFFF)
    assert philox.uniform53(0, 0) == 0.0
    assert philox.uniform53(top, top) == 1.0 - 2.0 ** -53
    assert philox.uniform53(0, 1 << 6) == 2.0 ** -53                 # lowest bit kept from wb
    assert philox.uniform53(0, (1 << 6) - 1) == 0.0                  # the 6 bits below are dropped
    assert philox.uniform53(1 << 5, 0) == 2.0 ** -27                 # lowest bit kept from wa
    assert philox.uniform53((1 << 5) - 1, 0) == 0.0
    assert philox.uniform53(1 << 31, 0) == 0.5
    ks = np.array([0x12345678, 0xDEADBEEF], dtype=np.uint64)
    u = philox.uniform53(ks[0], ks[1])
    assert u * 2.0 ** 53 == float((0x12345678 >> 5) * (1 << 26) + (0xDEADBEEF >> 6))


def test_uniform_and_normal_draws():
    u_sel, u_out = philox.measure_draws(seed=12345, traj_id=7, step=3, L=200000)
    for u in (u_sel, u_out):
        assert u.min() >= 0.0 and u.max() < 1.0
        assert abs(u.mean() - 0.5) < 4 * np.sqrt(1 / 12 / u.size)
        assert abs(u.var() - 1 / 12) < 0.002
    assert abs(np.corrcoef(u_sel, u_out)[0, 1]) < 0.01
    xi = philox.noise_normals(seed=12345, traj_id=7, step=3, L=200000)
    assert abs(xi.mean()) < 4 / np.sqrt(xi.size)
    assert abs(xi.var() - 1.0) < 0.015
    assert abs(np.mean(xi ** 4) - 3.0) < 0.06          # Gaussian kurtosis
    # distinct steps / trajectories / tags give distinct streams
    a = philox.noise_normals(1, 0, 0, 64)
    assert not np.allclose(a, philox.noise_normals(1, 0, 1, 64))
    assert not np.allclose(a, philox.noise_normals(1, 1, 0, 64))
    # 64-bit trajectory ids use the high counter bits
    assert not np.allclose(philox.noise_normals(1, 5, 0, 64), philox.noise_normals(1, 5 + (1 << 32), 0, 64))


# ---------------------------------------------------------------- propagator

@pytest.mark.parametrize("Lx,Ly", [(2, 1), (3, 1), (8, 1), (17, 1), (64, 1), (4, 4), (4, 6), (6, 3)])
def test_propagator_is_expm_of_hopping(Lx, Ly):
    dt = 0.05
    H = lattice.hopping_matrix(Lx, Ly, 1.0)
    P = lattice.propagator(Lx, Ly, 1.0, dt)
    ref = scipy.linalg.expm(-1j * dt * H)
    assert np.max(np.abs(P - ref)) < 1e-13


def test_hopping_matrix_bonds():
    H = lattice.hopping_matrix(6, 1, 1.0)
    assert H[0, 1] == 1.0 and H[0, 5] == 1.0 and H[0, 2] == 0.0 and np.allclose(H, H.T)
    H2 = lattice.hopping_matrix(4, 3, 1.0)
    # site (1, 2) = 9 neighbours (0,2)=8, (2,2)=10, (1,1)=5, (1,0)=1
    assert sorted(np.nonzero(H2[9])[0].tolist()) == [1, 5, 8, 10]


def test_propagator_unitary_and_semigroup():
    P = lattice.propagator(32, 1, 1.0, 0.05)
    assert np.max(np.abs(P @ P.conj().T - np.eye(32))) < 1e-14
    P5 = lattice.propagator(32, 1, 1.0, 0.25)
    assert np.max(np.abs(np.linalg.matrix_power(P, 5) - P5)) < 1e-13


# ---------------------------------------------------------------- gamma = 0

def _neel_density_closed_form(Lx, Ly, J, t):
    """Unmonitored n_i(t) from the Neel / checkerboard start (derived in plane waves).

    n_i(t) = 1/2 + 1/2 (-1)^{x+y} (1/L) sum_k cos(2 eps_k t), eps_k = 2J(cos kx + cos ky),
    because eps_{k + (pi, pi)} = -eps_k.
    """
    kx = 2 * np.pi * np.arange(Lx) / Lx
    if Ly == 1:
        eps = 2 * J * np.cos(kx)
        stag = (-1.0) ** np.arange(Lx)
    else:
        ky = 2 * np.pi * np.arange(Ly) / Ly
        eps = (2 * J * (np.cos(kx)[None, :] + np.cos(ky)[:, None])).ravel()
        stag = np.array([(-1.0) ** (x + y) for y in range(Ly) for x in range(Lx)])
    return 0.5 + 0.5 * stag * np.mean(np.cos(2 * eps * t))


@pytest.mark.parametrize("Lx,Ly,nsteps", [(64, 1, 200), (1024, 1, 30), (8, 6, 60)])
def test_unmonitored_density_closed_form(Lx, Ly, nsteps):
    prm = Params(Lx=Lx, Ly=Ly, gamma=0.0, protocol=PROJECTIVE, reorth_interval=10)
    out = trajectory.run(prm, nsteps)
    n = trajectory.occupations(out["U"])
    ref = _neel_density_closed_form(Lx, Ly, 1.0, nsteps * prm.dt)
    assert np.max(np.abs(n - ref)) < 1e-12
    assert len(out["events"]) == 0


# ---------------------------------------------------------------- brute force

def _brute_setup(prm):
    L = prm.L
    occ = lattice.occupied_sites(prm.Lx, prm.Ly)
    sec = brute.Sector(L, len(occ))
    bonds = brute.ring_bonds(L) if prm.Ly == 1 else brute.torus_bonds(prm.Lx, prm.Ly)
    E = brute.evolution_operator(sec, bonds, prm.J, prm.dt)
    psi = np.zeros(sec.dim, dtype=np.complex128)
    psi[sec.index[sum(1 << int(i) for i in occ)]] = 1.0
    return sec, E, psi


def _compare_projective(prm, nsteps, oracle_step=trajectory.step):
    """Run oracle and brute force side by side; returns worst |C - conj(D)| and events."""
    sec, E, psi = _brute_setup(prm)
    U = lattice.initial_orbitals(prm.Lx, prm.Ly)
    P = lattice.propagator(prm.Lx, prm.Ly, prm.J, prm.dt)
    worst, all_events = 0.0, []
    for s in range(nsteps):
        U, events = oracle_step(U, P, prm, s)
        psi = E @ psi
        for (j, u, p, outcome) in events:
            psi_try, w1 = sec.project(psi, j, 1)
            assert abs(w1 - p) < 1e-11, (s, j, w1, p)
            assert outcome == (1 if u < w1 else 0)
            psi, _ = sec.project(psi, j, outcome)
        all_events.extend(events)
        D = sec.d_matrix(psi)
        worst = max(worst, np.max(np.abs(observables.correlation(U) - np.conj(D))))
    return worst, all_events, U, psi, sec


@pytest.mark.parametrize("Lx,Ly,gamma,seed", [(8, 1, 2.0, 11), (10, 1, 1.0, 5), (4, 3, 3.0, 2)])
def test_projective_matches_brute_force(Lx, Ly, gamma, seed):
    prm = Params(Lx=Lx, Ly=Ly, gamma=gamma, protocol=PROJECTIVE, reorth_interval=3, seed=seed, traj_id=1)
    worst, events, U, psi, sec = _compare_projective(prm, 40)
    assert worst < 1e-12
    outcomes = {e[3] for e in events}
    assert len(events) >= 10 and outcomes == {0, 1}
    # entropies of contiguous and non-contiguous subsystems vs Schmidt values
    L = prm.L
    for A in ([0, 1, 2], list(range(L // 2)), [0, 2, 5], [1, L - 1]):
        assert abs(observables.entanglement_entropy(U, A) - sec.entropy(psi, A)) < 1e-11


def _compare_homodyne(prm, nsteps, weight=trajectory.homodyne_weight):
    sec, E, psi = _brute_setup(prm)
    U = lattice.initial_orbitals(prm.Lx, prm.Ly)
    P = lattice.propagator(prm.Lx, prm.Ly, prm.J, prm.dt)
    worst = 0.0
    for s in range(nsteps):
        xi = philox.noise_normals(prm.seed, prm.traj_id, s, prm.L)
        U = trajectory.orthonormalize(weight(P @ U, xi, prm.gamma, prm.dt))
        psi = E @ psi
        n = sec.occupation(psi)
        m = np.sqrt(prm.gamma * prm.dt) * xi + (2 * n - 1) * prm.gamma * prm.dt
        psi = sec.weight(psi, m)
        worst = max(worst, np.max(np.abs(observables.correlation(U) - np.conj(sec.d_matrix(psi)))))
    return worst, U, psi, sec


@pytest.mark.parametrize("Lx,Ly,gamma", [(8, 1, 1.0), (10, 1, 0.3), (4, 2, 2.0)])
def test_homodyne_matches_brute_force(Lx, Ly, gamma):
    prm = Params(Lx=Lx, Ly=Ly, gamma=gamma, protocol=HOMODYNE, seed=99, traj_id=3)
    worst, U, psi, sec = _compare_homodyne(prm, 30)
    assert worst < 1e-12
    # the oracle's own step() follows the same sequence
    out = trajectory.run(prm, 30)
    assert np.max(np.abs(observables.correlation(out["U"]) - observables.correlation(U))) < 1e-13
    L = prm.L
    A, B = [0, 1], [4, 5]
    I_brute = sec.entropy(psi, A) + sec.entropy(psi, B) - sec.entropy(psi, A + B)
    assert abs(observables.mutual_information(U, A, B) - I_brute) < 1e-11
    assert abs(observables.entanglement_entropy(U, list(range(L // 2))) - sec.entropy(psi, list(range(L // 2)))) < 1e-11


# ---------------------------------------------------------------- Eqs. (A1), (A2)

def _random_state(L, N, seed):
    rng = np.random.default_rng(seed)
    Z = rng.standard_normal((L, N)) + 1j * rng.standard_normal((L, N))
    return np.linalg.qr(Z)[0]


def test_rank1_updates_equal_correlation_matrix_equations():
    """The U-form updates reproduce Eq. (A1) (click) and Eq. (A2) with '+' (no click)."""
    U = _random_state(12, 5, 0)
    C = observables.correlation(U)
    j = 4
    p = C[j, j].real
    # Eq. (A1): C'_ab = C_ab - C_aj C_jb / C_jj off row/column j, C'_jj = 1
    C1 = C - np.outer(C[:, j], C[j, :]) / p
    C1[j, :] = 0.0; C1[:, j] = 0.0; C1[j, j] = 1.0
    U1 = trajectory.project_site(U, j, 1)
    assert np.max(np.abs(observables.correlation(U1) - C1)) < 1e-13
    # Eq. (A2) read with '+': C'_ab = C_ab + C_aj C_jb / (1 - C_jj), row/column j zero
    C0 = C + np.outer(C[:, j], C[j, :]) / (1 - p)
    C0[j, :] = 0.0; C0[:, j] = 0.0
    U0 = trajectory.project_site(U, j, 0)
    assert np.max(np.abs(observables.correlation(U0) - C0)) < 1e-13
    # the sign printed in Eq. (A2) ('-') does not conserve the particle number
    Cm = C - np.outer(C[:, j], C[j, :]) / (1 - p)
    Cm[j, :] = 0.0; Cm[:, j] = 0.0
    assert abs(np.trace(Cm).real - 5) > 1e-3
    assert abs(np.trace(C0).real - 5) < 1e-12


# ---------------------------------------------------------------- invariants

def test_invariants_along_a_projective_trajectory():
    prm = Params(Lx=64, gamma=0.5, protocol=PROJECTIVE, reorth_interval=1, seed=3)
    out = trajectory.run(prm, 60)
    U = out["U"]
    N = U.shape[1]
    assert np.max(np.abs(U.conj().T @ U - np.eye(N))) < 1e-13
    C = observables.correlation(U)
    assert abs(np.trace(C).real - N) < 1e-12
    assert np.max(np.abs(C @ C - C)) < 1e-13
    A = list(range(20))
    Abar = list(range(20, 64))
    assert abs(observables.entanglement_entropy(U, A) - observables.entanglement_entropy(U, Abar)) < 1e-10
    I = observables.mutual_information(U, list(range(10)), list(range(30, 40)))
    assert I >= -1e-12
    I_comp = observables.mutual_information(U, A, Abar)
    assert abs(I_comp - 2 * observables.entanglement_entropy(U, A)) < 1e-10


def test_neel_has_zero_entropy_and_click_makes_c_diagonal():
    U0 = lattice.initial_orbitals(16)
    assert observables.entanglement_entropy(U0, list(range(8))) == 0.0
    U = _random_state(16, 8, 5)
    U1 = trajectory.project_site(U, 3, 1)
    C = observables.correlation(U1)
    assert abs(C[3, 3] - 1) < 1e-13
    assert np.max(np.abs(np.delete(C[3], 3))) < 1e-13
    U0_ = trajectory.project_site(U, 3, 0)
    assert np.max(np.abs(observables.correlation(U0_)[3])) < 1e-13


def test_entropy_of_half_filled_random_state_matches_schmidt():
    L, N = 10, 5
    U = _random_state(L, N, 8)
    sec = brute.Sector(L, N)
    psi = sec.from_orbitals(U)
    assert abs(np.linalg.norm(psi) - 1) < 1e-12
    assert np.max(np.abs(observables.correlation(U) - np.conj(sec.d_matrix(psi)))) < 1e-13
    for A in ([0, 1, 2, 3, 4], [0, 3, 7], [2, 9]):
        assert abs(observables.entanglement_entropy(U, A) - sec.entropy(psi, A)) < 1e-11


@pytest.mark.parametrize("Lx,Ly,N", [(10, 1, 5), (4, 3, 6)])
def test_density_correlations_match_occupation_statistics(Lx, Ly, N):
    """Eq. (2) and Eq. (GAB) against the joint occupation statistics of the brute-force
    state: cov(n_i, n_j) = <n_i n_j> - <n_i><n_j> summed from |psi|^2 over the basis."""
    L = Lx * Ly
    U = _random_state(L, N, 11 + L)
    sec = brute.Sector(L, N)
    prob = np.abs(sec.from_orbitals(U)) ** 2
    occ = sec.occ                                           # basis states x sites, 0/1
    mean = occ.T @ prob
    cov = (occ * prob[:, None]).T @ occ - np.outer(mean, mean)
    c = observables.displacement_correlation(U, Lx, Ly)
    x, y = np.arange(L) % Lx, np.arange(L) // Lx
    for dy in range(Ly):
        for dx in range(Lx):
            d = dx + Lx * dy
            if d == 0:
                assert c[0] == 0.0
                continue
            j = (x + dx) % Lx + Lx * ((y + dy) % Ly)
            assert abs(c[d] - np.mean(cov[np.arange(L), j])) < 1e-13, (dx, dy)
    A, B = [0, 1, L // 2], [L // 2 + 1, L - 1]
    NA, NB = occ[:, A].sum(axis=1), occ[:, B].sum(axis=1)
    covAB = np.sum(prob * NA * NB) - np.sum(prob * NA) * np.sum(prob * NB)
    assert abs(observables.particle_covariance(U, A, B) + covAB) < 1e-13
    with pytest.raises(ValueError):
        observables.particle_covariance(U, A, [0])


def test_density_correlation_sum_rule_and_ring_symmetry():
    """C^2 = C gives sum_j |C_ij|^2 = C_ii, so -sum_{d != 0} c[d] = mean_i n_i (1 - n_i);
    on the ring c[d] = c[L - d]."""
    L = 64
    U = _random_state(L, L // 2, 21)
    c = observables.displacement_correlation(U, L)
    n = np.real(np.diag(observables.correlation(U)))
    assert abs(-np.sum(c) - np.mean(n * (1 - n))) < 1e-13
    assert np.max(np.abs(c[1:] - c[1:][::-1])) < 1e-15


def test_rk4_step_is_the_quartic_taylor_polynomial_and_close_to_expm():
    """For the constant A of a step, RK4 equals sum_{k<=4} (A dt)^k / k! applied to U
    (written here from the series, not from the stages), and differs from
    expm(A dt) U by at most the series remainder."""
    L, N, dt, gamma = 12, 6, 0.05, 1.3
    U = _random_state(L, N, 31)
    H = lattice.hopping_matrix(6, 2)
    xi = np.random.default_rng(4).standard_normal(L)
    got = trajectory.step_rk4(U, H, xi, gamma, dt)
    n = np.real(np.sum(U * np.conj(U), axis=1))
    X = -1j * dt * H + np.diag(np.sqrt(gamma * dt) * xi + (2 * n - 1) * gamma * dt)
    series, term = U.copy(), U.copy()
    for k in range(1, 5):
        term = X @ term / k
        series = series + term
    assert np.max(np.abs(got - series)) < 1e-14
    nx = np.linalg.norm(X, 2)
    bound = nx ** 5 / 120 / (1 - nx / 6) * np.linalg.norm(U, 2)
    assert np.linalg.norm(scipy.linalg.expm(X) @ U - got, 2) <= bound


def test_rk4_and_split_step_agree_as_dt_goes_to_zero():
    """One step from the same state and the same normals: the Runge-Kutta step of
    Eq. (QSD_evo) and the split step (propagate, then weight) differ by the
    commutator of H~ and the weight, O(dt^(3/2)) -- the fixed-dt path is the dt -> 0
    limit of the paper's integrator.  Checked: the difference falls by ~8 when dt
    falls by 4."""
    L, N, gamma = 16, 8, 1.0
    U = _random_state(L, N, 41)
    H = lattice.hopping_matrix(L)
    xi = np.random.default_rng(6).standard_normal(L)
    diffs = []
    for dt in (0.02, 0.005, 0.00125):
        a = trajectory.orthonormalize(trajectory.step_rk4(U, H, xi, gamma, dt))
        P = scipy.linalg.expm(-1j * dt * H)
        b = trajectory.orthonormalize(trajectory.homodyne_weight(P @ U, xi, gamma, dt))
        diffs.append(np.max(np.abs(observables.correlation(a) - observables.correlation(b))))
    r1, r2 = diffs[0] / diffs[1], diffs[1] / diffs[2]
    assert 6.0 < r1 < 10.0 and 6.0 < r2 < 10.0, diffs


@pytest.mark.parametrize("Lx,Ly,gamma,seed", [(8, 1, 2.0, 3), (4, 2, 3.0, 7)])
def test_continuous_time_projective_matches_brute_force(Lx, Ly, gamma, seed):
    """App. A's continuous-time protocol: the many-body state driven by the same event
    sequence (waiting times, sites, Born draws) -- exp(-i H tau) between events, n_j or
    1 - n_j at each event -- has C = conj(D) of the oracle's orbitals at every step end."""
    prm = Params(Lx=Lx, Ly=Ly, gamma=gamma, protocol=trajectory.PROJECTIVE_POISSON, reorth_interval=2, seed=seed,
                 traj_id=4)
    L, N = prm.L, prm.N
    nsteps = 30
    out = trajectory.run(prm, nsteps)
    sec = brute.Sector(L, N)
    bonds = brute.ring_bonds(L) if Ly == 1 else brute.torus_bonds(Lx, Ly)
    Hmb = sec.hamiltonian(bonds, prm.J)
    psi = sec.from_orbitals(lattice.initial_orbitals(Lx, Ly))
    rate = gamma * N
    e, t = 0, 0.0
    t_next = -np.log1p(-philox.poisson_event(seed, 4, 0, L)[0]) / rate
    seen = []
    for s in range(nsteps):
        t1 = (s + 1) * prm.dt
        while t_next <= t1:
            psi = scipy.linalg.expm(-1j * (t_next - t) * Hmb) @ psi
            t = t_next
            _, j, u = philox.poisson_event(seed, 4, e, L)
            _, w1 = sec.project(psi, j, 1)
            outcome = 1 if u < w1 else 0
            psi, _ = sec.project(psi, j, outcome)
            seen.append((s, j, outcome, w1))
            e += 1
            t_next += -np.log1p(-philox.poisson_event(seed, 4, e, L)[0]) / rate
        psi = scipy.linalg.expm(-1j * (t1 - t) * Hmb) @ psi
        t = t1
    assert [(a, b, c) for a, b, c, _ in seen] == [(a, b, o) for a, b, u, p, o in out["events"]]
    assert max(abs(w - p) for (_, _, _, w), (_, _, _, p, _) in zip(seen, out["events"])) < 1e-11
    assert len(seen) >= 10 and {o for (_, _, o, _) in seen} == {0, 1}
    D = sec.d_matrix(psi)
    assert np.max(np.abs(observables.correlation(out["U"]) - np.conj(D))) < 1e-12


@pytest.mark.parametrize("Lx,Ly,protocol", [(64, 1, trajectory.HOMODYNE), (8, 6, trajectory.PROJECTIVE)])
def test_cross_block_identity_behind_the_entropy_sketch(Lx, Ly, protocol):
    """For orthonormal U, C = U U^dag is a projector, so C_A - C_A^2 = C_AB C_BA: the
    eigenvalues of C_A satisfy lambda (1 - lambda) = sigma^2 (sigma: singular values of
    C_AB, B the complement), and S_A, whose terms are symmetric under lambda <-> 1 - lambda,
    follows from the sigma^2 alone through lambda = 2 s / (1 + sqrt(1 - 4 s))."""
    prm = Params(Lx=Lx, Ly=Ly, gamma=0.8, protocol=protocol, seed=17)
    U = trajectory.run(prm, 25)["U"]
    L = Lx * Ly
    rng = np.random.default_rng(4)
    A = sorted(rng.choice(L, size=L // 3, replace=False).tolist())
    B = [i for i in range(L) if i not in set(A)]
    C = observables.correlation(U)
    lam = np.clip(np.linalg.eigvalsh(C[np.ix_(A, A)]), 0.0, 1.0)
    sig = np.linalg.svd(C[np.ix_(A, B)], compute_uv=False)
    x = np.sort(np.concatenate([sig**2, np.zeros(len(A) - len(sig))]))
    assert np.max(np.abs(np.sort(lam * (1 - lam)) - x)) < 1e-12
    y = np.clip(x, 0.0, 0.25)
    lam_low = 2 * y / (1 + np.sqrt(1 - 4 * y))
    keep = (lam_low > 0) & (lam_low < 1)
    S = -np.sum(lam_low[keep] * np.log(lam_low[keep]) + (1 - lam_low[keep]) * np.log1p(-lam_low[keep]))
    assert abs(S - observables.entanglement_entropy(U, A)) < 1e-10


def test_continuous_time_forced_replay():
    """Forcing every outcome to the oracle's own gives the same run; forcing one flip
    keeps every event's site and draws (they do not depend on the state) and logs the
    forced outcome, also when the run stops right after that event's step."""
    prm = Params(Lx=12, gamma=2.0, protocol=trajectory.PROJECTIVE_POISSON, seed=21, traj_id=1)
    a = trajectory.run(prm, 8)
    same = trajectory.run(prm, 8, forced={e: ev[4] for e, ev in enumerate(a["events"])})
    assert np.array_equal(a["U"], same["U"]) and a["events"] == same["events"]
    k = next(e for e, ev in enumerate(a["events"]) if 1e-3 < ev[3] < 1 - 1e-3)
    b = trajectory.run(prm, 8, forced={k: 1 - a["events"][k][4]})
    assert [ev[:3] for ev in b["events"]] == [ev[:3] for ev in a["events"]]
    assert b["events"][k][4] == 1 - a["events"][k][4]
    cut = a["events"][k][0]
    pre = trajectory.run(prm, cut + 1, forced={k: 1 - a["events"][k][4]})
    assert pre["events"][k][4] == b["events"][k][4]


def test_continuous_time_event_statistics():
    """Waiting times exponential with mean 1 / (gamma N), sites uniform over the lattice."""
    L, N, gamma = 40, 20, 1.5
    draws = [philox.poisson_event(9, 2, e, L) for e in range(20000)]
    taus = np.array([-np.log1p(-d[0]) / (gamma * N) for d in draws])
    assert abs(taus.mean() * gamma * N - 1.0) < 0.03
    assert abs(np.std(taus) * gamma * N - 1.0) < 0.03
    counts = np.bincount([d[1] for d in draws], minlength=L)
    assert counts.min() > 380 and counts.max() < 620


def test_binary_entropy_terms_edges():
    f = observables.binary_entropy_terms(np.array([0.0, 1.0, 0.5, -1e-17, 1 + 1e-16]))
    assert f[0] == 0 and f[1] == 0 and f[3] == 0 and f[4] == 0
    assert abs(f[2] - np.log(0.5)) < 1e-15


# ---------------------------------------------------------------- statistics

def test_homodyne_occupation_is_a_martingale():
    """With J = 0 the weight of Eq. (A4) leaves E[<n_i>] unchanged (Ito calculus)."""
    L, N, T = 4, 2, 4000
    rng = np.random.default_rng(1)
    U_init = _random_state(L, N, 2)
    n0 = trajectory.occupations(U_init)
    acc = np.zeros(L)
    for tr in range(T):
        xi = philox.noise_normals(77, tr, 0, L)
        U = trajectory.orthonormalize(trajectory.homodyne_weight(U_init, xi, 1.0, 0.05))
        acc += trajectory.occupations(U)
    drift = acc / T - n0
    assert np.max(np.abs(drift)) < 4e-3          # MC error ~1e-3; a wrong drift term gives ~5e-2
    del rng


def test_projective_selection_frequency():
    L, steps, gamma, dt = 512, 40, 1.0, 0.05
    hits = 0
    for s in range(steps):
        u_sel, _ = philox.measure_draws(5, 0, s, L)
        hits += int(np.sum(u_sel < 1 - np.exp(-gamma * dt)))
    p = 1 - np.exp(-gamma * dt)
    assert abs(hits / (L * steps) - p) < 4 * np.sqrt(p * (1 - p) / (L * steps))


# ---------------------------------------------------------------- planted mistakes

def _pin_fails(run):
    """True when a brute-force comparison rejects the (planted) oracle."""
    try:
        worst = run()[0]
    except AssertionError:
        return True
    return worst > 1e-6


def test_pins_catch_planted_mistakes(monkeypatch):
    """Each plausible slip in the oracle fails one of the pins above."""
    prm = Params(Lx=8, gamma=2.0, protocol=PROJECTIVE, reorth_interval=3, seed=11, traj_id=1)

    # (a) a sign slip in the no-click orbital: (v + sqrt(p) e_j) instead of (v - sqrt(p) e_j)
    good_project = trajectory.project_site

    def bad_project(U, j, outcome):
        if outcome == 1:
            return good_project(U, j, 1)
        x = U[j, :].copy(); p = float(np.real(np.vdot(x, x))); sp = np.sqrt(p)
        v = (U @ np.conj(x)) / sp
        ej = np.zeros(U.shape[0], complex); ej[j] = 1
        return U + np.outer((v + sp * ej) / np.sqrt(1 - p) - v, x) / sp
    monkeypatch.setattr(trajectory, "project_site", bad_project)
    assert _pin_fails(lambda: _compare_projective(prm, 40))
    monkeypatch.undo()

    # (a') the Born weight read from the neighbouring row
    def bad_measure(U, p_meas, u_sel, u_out, forced=None):
        events = []
        for j in np.nonzero(u_sel < p_meas)[0]:
            j = int(j)
            x = U[(j + 1) % U.shape[0], :]
            p = min(max(float(np.real(np.vdot(x, x))), 0.0), 1.0)
            outcome = 1 if u_out[j] < p else 0
            events.append((j, float(u_out[j]), p, outcome))
            U = trajectory.project_site(U, j, outcome)
        return U, events
    monkeypatch.setattr(trajectory, "projective_measurements", bad_measure)
    assert _pin_fails(lambda: _compare_projective(prm, 40))
    monkeypatch.undo()

    # (b) propagation with P^dag (time running backwards)
    def back_step(U, P, prm_, s):
        return trajectory.step(U, P.conj().T, prm_, s)
    assert _pin_fails(lambda: _compare_projective(prm, 20, oracle_step=back_step))

    # (c) the QSD drift without the factor 2 on <n>
    def bad_weight(U, xi, gamma, dt):
        n = trajectory.occupations(U)
        return np.exp(np.sqrt(gamma * dt) * xi + (n - 1.0) * gamma * dt)[:, None] * U
    prm_h = Params(Lx=8, gamma=1.0, protocol=HOMODYNE, seed=99, traj_id=3)
    assert _pin_fails(lambda: _compare_homodyne(prm_h, 10, weight=bad_weight))


def _rejected(pin, *args):
    """True when the pin (a test function above) fails on the planted oracle."""
    try:
        pin(*args)
    except AssertionError:
        return True
    return False


def test_pins_catch_planted_mistakes_in_observables_and_lattice(monkeypatch):
    """Slips in the entropy, mutual information, Eq. (2), Eq. (GAB), the Runge-Kutta stages,
    the initial state and the hopping bonds: each is rejected by a pin above, and the pins
    pass again once the slip is removed."""
    good_terms = observables.binary_entropy_terms

    # (e) the entropy without its (1 - lambda) ln(1 - lambda) half
    def terms_half(lam):
        lam = np.clip(np.asarray(lam, dtype=np.float64), 0.0, 1.0)
        out = np.zeros_like(lam)
        inner = lam > 0.0
        out[inner] = lam[inner] * np.log(lam[inner])
        return out
    monkeypatch.setattr(observables, "binary_entropy_terms", terms_half)
    assert _rejected(test_entropy_of_half_filled_random_state_matches_schmidt)
    monkeypatch.undo()

    # (e') the entropy in bits instead of nats
    monkeypatch.setattr(observables, "binary_entropy_terms", lambda lam: good_terms(lam) / np.log(2.0))
    assert _rejected(test_entropy_of_half_filled_random_state_matches_schmidt)
    monkeypatch.undo()

    # (f) mutual information with the joint entropy added instead of subtracted
    def mi_plus(U, A, B):
        return (observables.entanglement_entropy(U, list(A)) + observables.entanglement_entropy(U, list(B))
                + observables.entanglement_entropy(U, sorted(list(A) + list(B))))
    monkeypatch.setattr(observables, "mutual_information", mi_plus)
    # (I(A, Abar) = 2 S(A) and I >= 0 still hold for a pure state: S(A u Abar) = 0)
    assert not _rejected(test_invariants_along_a_projective_trajectory)
    assert _rejected(test_homodyne_matches_brute_force, 8, 1, 1.0)
    monkeypatch.undo()

    # (g) Eq. (2) with the partner site one further than the displacement
    def corr_shifted(U, Lx, Ly=1):
        L = Lx * Ly
        C2 = np.abs(observables.correlation(U)) ** 2
        site = np.arange(L)
        x, y = site % Lx, site // Lx
        out = np.zeros(L)
        for dy in range(Ly):
            for dx in range(Lx):
                d = dx + Lx * dy
                if d:
                    j = (x + dx + 1) % Lx + Lx * ((y + dy) % Ly)
                    out[d] = -float(np.mean(C2[site, j]))
        return out
    monkeypatch.setattr(observables, "displacement_correlation", corr_shifted)
    assert _rejected(test_density_correlations_match_occupation_statistics, 10, 1, 5)
    monkeypatch.undo()

    # (g') Eq. (GAB) summing C_ij instead of |C_ij|^2
    def cov_linear(U, A, B):
        A, B = list(A), list(B)
        return float(np.real(np.sum(U[A, :] @ np.conj(U[B, :]).T)))
    monkeypatch.setattr(observables, "particle_covariance", cov_linear)
    assert _rejected(test_density_correlations_match_occupation_statistics, 4, 3, 6)
    monkeypatch.undo()

    # (h) a Runge-Kutta stage taken over the full step instead of half of it
    def rk4_bad(U, H, xi, gamma, dt):
        n = trajectory.occupations(U)
        A = -1j * H + np.diag((np.sqrt(gamma * dt) * xi + (2.0 * n - 1.0) * gamma * dt) / dt)
        k1 = A @ U
        k2 = A @ (U + 0.5 * dt * k1)
        k3 = A @ (U + dt * k2)
        k4 = A @ (U + dt * k3)
        return U + (dt / 6.0) * (k1 + 2.0 * k2 + 2.0 * k3 + k4)
    monkeypatch.setattr(trajectory, "step_rk4", rk4_bad)
    assert _rejected(test_rk4_step_is_the_quartic_taylor_polynomial_and_close_to_expm)
    monkeypatch.undo()

    # (i) the Neel start on the odd sites (|0101...>, Sec. II's printing) instead of App. A's
    monkeypatch.setattr(lattice, "occupied_sites",
                        lambda Lx, Ly=1: np.arange(1, Lx, 2) if Ly == 1 else
                        np.array([x + Lx * y for y in range(Ly) for x in range(Lx) if (x + y) % 2 == 1]))
    assert _rejected(test_unmonitored_density_closed_form, 64, 1, 200)
    monkeypatch.undo()

    # (j) the ring without its wrap-around bond (open chain)
    good_hop = lattice.hopping_matrix

    def hop_open(Lx, Ly=1, J=1.0):
        H = good_hop(Lx, Ly, J).copy()
        if Ly == 1:
            H[0, Lx - 1] = H[Lx - 1, 0] = 0.0
        return H
    monkeypatch.setattr(lattice, "hopping_matrix", hop_open)
    assert _rejected(test_propagator_is_expm_of_hopping, 12, 1)
    monkeypatch.undo()

    # the pins pass on the real oracle
    test_entropy_of_half_filled_random_state_matches_schmidt()
    test_density_correlations_match_occupation_statistics(10, 1, 5)
    test_rk4_step_is_the_quartic_taylor_polynomial_and_close_to_expm()
    test_propagator_is_expm_of_hopping(12, 1)
