"""All-FP64 GPU path vs the FP64 oracle, element by element (needs a GB300).

Bars (FP64 mode): max |C_gpu - C_oracle| <= 1e-10 with C = U U^dag, entropy
relative error <= 1e-9 (relative to max(S, 1 nat)), projective outcomes and
their uniform draws bit-identical.
"""
import numpy as np
import pytest

from oracle import lattice, observables, philox, trajectory
from oracle.trajectory import HOMODYNE, PROJECTIVE, Params

pytestmark = pytest.mark.gpu

C_TOL = 1e-10
S_TOL = 1e-9


@pytest.fixture(scope="module")
def fm():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2508_18468_gb300 import build
    build.build()
    from paper_2508_18468_gb300 import fm as mod
    return mod


def pair(fm, Lx, Ly=1, gamma=0.5, protocol=PROJECTIVE, batch=1, seed=1, traj_id=0, reorth=1, events=0,
         precision=0):
    po = Params(Lx=Lx, Ly=Ly, gamma=gamma, protocol=protocol, reorth_interval=reorth, seed=seed, traj_id=traj_id)
    pg = fm.make_params(Lx, Ly, batch=batch, protocol=protocol, precision=precision, reorth_interval=reorth,
                        event_capacity=events, gamma=gamma, seed=seed, traj_id=traj_id)
    return po, fm.Trajectories(pg)


def cdiff(Ua, Ub):
    return float(np.max(np.abs(observables.correlation(Ua) - observables.correlation(Ub))))


def srel(a, b):
    return abs(a - b) / max(abs(b), 1.0)


def test_projective_draws_and_outcomes_bit_exact(fm):
    po, g = pair(fm, 64, gamma=2.0, events=100000, seed=77, traj_id=3)
    g.step(20)
    ev, dropped = g.take_events()
    ref = trajectory.run(po, 20)
    assert dropped == 0
    got = sorted((e[1], e[2], e[3], e[5]) for e in ev)          # (step, site, u, outcome)
    exp = sorted((s, j, u, o) for (s, j, u, p, o) in ref["events"])
    assert [(a, b, d) for a, b, c, d in got] == [(a, b, d) for a, b, c, d in exp]
    assert all(a[2] == b[2] for a, b in zip(got, exp))           # uniforms bit-identical
    # Born weights agree to rounding
    pg = {(e[1], e[2]): e[4] for e in ev}
    for (s, j, u, p, o) in ref["events"]:
        assert abs(pg[(s, j)] - p) < 1e-12
    # the selection is exactly the oracle's u_select < 1 - exp(-gamma dt)
    for s in range(20):
        us, _ = philox.measure_draws(77, 3, s, 64)
        sel = set(np.nonzero(us < 1 - np.exp(-2.0 * 0.05))[0].tolist())
        assert sel == {e[2] for e in ev if e[1] == s}


def test_ring64_projective_200_steps(fm):
    """Projective ring L = 64, gamma = 0.5, reorth every step, half-chain EE every 10 steps."""
    po, g = pair(fm, 64, gamma=0.5, seed=0x2508184681, events=100000)
    half = list(range(32))
    ref = trajectory.run(po, 200, ee_every=10, ee_sites=half)
    ee = []
    for k in range(20):
        g.step(10)
        ee.append(g.entropy(half))
    assert cdiff(g.copy_U(), ref["U"]) <= C_TOL
    for (done, s_ref), s in zip(ref["ee"], ee):
        assert srel(s, s_ref) <= S_TOL, (done, s, s_ref)
    ev, _ = g.take_events()
    assert sorted((e[1], e[2], e[5]) for e in ev) == sorted((s, j, o) for (s, j, u, p, o) in ref["events"])


@pytest.mark.parametrize("gamma,reorth", [(1.0, 1), (0.3, 2)])
def test_ring64_homodyne(fm, gamma, reorth):
    po, g = pair(fm, 64, gamma=gamma, protocol=HOMODYNE, seed=11, traj_id=2, reorth=reorth)
    ref = trajectory.run(po, 100)
    g.step(100)
    U = g.copy_U()
    assert cdiff(U, ref["U"]) <= C_TOL
    half = list(range(32))
    assert srel(g.entropy(half), observables.entanglement_entropy(ref["U"], half)) <= S_TOL


@pytest.mark.parametrize("protocol,gamma", [(PROJECTIVE, 1.5), (HOMODYNE, 1.0)])
def test_torus_8x6(fm, protocol, gamma):
    po, g = pair(fm, 8, 6, gamma=gamma, protocol=protocol, seed=5)
    ref = trajectory.run(po, 40)
    g.step(40)
    assert cdiff(g.copy_U(), ref["U"]) <= C_TOL
    strip = [x + 8 * y for y in range(6) for x in range(4)]
    assert srel(g.entropy(strip), observables.entanglement_entropy(ref["U"], strip)) <= S_TOL


def test_batch_with_per_trajectory_rates(fm):
    gam = [0.2, 1.0, 3.0]
    _, g = pair(fm, 32, batch=3, protocol=PROJECTIVE, seed=9, traj_id=5)
    g.set_gammas(gam)
    g.step(30)
    for b in range(3):
        po = Params(Lx=32, gamma=gam[b], protocol=PROJECTIVE, seed=9, traj_id=5 + b)
        ref = trajectory.run(po, 30)
        assert cdiff(g.copy_U(b), ref["U"]) <= C_TOL


@pytest.mark.parametrize("Lx", [2, 6, 70, 130])
@pytest.mark.parametrize("protocol", [PROJECTIVE, HOMODYNE])
def test_ragged_sizes(fm, Lx, protocol):
    po, g = pair(fm, Lx, gamma=1.0, protocol=protocol, seed=3)
    ref = trajectory.run(po, 15)
    g.step(15)
    assert cdiff(g.copy_U(), ref["U"]) <= C_TOL
    A = list(range(Lx // 2))
    assert srel(g.entropy(A), observables.entanglement_entropy(ref["U"], A)) <= S_TOL


def test_unmonitored_ring1024_closed_form(fm):
    _, g = pair(fm, 1024, gamma=0.0, reorth=8)
    g.step(40)
    n = g.occupations()
    k = 2 * np.pi * np.arange(1024) / 1024
    ref = 0.5 + 0.5 * (-1.0) ** np.arange(1024) * np.mean(np.cos(4.0 * 40 * 0.05 * np.cos(k)))
    assert np.max(np.abs(n - ref)) < 1e-12


def test_ring1024_projective_short(fm):
    po, g = pair(fm, 1024, gamma=2.0, seed=0x2508184682, traj_id=1)
    ref = trajectory.run(po, 6)
    g.step(6)
    assert cdiff(g.copy_U(), ref["U"]) <= C_TOL
    for ell in (128, 256, 512):
        A = list(range(ell))
        assert srel(g.entropy(A), observables.entanglement_entropy(ref["U"], A)) <= S_TOL


def test_entropy_edge_cases(fm):
    po, g = pair(fm, 48, gamma=0.8, protocol=HOMODYNE, seed=21)
    g.step(25)
    ref = trajectory.run(po, 25)["U"]
    assert g.entropy([]) == 0.0
    assert abs(g.entropy(list(range(48)))) < 1e-10               # pure state
    A = [0, 3, 4, 17, 30]
    Abar = [i for i in range(48) if i not in A]
    assert abs(g.entropy(A) - g.entropy(Abar)) < 1e-10
    assert srel(g.entropy(A), observables.entanglement_entropy(ref, A)) <= S_TOL
    assert srel(g.entropy(Abar), observables.entanglement_entropy(ref, Abar)) <= S_TOL


def test_mutual_info_vs_oracle(fm):
    po, g = pair(fm, 8, 6, gamma=1.0, protocol=HOMODYNE, seed=4)
    g.step(20)
    ref = trajectory.run(po, 20)["U"]
    A = [0, 1, 8, 9]
    B = [4, 5, 12, 13]
    I = g.mutual_info(A, B)
    assert abs(I - observables.mutual_information(ref, A, B)) <= 1e-9
    with pytest.raises(fm.FmError):
        g.mutual_info(A, [1, 2])
    g.step(1)                                                       # argument errors are not sticky


def test_checkpoint_resume_is_bitwise(fm, tmp_path):
    _, g1 = pair(fm, 40, gamma=1.0, protocol=HOMODYNE, seed=8)
    g1.step(20)
    _, g2 = pair(fm, 40, gamma=1.0, protocol=HOMODYNE, seed=8)
    g2.step(10)
    g2.save(tmp_path / "ck.bin")
    _, g3 = pair(fm, 40, gamma=1.0, protocol=HOMODYNE, seed=8)
    g3.load(tmp_path / "ck.bin")
    g3.step(10)
    assert np.array_equal(g1.copy_U(), g3.copy_U())
    assert g3.steps_done() == 20


def test_reset_trajectory_matches_fresh_run(fm):
    _, g = pair(fm, 32, batch=2, gamma=1.0, protocol=PROJECTIVE, seed=12, traj_id=0)
    g.step(7)
    g.reset_trajectory(1, traj_id=40, gamma=0.5)
    g.step(9)
    assert g.steps_done(1) == 9 and g.steps_done(0) == 16
    ref = trajectory.run(Params(Lx=32, gamma=0.5, protocol=PROJECTIVE, seed=12, traj_id=40), 9)
    assert cdiff(g.copy_U(1), ref["U"]) <= C_TOL


def test_orthonormality_and_invariants(fm):
    _, g = pair(fm, 96, gamma=1.0, protocol=HOMODYNE, seed=6)
    g.step(30)
    assert g.orthonormality_error(list(range(0, 48, 3))) < 1e-13
    U = g.copy_U()
    C = observables.correlation(U)
    assert abs(np.trace(C).real - 48) < 1e-11
    assert np.max(np.abs(C @ C - C)) < 1e-12


def test_invalid_arguments_are_rejected(fm):
    _, g = pair(fm, 16)
    with pytest.raises(fm.FmError):
        g.entropy([0, 0])
    with pytest.raises(fm.FmError):
        g.entropy([16])
    with pytest.raises(fm.FmError):
        g.step(-1)
    with pytest.raises(fm.FmError):
        g.orthonormality_error([99])
    g.step(2)
    assert g.steps_done() == 2


def test_large_batch_uses_one_cta_per_trajectory_path(fm):
    """64 trajectories take the one-CTA-per-trajectory projective kernel."""
    _, g = pair(fm, 32, batch=64, protocol=PROJECTIVE, gamma=2.0, seed=17, traj_id=0)
    g.step(12)
    for b in (0, 31, 63):
        ref = trajectory.run(Params(Lx=32, gamma=2.0, protocol=PROJECTIVE, seed=17, traj_id=b), 12)
        assert cdiff(g.copy_U(b), ref["U"]) <= C_TOL


@pytest.mark.parametrize("Lx,Ly,protocol", [(64, 1, PROJECTIVE), (8, 6, HOMODYNE), (70, 1, HOMODYNE)])
def test_density_correlation_and_particle_covariance(fm, Lx, Ly, protocol):
    po, g = pair(fm, Lx, Ly, gamma=1.0, protocol=protocol, seed=19)
    g.step(25)
    U = trajectory.run(po, 25)["U"]
    c = g.density_correlation()
    assert np.max(np.abs(c - observables.displacement_correlation(U, Lx, Ly))) <= 1e-13
    L = Lx * Ly
    A, B = list(range(0, L // 4)), list(range(L // 2, L // 2 + L // 5))
    G = g.particle_covariance(A, B)
    assert abs(G - observables.particle_covariance(U, A, B)) <= 1e-13
    assert g.particle_covariance([], B) == 0.0
    with pytest.raises(fm.FmError):
        g.particle_covariance(A, A[:2])


@pytest.mark.parametrize("Lx,Ly,protocol", [(64, 1, PROJECTIVE), (8, 6, HOMODYNE), (1024, 1, HOMODYNE),
                                             (6, 1, PROJECTIVE)])
def test_banded_propagation_matches_dense_oracle(fm, Lx, Ly, protocol):
    """Stencils of the circulant propagator (taps above 1e-15) against the oracle's dense P."""
    po, g = pair(fm, Lx, Ly, gamma=1.0, protocol=protocol, seed=23, reorth=2)
    g.set_propagation(fm.FM_PROP_BANDED)
    n = 12
    g.step(n)
    ref = trajectory.run(po, n)
    assert cdiff(g.copy_U(), ref["U"]) <= C_TOL


@pytest.mark.parametrize("Lx,Ly,reorth", [(64, 1, 1), (8, 6, 2), (2, 4, 1), (130, 1, 3)])
def test_runge_kutta_protocol_matches_oracle(fm, Lx, Ly, reorth):
    """App. A's integrator (RK4 of Eq. (QSD_evo), nearest-neighbour H~) against the oracle."""
    po, g = pair(fm, Lx, Ly, gamma=1.2, protocol=trajectory.HOMODYNE_RK4, seed=27, reorth=reorth)
    n = 20
    g.step(n)
    ref = trajectory.run(po, n)
    assert cdiff(g.copy_U(), ref["U"]) <= C_TOL
    A = list(range(Lx * Ly // 2))
    assert srel(g.entropy(A), observables.entanglement_entropy(ref["U"], A)) <= S_TOL


@pytest.mark.parametrize("Lx,Ly,gamma,reorth", [(64, 1, 3.0, 1), (16, 1, 6.0, 2), (20, 4, 1.5, 3), (6, 6, 2.0, 1)])
def test_continuous_time_projective_matches_oracle(fm, Lx, Ly, gamma, reorth):
    """App. A's continuous-time projective protocol: Poisson events, exp(-i H~ tau) between
    them (Bessel-tap stencils on long directions, the plane-wave row on short ones)."""
    po, g = pair(fm, Lx, Ly, gamma=gamma, protocol=trajectory.PROJECTIVE_POISSON, seed=41, traj_id=5,
                 reorth=reorth, events=100000)
    n = 30
    g.step(n)
    ref = trajectory.run(po, n)
    ev, dropped = g.take_events()
    assert dropped == 0 and len(ev) == len(ref["events"]) > 0
    got = [(e[1], e[2], e[3], e[5]) for e in ev]                 # event order is the time order
    exp = [(s, j, u, o) for (s, j, u, p, o) in ref["events"]]
    assert got == exp                                            # sites, draws, outcomes bit-identical
    assert max(abs(e[4] - r[3]) for e, r in zip(ev, ref["events"])) < 1e-12
    assert cdiff(g.copy_U(), ref["U"]) <= C_TOL
    A = list(range(Lx * Ly // 2))
    assert srel(g.entropy(A), observables.entanglement_entropy(ref["U"], A)) <= S_TOL


def test_continuous_time_projective_batch_rates_and_restart(fm):
    """Three trajectories at their own rates, one restarted halfway: each equals its own
    oracle trajectory (the event schedule is per trajectory)."""
    Lx, rates = 32, [0.0, 2.0, 5.0]
    pg = fm.make_params(Lx, batch=3, protocol=fm.FM_PROJECTIVE_POISSON, precision=fm.FM_FP64, gamma=1.0,
                        seed=9, traj_id=100)
    g = fm.Trajectories(pg)
    g.set_gammas(rates)
    g.step(10)
    g.reset_trajectory(1, 777, 3.0)
    g.step(15)
    for b, (tid, gam, n) in enumerate([(100, 0.0, 25), (777, 3.0, 15), (102, 5.0, 25)]):
        ref = trajectory.run(Params(Lx=Lx, gamma=gam, protocol=trajectory.PROJECTIVE_POISSON, seed=9,
                                    traj_id=tid), n)
        assert cdiff(g.copy_U(b), ref["U"]) <= C_TOL, b


def test_continuous_time_projective_checkpoint_and_graph_request(fm, tmp_path):
    """A checkpoint restores the event schedule (replayed from the step counts), and
    asking for CUDA graphs leaves the host-scheduled protocol eager: both equal an
    uninterrupted run bit for bit."""
    pg = fm.make_params(24, batch=2, protocol=fm.FM_PROJECTIVE_POISSON, precision=fm.FM_FP64, gamma=2.5,
                        seed=13, reorth_interval=2)
    a = fm.Trajectories(pg)
    a.step(17)
    b = fm.Trajectories(pg)
    b.set_graphs(True)
    b.step(7)
    path = str(tmp_path / "pois.ckpt")
    b.save(path)
    c = fm.Trajectories(pg)
    c.load(path)
    c.step(10)
    for t in range(2):
        assert np.array_equal(a.copy_U(t), c.copy_U(t))


def test_forced_outcomes_replay_oracle(fm):
    """fm_force_outcomes against the oracle's forced replay: in five of steps 2-11 the first
    measurement with 0.05 < p < 0.95 gets the outcome opposite to the natural one; every
    other measurement is decided by its draw.  Outcomes and C = U U^dag equal the oracle's
    run with the same forced outcomes, and the forced measurements are logged with u = -1
    (click) or 2 (no-click)."""
    po, g = pair(fm, 64, gamma=2.0, events=100000, seed=91, traj_id=5)
    natural = trajectory.run(po, 12)["events"]
    forced = {}
    for s in range(2, 12):
        for (st, j, u, p, o) in natural:
            if st == s and 0.05 < p < 0.95 and len(forced) < 5:
                forced[s] = {j: 1 - o}
                break
    assert len(forced) == 5
    ref = trajectory.run(po, 12, forced=forced)
    g.force_outcomes([(0, s, j, o) for s, d in forced.items() for j, o in d.items()])
    g.step(12)
    ev, dropped = g.take_events()
    assert dropped == 0
    assert cdiff(g.copy_U(), ref["U"]) <= C_TOL
    assert sorted((e[1], e[2], e[5]) for e in ev) == sorted((s, j, o) for (s, j, u, p, o) in ref["events"])
    flagged = {(e[1], e[2]): e[3] for e in ev if not (0.0 <= e[3] <= 1.0)}
    assert flagged == {(s, j): (-1.0 if o else 2.0) for s, d in forced.items() for j, o in d.items()}
    # the same list on a second state, then cleared: natural outcomes again
    g2 = pair(fm, 64, gamma=2.0, events=100000, seed=91, traj_id=5)[1]
    g2.force_outcomes([(0, s, j, o) for s, d in forced.items() for j, o in d.items()])
    g2.force_outcomes([])
    g2.step(12)
    ev2, _ = g2.take_events()
    assert sorted((e[1], e[2], e[5]) for e in ev2) == sorted((s, j, o) for (s, j, u, p, o) in natural)
