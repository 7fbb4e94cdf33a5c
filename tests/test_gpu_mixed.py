"""Mixed-precision (split-fp16 tensor-core) path vs the FP64 oracle (needs a GB300).

Tolerances come from the arithmetic: the float32 state (2^-24), split-fp16
products (2^-22) and fp32 tensor-core accumulation (about 2^-24 per 16-deep
update on the banded propagation sums) give a per-step error in C = U U^dag
of at most ~2e-6, so after n steps max|dC| <= 2e-6 n.  The entropy bar is the
method's: relative error <= 1e-3; orthonormality <= 1e-6 after a full
CholeskyQR2 step.
"""
import numpy as np
import pytest

from oracle import observables, trajectory
from oracle.trajectory import HOMODYNE, PROJECTIVE, Params

pytestmark = pytest.mark.gpu

PER_STEP_C = 2e-6
S_REL = 1e-3
ORTHO = 1e-6


@pytest.fixture(scope="module")
def fm():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2508_18468_gb300 import build
    build.build()
    from paper_2508_18468_gb300 import fm as mod
    return mod


def mixed(fm, Lx, Ly=1, **kw):
    return fm.Trajectories(fm.make_params(Lx, Ly, precision=fm.FM_MIXED, **kw))


def cdiff(Ua, Ub):
    return float(np.max(np.abs(observables.correlation(Ua) - observables.correlation(Ub))))


def srel(a, b):
    return abs(a - b) / max(abs(b), 1.0)


NEAR_TIE = 1e-4   # |u - p| below which the mixed precision may decide a Born draw either way


def replay_if_needed(got, prm, n, poisson=False):
    """Outcome agreement with replay of near ties.  ``got``: the GPU's events as
    (step, site, outcome) in time order.  The oracle runs on its own; if an outcome
    differs, it runs again with every outcome forced to the GPU's, and each forced
    outcome that the oracle's own decision would not take must be a near tie.
    Returns the oracle run the GPU state is compared with."""
    ref = trajectory.run(prm, n)
    exp = [(s, j, o) for (s, j, u, p, o) in ref["events"]]
    if sorted(got) == sorted(exp):
        return ref
    if poisson:
        forced = {e: o for e, (s, j, o) in enumerate(got)}
    else:
        forced = {}
        for (s, j, o) in got:
            forced.setdefault(s, {})[j] = o
    ref = trajectory.run(prm, n, forced=forced)
    assert sorted((s, j) for (s, j, u, p, o) in ref["events"]) == sorted((s, j) for (s, j, o) in got)
    flips = [abs(u - p) for (s, j, u, p, o) in ref["events"] if o != (1 if u < p else 0)]
    assert flips and max(flips) < NEAR_TIE, "outcome mismatch away from a near tie"
    print("replayed %d near-tie outcome(s), margins %s" % (len(flips), flips))
    return ref


@pytest.mark.parametrize("gamma,reorth", [(1.0, 1), (0.3, 1), (1.0, 4)])
def test_homodyne_ring256(fm, gamma, reorth):
    n = 48
    g = mixed(fm, 256, protocol=fm.FM_HOMODYNE, gamma=gamma, seed=31, reorth_interval=reorth)
    g.step(n)
    ref = trajectory.run(Params(Lx=256, gamma=gamma, protocol=HOMODYNE, seed=31), n)["U"]
    U = g.copy_U()
    dc = cdiff(U, ref)
    half = list(range(128))
    S, S_ref = g.entropy(half), observables.entanglement_entropy(ref, half)
    ortho = g.orthonormality_error(list(range(0, 128, 4)))
    print("homodyne L=256 gamma=%g reorth=%d: max|dC|=%.2e  S=%.6f S_ref=%.6f rel=%.2e  ortho=%.2e"
          % (gamma, reorth, dc, S, S_ref, srel(S, S_ref), ortho))
    assert dc <= PER_STEP_C * n
    assert srel(S, S_ref) <= S_REL
    assert ortho <= ORTHO


@pytest.mark.parametrize("drain", [1, 2])
def test_homodyne_ring1024_longer_drain_interval(fm, drain):
    """The first-pass product drained every 4 or 8 K-blocks between second passes (tile_config
    bits 5-6; second pass every 4 steps): within the per-step bound of the oracle, the entropy
    within the method's bar, U^dag U = 1 to 1e-6 after the period, ~1e-6 inside it."""
    n = 24
    g = mixed(fm, 1024, protocol=fm.FM_HOMODYNE, gamma=1.0, seed=37, reorth_interval=4,
              tile_config=drain << 5)
    g.step(n - 1)
    mid = g.orthonormality_error(list(range(0, 512, 8)))
    g.step(1)
    ref = trajectory.run(Params(Lx=1024, gamma=1.0, protocol=HOMODYNE, seed=37), n)["U"]
    dc = cdiff(g.copy_U(), ref)
    half = list(range(512))
    S, S_ref = g.entropy(half), observables.entanglement_entropy(ref, half)
    ortho = g.orthonormality_error(list(range(0, 512, 8)))
    print("drain every %d K-blocks: max|dC|=%.2e rel S %.2e ortho %.2e (inside the period %.2e)"
          % (2 << drain, dc, srel(S, S_ref), ortho, mid))
    assert dc <= PER_STEP_C * n
    assert srel(S, S_ref) <= S_REL
    assert ortho <= ORTHO
    assert mid <= 1e-4


def test_projective_ring256(fm):
    n = 40
    g = mixed(fm, 256, protocol=fm.FM_PROJECTIVE, gamma=1.0, seed=44, event_capacity=100000)
    g.step(n)
    ev, _ = g.take_events()
    got = [(e[1], e[2], e[5]) for e in ev]
    ref = replay_if_needed(got, Params(Lx=256, gamma=1.0, protocol=PROJECTIVE, seed=44), n)
    dc = cdiff(g.copy_U(), ref["U"])
    half = list(range(128))
    S, S_ref = g.entropy(half), observables.entanglement_entropy(ref["U"], half)
    print("projective L=256: events=%d max|dC|=%.2e S rel=%.2e" % (len(ev), dc, srel(S, S_ref)))
    assert dc <= PER_STEP_C * n
    assert srel(S, S_ref) <= S_REL


def test_homodyne_torus_16x16(fm):
    n = 30
    g = mixed(fm, 16, 16, protocol=fm.FM_HOMODYNE, gamma=1.5, seed=7)
    g.step(n)
    ref = trajectory.run(Params(Lx=16, Ly=16, gamma=1.5, protocol=HOMODYNE, seed=7), n)["U"]
    assert cdiff(g.copy_U(), ref) <= PER_STEP_C * n
    A = [x + 16 * y for y in range(4) for x in range(4)]
    B = [x + 16 * y for y in range(4) for x in range(8, 12)]
    I, I_ref = g.mutual_info(A, B), observables.mutual_information(ref, A, B)
    print("torus 16x16: I=%.6f I_ref=%.6f" % (I, I_ref))
    assert abs(I - I_ref) <= S_REL * max(1.0, abs(I_ref))


def test_batch_of_three_with_rates(fm):
    n = 20
    gam = [0.3, 1.0, 2.0]
    g = mixed(fm, 512, batch=3, protocol=fm.FM_HOMODYNE, seed=5, traj_id=10)
    g.set_gammas(gam)
    g.step(n)
    for b in range(3):
        ref = trajectory.run(Params(Lx=512, gamma=gam[b], protocol=HOMODYNE, seed=5, traj_id=10 + b), n)["U"]
        assert cdiff(g.copy_U(b), ref) <= PER_STEP_C * n


def test_unmonitored_ring1024_closed_form(fm):
    n = 40
    g = mixed(fm, 1024, protocol=fm.FM_PROJECTIVE, gamma=0.0, reorth_interval=1)
    g.step(n)
    occ = g.occupations()
    k = 2 * np.pi * np.arange(1024) / 1024
    ref = 0.5 + 0.5 * (-1.0) ** np.arange(1024) * np.mean(np.cos(4.0 * n * 0.05 * np.cos(k)))
    err = float(np.max(np.abs(occ - ref)))
    print("unmonitored L=1024 mixed: max|dn|=%.2e" % err)
    assert err <= PER_STEP_C * n


def test_mixed_against_fp64_gpu_ring2048(fm):
    n = 12
    kw = dict(protocol=fm.FM_HOMODYNE, gamma=0.5, seed=9)
    gm = mixed(fm, 2048, **kw)
    gd = fm.Trajectories(fm.make_params(2048, precision=fm.FM_FP64, **kw))
    gm.step(n)
    gd.step(n)
    half = list(range(1024))
    Sm, Sd = gm.entropy(half), gd.entropy(half)
    print("L=2048 mixed vs fp64 GPU: S=%.8f vs %.8f rel=%.2e" % (Sm, Sd, srel(Sm, Sd)))
    assert srel(Sm, Sd) <= S_REL
    assert gm.orthonormality_error(list(range(0, 1024, 16))) <= ORTHO


def _compare_projective(fm, g, L, gamma, seed, n, batch):
    ev, dropped = g.take_events()
    assert dropped == 0
    for b in range(batch):
        got = [(e[1], e[2], e[5]) for e in ev if e[0] == b]
        ref = replay_if_needed(got, Params(Lx=L, gamma=gamma, protocol=PROJECTIVE, seed=seed, traj_id=b), n)
        dc = cdiff(g.copy_U(b), ref["U"])
        print("projective L=%d gamma=%g traj %d: %d events, max|dC|=%.2e" % (L, gamma, b, len(got), dc))
        assert dc <= PER_STEP_C * n


def test_projective_block_update_many_events(fm):
    """~97 measured sites per step: the block update (events on the selected block, one
    tensor-core update of U) against the oracle's event-by-event rank-1 updates."""
    L, n = 1024, 6
    g = mixed(fm, L, batch=2, protocol=fm.FM_PROJECTIVE, gamma=2.0, seed=45, event_capacity=100000)
    g.step(n)
    _compare_projective(fm, g, L, 2.0, 45, n, 2)
    assert g.orthonormality_error(list(range(0, 512, 16))) <= ORTHO


def test_projective_more_sites_than_the_block_holds(fm):
    """gamma dt large enough that nearly every site is measured: the step falls back to
    the event-by-event path and still matches the oracle."""
    L, n = 256, 3
    g = mixed(fm, L, batch=1, protocol=fm.FM_PROJECTIVE, gamma=60.0, seed=46, event_capacity=100000)
    g.step(n)
    _compare_projective(fm, g, L, 60.0, 46, n, 1)


@pytest.mark.parametrize("Lx,Ly", [(256, 1), (16, 16)])
def test_density_correlation_and_particle_covariance_mixed(fm, Lx, Ly):
    n = 20
    g = mixed(fm, Lx, Ly, protocol=fm.FM_HOMODYNE, gamma=0.7, seed=32)
    g.step(n)
    U = trajectory.run(Params(Lx=Lx, Ly=Ly, gamma=0.7, protocol=HOMODYNE, seed=32), n)["U"]
    c = g.density_correlation()
    ref = observables.displacement_correlation(U, Lx, Ly)
    print("C(d) L=%dx%d: max|dc| = %.2e (max |c| %.2e)" % (Lx, Ly, np.max(np.abs(c - ref)), np.max(np.abs(ref))))
    assert np.max(np.abs(c - ref)) <= PER_STEP_C * n
    L = Lx * Ly
    A, B = list(range(0, L // 4)), list(range(L // 2, L // 2 + L // 4))
    G, Gref = g.particle_covariance(A, B), observables.particle_covariance(U, A, B)
    assert abs(G - Gref) <= PER_STEP_C * n * max(1.0, Gref)


@pytest.mark.parametrize("Lx,Ly,protocol", [(256, 1, HOMODYNE), (16, 16, PROJECTIVE), (512, 1, PROJECTIVE)])
def test_banded_propagation_mixed(fm, Lx, Ly, protocol):
    n = 16
    prot = fm.FM_HOMODYNE if protocol == HOMODYNE else fm.FM_PROJECTIVE
    g = mixed(fm, Lx, Ly, protocol=prot, gamma=0.8, seed=24, batch=2)
    g.set_propagation(fm.FM_PROP_BANDED)
    g.step(n)
    for b in range(2):
        ref = trajectory.run(Params(Lx=Lx, Ly=Ly, gamma=0.8, protocol=protocol, seed=24, traj_id=b), n)
        dc = cdiff(g.copy_U(b), ref["U"])
        print("banded mixed %dx%d traj %d: max|dC| = %.2e" % (Lx, Ly, b, dc))
        assert dc <= PER_STEP_C * n
    assert g.orthonormality_error(list(range(0, Lx * Ly // 2, 8))) <= ORTHO


@pytest.mark.parametrize("Lx,Ly", [(256, 1), (16, 16)])
def test_runge_kutta_protocol_mixed(fm, Lx, Ly):
    n = 24
    g = mixed(fm, Lx, Ly, protocol=fm.FM_HOMODYNE_RK4, gamma=0.9, seed=28)
    g.step(n)
    ref = trajectory.run(Params(Lx=Lx, Ly=Ly, gamma=0.9, protocol=trajectory.HOMODYNE_RK4, seed=28), n)["U"]
    dc = cdiff(g.copy_U(), ref)
    A = list(range(Lx * Ly // 2))
    S, S_ref = g.entropy(A), observables.entanglement_entropy(ref, A)
    print("RK4 mixed %dx%d: max|dC| = %.2e, S rel = %.2e" % (Lx, Ly, dc, srel(S, S_ref)))
    assert dc <= PER_STEP_C * n
    assert srel(S, S_ref) <= S_REL


@pytest.mark.parametrize("Lx,Ly,reorth", [(256, 1, 1), (16, 16, 2)])
def test_continuous_time_projective_mixed(fm, Lx, Ly, reorth):
    """The continuous-time projective protocol on the float state against the FP64 oracle."""
    n = 30
    g = mixed(fm, Lx, Ly, protocol=fm.FM_PROJECTIVE_POISSON, gamma=0.8, seed=52, reorth_interval=reorth,
              event_capacity=100000)
    g.step(n)
    ev, _ = g.take_events()
    got = [(e[1], e[2], e[5]) for e in ev]
    ref = replay_if_needed(got, Params(Lx=Lx, Ly=Ly, gamma=0.8, protocol=trajectory.PROJECTIVE_POISSON, seed=52,
                                       reorth_interval=reorth), n, poisson=True)
    dc = cdiff(g.copy_U(), ref["U"])
    A = list(range(Lx * Ly // 2))
    S, S_ref = g.entropy(A), observables.entanglement_entropy(ref["U"], A)
    print("continuous-time projective mixed %dx%d: events=%d max|dC|=%.2e S rel=%.2e"
          % (Lx, Ly, len(ev), dc, srel(S, S_ref)))
    assert dc <= PER_STEP_C * n
    assert srel(S, S_ref) <= S_REL


def test_projective_ring1024_forced_to_oracle_over_200_steps(fm):
    """The mixed path held on the oracle's outcome sequence (fm_force_outcomes) for 200
    projective steps at L = 1024, gamma = 0.5: no near tie can branch the two runs, so the
    states stay comparable for the whole run; C within the per-step bound and the
    half-chain entropy within the method's bar."""
    n = 200
    prm = Params(Lx=1024, gamma=0.5, protocol=PROJECTIVE, seed=0x2508184689)
    half = list(range(512))
    ref = trajectory.run(prm, n)
    forced = [(0, s, j, o) for (s, j, u, p, o) in ref["events"]]
    g = mixed(fm, 1024, protocol=fm.FM_PROJECTIVE, gamma=0.5, seed=0x2508184689, event_capacity=1 << 16)
    g.force_outcomes(forced)
    g.step(n)
    ev, dropped = g.take_events()
    assert dropped == 0
    assert sorted((e[1], e[2], e[5]) for e in ev) == sorted((s, j, o) for (s, j, u, p, o) in ref["events"])
    dc = cdiff(g.copy_U(), ref["U"])
    S, S_ref = g.entropy(half), observables.entanglement_entropy(ref["U"], half)
    print("forced replay, L=1024, %d steps, %d events: max|dC| %.2e, S %.9f vs %.9f (rel %.2e)"
          % (n, len(ev), dc, S, S_ref, srel(S, S_ref)))
    assert dc <= PER_STEP_C * n
    assert srel(S, S_ref) <= S_REL


def test_projective_event_paths_agree_bit_for_bit(fm):
    """The step's projective events run in one launch per step when many trajectories keep
    the GPU busy (here 64) and as per-phase launches spread over the GPU when a few
    trajectories have long event lists (here one, ~390 events per step at gamma = 2, L = 4096):
    trajectory 0 alone and inside the 64-trajectory batch ends in the same bits."""
    kw = dict(protocol=fm.FM_PROJECTIVE, gamma=2.0, seed=0x250818468A, event_capacity=1 << 16)
    alone = mixed(fm, 4096, batch=1, **kw)
    batch = mixed(fm, 4096, batch=64, **kw)
    alone.step(3)
    batch.step(3)
    ev, _ = alone.take_events()
    assert len(ev) > 3 * 300
    assert np.array_equal(alone.copy_U(0), batch.copy_U(0))
