"""Full-size checks in the launch configuration the benchmark uses (needs a GB300).

The oracle cannot follow an L = 16384 ring or a 160 x 160 torus for long, so
these check what holds at any size: the unmonitored closed form, U^dag U = 1,
Tr C = N, measured sites ending the step with n_j in {0, 1}, and 0 <= MI.
"""
import numpy as np
import pytest

from paper_2508_18468_gb300 import workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fm():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2508_18468_gb300 import build
    build.build()
    from paper_2508_18468_gb300 import fm as mod
    return mod


def test_ring16384_unmonitored_closed_form(fm):
    L, n = 16384, 20
    g = fm.Trajectories(fm.make_params(L, protocol=fm.FM_PROJECTIVE, precision=fm.FM_MIXED, gamma=0.0))
    g.step(n)
    occ = g.occupations()
    k = 2 * np.pi * np.arange(L) / L
    ref = 0.5 + 0.5 * (-1.0) ** np.arange(L) * np.mean(np.cos(4.0 * n * 0.05 * np.cos(k)))
    assert np.max(np.abs(occ - ref)) <= 2e-6 * n


def test_ring16384_homodyne_invariants(fm):
    L = 16384
    wl = workloads.WORKLOADS["ring16384_homodyne"]
    g = fm.Trajectories(fm.make_params(L, batch=4, protocol=fm.FM_HOMODYNE, precision=fm.FM_MIXED,
                                       seed=workloads.seed_of("ring16384_homodyne")))
    g.set_gammas(wl["gammas"])
    g.step(3)
    for b in range(4):
        assert g.orthonormality_error(list(range(b, L // 2, 131))[:64], b) <= 1e-6
        occ = g.occupations(b)
        assert abs(occ.sum() - L // 2) <= 1e-6 * L
        assert occ.min() >= -1e-6 and occ.max() <= 1 + 1e-6


def test_torus160_projective_step_invariants(fm):
    Lx = 160
    L = Lx * Lx
    g = fm.Trajectories(fm.make_params(Lx, Lx, protocol=fm.FM_PROJECTIVE, precision=fm.FM_MIXED, gamma=2.0,
                                       seed=workloads.seed_of("torus160_both"), event_capacity=1 << 16))
    g.step(1)
    ev, dropped = g.take_events()
    assert dropped == 0 and len(ev) > 1500             # about 0.095 L measurements per step
    occ = g.occupations()
    measured = np.array(sorted({e[2] for e in ev}))
    dist = np.minimum(np.abs(occ[measured]), np.abs(occ[measured] - 1.0))
    assert dist.max() <= 1e-5
    assert abs(occ.sum() - L // 2) <= 1e-6 * L
    assert g.orthonormality_error(list(range(0, L // 2, 211))[:64]) <= 1e-6


def test_torus160_homodyne_mutual_information(fm):
    g = fm.Trajectories(fm.make_params(160, 160, protocol=fm.FM_HOMODYNE, precision=fm.FM_MIXED, gamma=1.0,
                                       seed=workloads.seed_of("torus160_both")))
    g.step(4)
    A, B, _ = workloads.torus_blocks()
    I = g.mutual_info(A, B)
    assert I >= -1e-9
    assert g.orthonormality_error(list(range(0, 12800, 199))[:64]) <= 1e-6


def test_ring4096_mixed_against_fp64_gpu_over_60_steps(fm):
    """The mixed path against the all-FP64 GPU path (itself pinned to the oracle)
    over a long run: half-chain EE within the method's 1e-3 bar, C = U U^dag on
    a 256-site block within the per-step bound, and U^dag U = 1 to 1e-6."""
    n = 60
    kw = dict(protocol=fm.FM_HOMODYNE, gamma=1.0, seed=0x2508184685)
    gm = fm.Trajectories(fm.make_params(4096, precision=fm.FM_MIXED, **kw))
    gd = fm.Trajectories(fm.make_params(4096, precision=fm.FM_FP64, **kw))
    gm.step(n)
    gd.step(n)
    half = list(range(2048))
    Sm, Sd = gm.entropy(half), gd.entropy(half)
    Um, Ud = gm.copy_U()[:256], gd.copy_U()[:256]
    dc = float(np.max(np.abs(Um @ Um.conj().T - Ud @ Ud.conj().T)))
    rel = abs(Sm - Sd) / max(abs(Sd), 1.0)
    print("L=4096, %d steps: S mixed %.8f fp64 %.8f rel %.2e, max|dC| (256 block) %.2e" % (n, Sm, Sd, rel, dc))
    assert rel <= 1e-3
    assert dc <= 2e-6 * n
    assert gm.orthonormality_error(list(range(0, 2048, 32))) <= 1e-6


def test_torus160_density_correlation_sum_rule_and_block_covariance(fm):
    """At 160 x 160: -sum_d c[d] = mean n (1 - n) (C^2 = C), c symmetric under d -> -d, and
    the covariance of the two 40 x 40 blocks is non-negative."""
    g = fm.Trajectories(fm.make_params(160, 160, protocol=fm.FM_HOMODYNE, precision=fm.FM_MIXED, gamma=1.0,
                                       seed=workloads.seed_of("torus160_both")))
    g.step(3)
    c = g.density_correlation()
    n = g.occupations()
    assert abs(-np.sum(c) - np.mean(n * (1 - n))) <= 1e-5 * np.mean(n * (1 - n))
    cc = c.reshape(160, 160)                       # [dy, dx]
    flip = np.roll(np.roll(cc[::-1, ::-1], 1, axis=0), 1, axis=1)
    assert np.max(np.abs(cc - flip)) <= 1e-7
    A, B, _ = workloads.torus_blocks()
    assert g.particle_covariance(A, B) >= 0.0


def test_ring16384_entropy_sketch_equals_full_method(fm):
    """The bench's entropy configuration at full size: the half-chain sketch of every
    trajectory of the L = 16384 homodyne batch after 60 steps against the full method on the
    same state (<= 1e-5 of max(S, 1)); the asynchronous sketch equals the synchronous one."""
    L = 16384
    wl = workloads.WORKLOADS["ring16384_homodyne"]
    g = fm.Trajectories(fm.make_params(L, batch=4, protocol=fm.FM_HOMODYNE, precision=fm.FM_MIXED,
                                       seed=workloads.seed_of("ring16384_homodyne")))
    g.set_gammas(wl["gammas"])
    g.step(60)
    half = workloads.half_chain(L)
    g.set_entropy_method(fm.FM_EE_SKETCH)
    sk = [g.entropy(half, b) for b in range(4)]
    tickets = [g.entropy_async(half, b) for b in range(4)]
    assert [g.entropy_wait(t) for t in tickets] == sk
    g.set_entropy_method(fm.FM_EE_FULL)
    full = g.entropy(half, 0)
    print("L=16384 after 60 steps: sketch %s, full (trajectory 0) %.9f" % (sk, full))
    assert abs(sk[0] - full) <= 1e-5 * max(full, 1.0)
    assert all(s > 0.0 for s in sk)
