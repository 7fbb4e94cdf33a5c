"""The entropy sketch (FM_EE_SKETCH) against the full method and the FP64 references
(needs a GB300).

The sketch computes S_A from the singular values of the cross block C_AB (Sec. II:
lambda (1 - lambda) = sigma^2 for a projector C).  Bars: against the full method on the
same mixed-precision state, |dS| <= 1e-5 max(S, 1 nat) (both see the same float state;
the sketch drops sigma^2 below ~1e-9); against the FP64 GPU path or the FP64 oracle, the
method's 1e-3 bar.
"""
import numpy as np
import pytest

from oracle import observables, trajectory
from oracle.trajectory import HOMODYNE, PROJECTIVE, Params

pytestmark = pytest.mark.gpu

REL_FULL = 1e-5


@pytest.fixture(scope="module")
def fm():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2508_18468_gb300 import build
    build.build()
    from paper_2508_18468_gb300 import fm as mod
    return mod


def rel(a, b):
    return abs(a - b) / max(abs(b), 1.0)


def both(fm, g, sites, b=0):
    g.set_entropy_method(fm.FM_EE_FULL)
    full = g.entropy(sites, b)
    g.set_entropy_method(fm.FM_EE_SKETCH)
    sk = g.entropy(sites, b)
    return sk, full, g.entropy_sketch_info()


@pytest.mark.parametrize("protocol,gamma,steps", [(1, 0.3, 10), (1, 1.0, 150), (0, 0.5, 60), (0, 2.0, 20)])
def test_sketch_equals_full_method_ring2048(fm, protocol, gamma, steps):
    g = fm.Trajectories(fm.make_params(2048, batch=2, protocol=protocol, precision=fm.FM_MIXED, gamma=gamma,
                                       seed=61))
    g.step(steps)
    for sites in (list(range(1024)), list(range(300, 1100)), list(range(400)) + list(range(1200, 1600))):
        sk, full, (rank, chk, fb) = both(fm, g, sites, 1)
        print("protocol %d gamma %.1f steps %d |A| %d: S sketch %.10f full %.10f rel %.1e rank %d chk %.1e"
              % (protocol, gamma, steps, len(sites), sk, full, rel(sk, full), rank, chk))
        assert not fb and rank >= 128
        assert rel(sk, full) <= REL_FULL


def test_sketch_against_fp64_oracle_ring1024(fm):
    n = 40
    po = Params(Lx=1024, gamma=0.7, protocol=HOMODYNE, seed=71)
    g = fm.Trajectories(fm.make_params(1024, protocol=fm.FM_HOMODYNE, precision=fm.FM_MIXED, gamma=0.7, seed=71))
    g.step(n)
    g.set_entropy_method(fm.FM_EE_SKETCH)
    U = trajectory.run(po, n)["U"]
    for sites in (list(range(512)), list(range(200, 712))):
        S = g.entropy(sites)
        S_ref = observables.entanglement_entropy(U, sites)
        print("L=1024 |A|=%d: sketch %.9f oracle %.9f rel %.1e" % (len(sites), S, S_ref, rel(S, S_ref)))
        assert rel(S, S_ref) <= 1e-4
        assert not g.entropy_sketch_info()[2]


def test_sketch_mutual_information_torus(fm):
    """MI of two 24 x 24 blocks of a 48 x 48 torus (non-contiguous site lists) and the
    half-torus strip: the sketch equals the full method."""
    g = fm.Trajectories(fm.make_params(48, 48, protocol=fm.FM_HOMODYNE, precision=fm.FM_MIXED, gamma=1.0, seed=5))
    g.step(8)
    A = [x + 48 * y for y in range(24) for x in range(24)]
    B = [x + 48 * y for y in range(24) for x in range(24, 48)]
    strip = [x + 48 * y for y in range(48) for x in range(24)]
    g.set_entropy_method(fm.FM_EE_FULL)
    I_full, S_full = g.mutual_info(A, B), g.entropy(strip)
    g.set_entropy_method(fm.FM_EE_SKETCH)
    I_sk, S_sk = g.mutual_info(A, B), g.entropy(strip)
    print("torus 48: MI sketch %.9f full %.9f; strip S %.9f %.9f" % (I_sk, I_full, S_sk, S_full))
    assert abs(I_sk - I_full) <= REL_FULL * max(abs(I_full), 1.0) * 3
    assert rel(S_sk, S_full) <= REL_FULL


def test_sketch_falls_back_on_a_high_rank_state(fm):
    """A random orthonormal U (volume law: every sigma is O(1)) has full numerical rank, so
    the sketch cannot converge within its rank cap and the full method runs: the result is
    the full method's, bit for bit, synchronously and asynchronously."""
    L, N = 2048, 1024
    rng = np.random.default_rng(3)
    Q, _ = np.linalg.qr(rng.standard_normal((L, N)) + 1j * rng.standard_normal((L, N)))
    g = fm.Trajectories(fm.make_params(L, protocol=fm.FM_HOMODYNE, precision=fm.FM_MIXED, gamma=1.0, seed=9))
    g.set_U(Q)
    half = list(range(N))
    sk, full, (rank, chk, fb) = both(fm, g, half)
    assert fb and rank == 0 and chk > 1e-9
    assert sk == full
    t = g.entropy_async(half)
    assert g.entropy_wait(t) == full


def test_async_sketch_equals_sync_sketch(fm):
    """Tickets issued between steps (more than the four C_A buffers) return the synchronous
    sketch of a twin state, bit for bit."""
    kw = dict(protocol=fm.FM_HOMODYNE, precision=fm.FM_MIXED, gamma=0.6, seed=13, batch=2)
    a = fm.Trajectories(fm.make_params(2048, **kw))
    b = fm.Trajectories(fm.make_params(2048, **kw))
    for g in (a, b):
        g.set_entropy_method(fm.FM_EE_SKETCH)
    sites = list(range(1024))
    tickets, ref = [], []
    for k in range(6):
        a.step(3)
        b.step(3)
        tickets.append(a.entropy_async(sites, k % 2))
        ref.append(b.entropy(sites, k % 2))
    got = [a.entropy_wait(t) for t in tickets]
    assert got == ref


def test_sketch_method_needs_mixed_precision(fm):
    g = fm.Trajectories(fm.make_params(64, precision=fm.FM_FP64))
    with pytest.raises(fm.FmError):
        g.set_entropy_method(fm.FM_EE_SKETCH)
    g2 = fm.Trajectories(fm.make_params(256, precision=fm.FM_MIXED, protocol=fm.FM_HOMODYNE))
    with pytest.raises(fm.FmError):
        g2.set_entropy_method(7)
    # small subsystems take the full method
    g2.set_entropy_method(fm.FM_EE_SKETCH)
    g2.step(2)
    s = g2.entropy(list(range(64)))
    assert g2.entropy_sketch_info()[2]
    g2.set_entropy_method(fm.FM_EE_FULL)
    assert g2.entropy(list(range(64))) == s


def test_auto_method_picks_by_size(fm):
    """FM_EE_AUTO: the sketch for subsystems (and complements) of 1024 sites or more, the
    full method below; each result equals that method's."""
    g = fm.Trajectories(fm.make_params(4096, protocol=fm.FM_HOMODYNE, precision=fm.FM_MIXED, gamma=0.5, seed=19))
    g.step(20)
    big, small = list(range(2048)), list(range(700))
    g.set_entropy_method(fm.FM_EE_SKETCH)
    s_big = g.entropy(big)
    g.set_entropy_method(fm.FM_EE_FULL)
    f_small = g.entropy(small)
    g.set_entropy_method(fm.FM_EE_AUTO)
    assert g.entropy(big) == s_big and not g.entropy_sketch_info()[2]
    assert g.entropy(small) == f_small and g.entropy_sketch_info()[2]
