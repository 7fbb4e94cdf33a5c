"""The mixed path against the all-FP64 GPU path at the sizes the headline figure is
quoted at, and at the ill-conditioned end of the second CholeskyQR pass (needs a GB300).

The FP64 reference here is the library's FP64 path (complex128 state, FP64 products,
FP64 Cholesky), itself pinned to the oracle at small L (test_gpu_fp64.py), run with two
settings that change its result only at the 1e-14 level and make long runs affordable:
the propagation as stencils of the circulant propagator (every tap above 1e-15 kept;
equal to the dense product to that level, test_gpu_fp64.py) and one FP64 CholeskyQR pass
per step (a float64 pass leaves U^dag U - 1 at ~kappa^2 1e-16; the test checks <= 1e-12).
The mixed side runs as the benchmark does at L = 16384 (dense split-fp16 propagation, the first
CholeskyQR pass every step, the second every reorth_interval steps of the workload) and with
the second pass every step elsewhere unless the test says otherwise.

Bars (the method's): half-chain entropy relative error |dS| / max(S, 1) <= 1e-3;
C = U U^dag on a block of rows within 2e-6 per step (the per-step bound of the mixed
arithmetic, test_gpu_mixed.py); U^dag U = 1 to 1e-6.
"""
import numpy as np
import pytest

from paper_2508_18468_gb300 import workloads

pytestmark = pytest.mark.gpu

S_REL = 1e-3
PER_STEP_C = 2e-6
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


def fp64_reference(fm, Lx, Ly=1, **kw):
    g = fm.Trajectories(fm.make_params(Lx, Ly, precision=fm.FM_FP64, reorth_interval=1 << 30, **kw))
    g.set_propagation(fm.FM_PROP_BANDED)
    return g


def cblock(U, rows):
    Ub = U[rows]
    return Ub @ Ub.conj().T


def srel(a, b):
    return abs(a - b) / max(abs(b), 1.0)


def sample_cols(N):
    return list(range(0, N, max(1, N // 64)))[:64]


def compare(gm, gd, n, sites, rows, label):
    Sm, Sd = gm.entropy(sites), gd.entropy(sites)
    dc = float(np.max(np.abs(cblock(gm.copy_U(), rows) - cblock(gd.copy_U(), rows))))
    om, od = gm.orthonormality_error(sample_cols(gm.N)), gd.orthonormality_error(sample_cols(gd.N))
    print("%s after %d steps: S mixed %.9f fp64 %.9f rel %.2e; max|dC| %.2e; ortho mixed %.1e fp64 %.1e"
          % (label, n, Sm, Sd, srel(Sm, Sd), dc, om, od))
    assert srel(Sm, Sd) <= S_REL
    assert dc <= PER_STEP_C * n
    assert om <= ORTHO
    assert od <= 1e-12
    return Sm, Sd


def test_ring16384_mixed_vs_fp64(fm):
    """The benchmark's lattice and protocol (ring L = 16384, N = 8192, homodyne, dt = 0.05),
    its trajectory with gamma = 1.0, 8 steps: products K = 2L = 32768 deep, the depth no
    smaller lattice reaches.  Both entropy methods of the mixed path (the sketch the
    benchmark uses at this size, and the full eigen-decomposition) against FP64."""
    L, n = 16384, 8
    wl = workloads.WORKLOADS["ring16384_homodyne"]
    seed = workloads.seed_of("ring16384_homodyne")
    kw = dict(protocol=fm.FM_HOMODYNE, gamma=1.0, seed=seed, traj_id=2)
    gm = fm.Trajectories(fm.make_params(L, precision=fm.FM_MIXED, reorth_interval=wl["reorth_interval"],
                                        tile_config=wl["tile_config"], **kw))
    gm.step(n)
    gd = fp64_reference(fm, L, **kw)
    gd.step(n)
    half = workloads.half_chain(L)
    gm.set_entropy_method(fm.FM_EE_AUTO)
    Sm_sketch, Sd = compare(gm, gd, n, half, list(range(512)), "ring L=16384 (sketch entropy)")
    gm.set_entropy_method(fm.FM_EE_FULL)
    Sm_full = gm.entropy(half)
    print("full-method mixed entropy %.9f rel %.2e" % (Sm_full, srel(Sm_full, Sd)))
    assert srel(Sm_full, Sd) <= S_REL
    checks, extra, mx = gm.reorth_stats()
    print("second-pass guard: %d checks, %d extra passes, max |diag E| %.2e, max |offdiag E| %.2e"
          % (checks, extra, mx[0], mx[1]))
    assert checks == n // wl["reorth_interval"]


def test_ring16384_tuned_interval_against_every_step_over_100_steps(fm):
    """The benchmark's second-pass interval (every 8 steps, fm_autotune's choice for this batch)
    against the second pass every step, ring L = 16384, gamma = 1.0: the half-chain entropy every
    25 steps up to 100 within the method's bar, and U^dag U = 1 to 1e-6 at the end."""
    L = 16384
    wl = workloads.WORKLOADS["ring16384_homodyne"]
    k = wl["reorth_interval"]
    assert k > 1
    kw = dict(protocol=fm.FM_HOMODYNE, precision=fm.FM_MIXED, gamma=1.0, seed=workloads.seed_of("ring16384_homodyne"),
              traj_id=2)
    ga = fm.Trajectories(fm.make_params(L, reorth_interval=k, tile_config=wl["tile_config"], **kw))
    gb = fm.Trajectories(fm.make_params(L, reorth_interval=1, **kw))
    half = workloads.half_chain(L)
    for g in (ga, gb):
        g.set_entropy_method(fm.FM_EE_AUTO)
    for t in range(25, 101, 25):
        ga.step(25)
        gb.step(25)
        Sa, Sb = ga.entropy(half), gb.entropy(half)
        print("ring L=16384 step %d: S (second pass every %d) %.9f, every step %.9f, rel %.2e"
              % (t, k, Sa, Sb, srel(Sa, Sb)))
        assert srel(Sa, Sb) <= S_REL
    assert ga.orthonormality_error(sample_cols(L // 2)) <= ORTHO


def test_ring8192_mixed_vs_fp64_over_100_steps(fm):
    """A long horizon at K = 2L = 16384: ring L = 8192, homodyne gamma = 1.0, the half-chain
    entropy of both paths every 25 steps up to 100, then C on a 512-row block."""
    L, n, every = 8192, 100, 25
    kw = dict(protocol=fm.FM_HOMODYNE, gamma=1.0, seed=0x2508184686)
    gm = fm.Trajectories(fm.make_params(L, precision=fm.FM_MIXED, **kw))
    gd = fp64_reference(fm, L, **kw)
    gm.set_entropy_method(fm.FM_EE_AUTO)
    half = workloads.half_chain(L)
    for t in range(every, n + 1, every):
        gm.step(every)
        gd.step(every)
        if t < n:
            Sm, Sd = gm.entropy(half), gd.entropy(half)
            print("ring L=8192 step %d: S mixed %.9f fp64 %.9f rel %.2e" % (t, Sm, Sd, srel(Sm, Sd)))
            assert srel(Sm, Sd) <= S_REL
    compare(gm, gd, n, half, list(range(512)), "ring L=8192")


def test_torus160_mixed_vs_fp64(fm):
    """The 160 x 160 torus (L = 25600, N = 12800: the automatic 256-wide tiles), homodyne
    gamma = 1.0, 2 steps: the mutual information of the two 40 x 40 blocks, each block's
    entropy, and C on 512 rows against FP64."""
    n = 2
    kw = dict(protocol=fm.FM_HOMODYNE, gamma=1.0, seed=workloads.seed_of("torus160_both"))
    gm = fm.Trajectories(fm.make_params(160, 160, precision=fm.FM_MIXED, **kw))
    gm.step(n)
    gd = fp64_reference(fm, 160, 160, **kw)
    gd.step(n)
    A, B, _ = workloads.torus_blocks()
    Im, Id = gm.mutual_info(A, B), gd.mutual_info(A, B)
    print("torus 160x160 after %d steps: MI mixed %.3e fp64 %.3e" % (n, Im, Id))
    assert abs(Im - Id) <= S_REL * max(abs(Id), 1.0)
    compare(gm, gd, n, A, list(range(512)), "torus 160x160 block A")


@pytest.mark.parametrize("reorth", [1, 4])
def test_homodyne_gamma2_ring4096_ill_conditioned(fm, reorth):
    """The ill-conditioned end of the first CholeskyQR pass: homodyne gamma = 2 (weights
    exp(sqrt(0.1) xi + ...), the widest spread of the configurations), second pass every
    `reorth` steps, 64 steps, against FP64; the second-pass guard's measurements printed."""
    L, n = 4096, 64
    kw = dict(protocol=fm.FM_HOMODYNE, gamma=2.0, seed=0x2508184687)
    gm = fm.Trajectories(fm.make_params(L, precision=fm.FM_MIXED, reorth_interval=reorth, **kw))
    gm.step(n)
    gd = fp64_reference(fm, L, **kw)
    gd.step(n)
    compare(gm, gd, n, workloads.half_chain(L), list(range(256)), "gamma=2 L=4096 reorth %d" % reorth)
    checks, extra, mx = gm.reorth_stats()
    print("second-pass guard: %d checks, %d extra passes, max |diag E| %.2e, max |offdiag E| %.2e, after extra "
          "%.2e %.2e" % (checks, extra, mx[0], mx[1], mx[2], mx[3]))
    assert checks == n // reorth


def test_projective_reorth8_ring4096_forced_to_fp64_outcomes(fm):
    """Projective gamma = 0.5 with CholeskyQR2 only every 8 steps (rank-1 updates in float
    between them), 64 steps, the mixed run held on the FP64 run's outcome sequence
    (fm_force_outcomes), so that a near tie cannot send the two down different branches."""
    L, n = 4096, 64
    kw = dict(protocol=fm.FM_PROJECTIVE, gamma=0.5, seed=0x2508184688, reorth_interval=8, event_capacity=1 << 15)
    gd = fm.Trajectories(fm.make_params(L, precision=fm.FM_FP64, **kw))
    gd.step(n)
    ev_d, dropped = gd.take_events()
    assert dropped == 0 and len(ev_d) > 50 * n
    gm = fm.Trajectories(fm.make_params(L, precision=fm.FM_MIXED, **kw))
    gm.force_outcomes(ev_d)
    gm.step(n)
    ev_m, dropped = gm.take_events()
    assert dropped == 0
    assert sorted((e[1], e[2], e[5]) for e in ev_m) == sorted((e[1], e[2], e[5]) for e in ev_d)
    natural = sum(1 for e in ev_m if e[3] >= 0.0 and e[3] <= 1.0)
    assert natural == 0                                    # every measurement came from the list
    half = workloads.half_chain(L)
    Sm, Sd = gm.entropy(half), gd.entropy(half)
    dc = float(np.max(np.abs(cblock(gm.copy_U(), list(range(256))) - cblock(gd.copy_U(), list(range(256))))))
    om = gm.orthonormality_error(sample_cols(L // 2))
    print("projective reorth 8, L=4096, %d steps, %d events: S mixed %.9f fp64 %.9f rel %.2e, max|dC| %.2e, "
          "ortho %.1e" % (n, len(ev_d), Sm, Sd, srel(Sm, Sd), dc, om))
    assert srel(Sm, Sd) <= S_REL
    assert dc <= PER_STEP_C * n
    assert om <= ORTHO
