"""Runtime features on the GPU: CUDA-graph stepping and the continuous-batching server.

Graph replay must reproduce eager stepping bit for bit, and a request's result
must not depend on the requests it is batched with (each slot's arithmetic is
independent of the others), so both are checked for exact equality.
"""
import numpy as np
import pytest

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


@pytest.mark.parametrize("precision,protocol,L,reorth", [(0, 1, 64, 1), (0, 0, 64, 2), (1, 1, 256, 1),
                                                          (1, 0, 512, 3), (0, 2, 64, 2), (1, 2, 256, 1)])
def test_graph_replay_equals_eager(fm, precision, protocol, L, reorth):
    kw = dict(batch=2, protocol=protocol, precision=precision, reorth_interval=reorth, gamma=1.0, seed=4)
    a = fm.Trajectories(fm.make_params(L, **kw))
    b = fm.Trajectories(fm.make_params(L, **kw))
    b.set_graphs(True)
    a.step(3)
    b.step(3)            # one eager step to align, then one graph period, ...
    a.step(11)
    b.step(11)           # ... several replays and an eager remainder
    for t in range(2):
        assert np.array_equal(a.copy_U(t), b.copy_U(t))
    assert a.steps_done(1) == b.steps_done(1) == 14
    assert b.kernel_launches > 0


def test_served_mix_equals_each_request_alone(fm):
    from paper_2508_18468_gb300 import serve
    kinds = [(256, "homodyne"), (512, "projective"), (256, "projective")]
    reqs = [serve.Request(rid=i, L=kinds[i % 3][0], protocol=kinds[i % 3][1], gamma=0.3 + 0.2 * i,
                          traj_id=100 + i, steps=12 + 2 * (i % 2)) for i in range(7)]
    srv = serve.Server(slots=2, memory_budget=8 << 30)
    res, st = srv.run(reqs, realtime=False)
    assert sorted(r.rid for r in res) == list(range(7))
    assert st["step_latency_ms_p99"] >= st["step_latency_ms_p50"] > 0
    for r in res:
        q = reqs[r.rid]
        alone = serve.Server(slots=1, memory_budget=8 << 30)
        (ra,), _ = alone.run([serve.Request(rid=0, L=q.L, protocol=q.protocol, gamma=q.gamma, traj_id=q.traj_id,
                                            steps=q.steps)], realtime=False)
        assert ra.S == r.S, (q, ra.S, r.S)


def test_served_poisson_arrivals_in_real_time_equal_each_request_alone(fm):
    """Requests arriving as a Poisson stream in real time (mean gap 4 ms) while other
    groups run: admitted into free slots of idle groups or new groups, answered by
    asynchronous entropies; each answer equals the request served alone, bit for bit."""
    from paper_2508_18468_gb300 import serve
    rng = np.random.default_rng(5)
    kinds = [(256, "homodyne"), (512, "projective"), (1024, "homodyne"), (256, "projective")]
    t = np.cumsum(rng.exponential(0.004, size=10))
    reqs = [serve.Request(rid=i, L=kinds[i % 4][0], protocol=kinds[i % 4][1], gamma=0.2 + 0.15 * i,
                          traj_id=200 + i, steps=10 + (i % 3), arrival=float(t[i])) for i in range(10)]
    srv = serve.Server(slots=2, memory_budget=16 << 30)
    res, st = srv.run(reqs, realtime=True)
    assert sorted(r.rid for r in res) == list(range(10))
    assert st["latency_samples"] == st["trajectory_steps"] == sum(q.steps for q in reqs)
    assert st["step_latency_ms_p99"] >= st["step_latency_ms_p50"] > 0
    for r in res:
        q = reqs[r.rid]
        assert r.steps == q.steps
        alone = serve.Server(slots=1, memory_budget=8 << 30)
        (ra,), _ = alone.run([serve.Request(rid=0, L=q.L, protocol=q.protocol, gamma=q.gamma, traj_id=q.traj_id,
                                            steps=q.steps)], realtime=False)
        assert ra.S == r.S, (q, ra.S, r.S)


@pytest.mark.parametrize("precision", [0, 1])
def test_async_entropy_sees_the_state_when_requested(fm, precision):
    L = 512 if precision else 96
    kw = dict(batch=2, protocol=1, precision=precision, gamma=0.7, seed=21)
    a = fm.Trajectories(fm.make_params(L, **kw))
    b = fm.Trajectories(fm.make_params(L, **kw))
    half = list(range(L // 2))
    a.step(5)
    b.step(5)
    t0 = a.entropy_async(half, 0)
    t1 = a.entropy_async(list(range(0, L, 3)), 1)
    a.step(7)                                   # the state moves on while the solves run
    ref0 = b.entropy(half, 0)
    ref1 = b.entropy(list(range(0, L, 3)), 1)
    assert a.entropy_wait(t0) == ref0
    assert a.entropy_wait(t1) == ref1
    b.step(7)
    assert np.array_equal(a.copy_U(1), b.copy_U(1))
    assert a.entropy(half, 1) == b.entropy(half, 1)


@pytest.mark.parametrize("precision", [0, 1])
def test_many_async_entropies_interleaved_with_steps(fm, precision):
    """More tickets than C_A buffers, issued between steps (including graph replays),
    each equal to the synchronous entropy of a twin state at the same point."""
    L = 512 if precision else 64
    kw = dict(batch=3, protocol=0, precision=precision, gamma=1.2, seed=33)
    a = fm.Trajectories(fm.make_params(L, **kw))
    b = fm.Trajectories(fm.make_params(L, **kw))
    a.set_graphs(True)
    sites = [list(range(L // 2)), list(range(0, L, 2)), list(range(L // 4, L))]
    tickets, refs, got = [], [], []
    for k in range(9 if precision else 60):        # FP64: more tickets than C_A buffers (64 here)
        for t in range(3):
            if (k + t) % 2 == 0:
                tickets.append(a.entropy_async(sites[(k + t) % 3], t))
                refs.append(b.entropy(sites[(k + t) % 3], t))
        while len(tickets) - len(got) > 40:        # at most 64 results may be outstanding
            got.append(a.entropy_wait(tickets[len(got)]))
        a.step(2)
        b.step(2)
    got += [a.entropy_wait(t) for t in tickets[len(got):]]
    assert len(got) > 4
    assert got == refs
    for t in range(3):
        assert np.array_equal(a.copy_U(t), b.copy_U(t))


def test_tile_configurations_give_identical_states(fm):
    """Every output element is one fixed-order K sum whatever the tile shape, so
    the tile width and raster groups do not change a single bit."""
    kw = dict(batch=2, protocol=1, precision=1, gamma=0.8, seed=7)
    ref = fm.Trajectories(fm.make_params(1024, **kw))
    ref.step(5)
    for tc in (1 | (2 << 2), 2 | (4 << 2), 1 | (3 << 2)):
        g = fm.Trajectories(fm.make_params(1024, tile_config=tc, **kw))
        g.step(5)
        for t in range(2):
            assert np.array_equal(g.copy_U(t), ref.copy_U(t)), tc


def test_cholesky_chains_give_identical_states(fm):
    """One first-pass Cholesky chain per trajectory (tile_config bit 7, three streams here)
    against two halves of the batch: every factor is one trajectory's and every product
    tile one fixed-order sum in any tile order, so not a bit changes (N = 1024: the
    recursion's products of 512 and 256 run in the paired and Hermitian tile orders)."""
    kw = dict(batch=3, protocol=1, precision=1, gamma=0.8, seed=9, reorth_interval=2)
    ref = fm.Trajectories(fm.make_params(2048, **kw))
    ref.step(5)
    g = fm.Trajectories(fm.make_params(2048, tile_config=1 << 7, **kw))
    g.step(5)
    for t in range(3):
        assert np.array_equal(g.copy_U(t), ref.copy_U(t)), t


def test_autotune_picks_a_configuration_that_meets_the_bar(fm):
    p = fm.make_params(512, batch=2, protocol=1, precision=1, gamma=1.0, seed=3)
    res = fm.autotune(p, steps=2, max_reorth=2, ortho_tol=1e-6)
    # widths 128/256 x groups 8/16/32 x reorth 1, 2, then the two other drain intervals of the
    # winner when its interval is 2
    assert res["tried"] == 2 * 3 * 2 + (2 if res["reorth_interval"] == 2 else 0)
    assert res["reorth_interval"] in (1, 2)
    assert res["ms_per_step"] > 0
    assert res["ortho_err"] <= 1e-6
    q = fm.make_params(512, batch=2, protocol=1, precision=1, gamma=1.0, seed=3,
                       tile_config=res["tile_config"], reorth_interval=res["reorth_interval"])
    g = fm.Trajectories(q)
    g.step(4)
    assert g.orthonormality_error(list(range(0, 256, 8))) <= 1e-6


def test_graphs_with_banded_propagation_equal_eager(fm):
    kw = dict(batch=2, protocol=1, precision=1, gamma=0.9, seed=8)
    a = fm.Trajectories(fm.make_params(512, **kw))
    b = fm.Trajectories(fm.make_params(512, **kw))
    for g in (a, b):
        g.set_propagation(fm.FM_PROP_BANDED)
    b.set_graphs(True)
    a.step(9)
    b.step(9)
    for t in range(2):
        assert np.array_equal(a.copy_U(t), b.copy_U(t))


def test_group_graph_advances_uneven_lattices_bit_identically(fm):
    """Batches of different L, protocol and precision advanced by one CUDA graph (fm_group):
    after two replays of the group period each state equals a twin stepped alone, bit for
    bit; the period is the lcm of the members' 2 reorth_interval; a step count that is not a
    multiple of it is refused; a member's propagation change re-captures the graph."""
    specs = [dict(Lx=256, batch=2, protocol=1, precision=1, reorth_interval=1, gamma=0.7, seed=61),
             dict(Lx=512, batch=3, protocol=1, precision=1, reorth_interval=2, gamma=1.1, seed=62),
             dict(Lx=1024, batch=1, protocol=2, precision=1, reorth_interval=1, gamma=0.5, seed=63),
             dict(Lx=64, batch=64, protocol=0, precision=0, reorth_interval=1, gamma=0.9, seed=64)]

    def make(sp):
        sp = dict(sp)
        return fm.Trajectories(fm.make_params(sp.pop("Lx"), **sp))
    members = [make(sp) for sp in specs]
    twins = [make(sp) for sp in specs]
    grp = fm.Group(members)
    assert grp.period == 4
    with pytest.raises(fm.FmError):
        grp.step(6)
    for g in members + twins:
        g.step(4)
    l0 = [m.kernel_launches for m in members]
    grp.step(8)
    for t in twins:
        t.step(8)
    for m, t, sp in zip(members, twins, specs):
        assert m.steps_done(0) == t.steps_done(0) == 12
        assert m.kernel_launches > l0[members.index(m)]
        for b in range(sp["batch"] if sp["batch"] < 4 else 2):
            assert np.array_equal(m.copy_U(b), t.copy_U(b)), sp
    # a member's configuration changes: the group graph is captured again
    members[0].set_propagation(fm.FM_PROP_BANDED)
    twins[0].set_propagation(fm.FM_PROP_BANDED)
    grp.step(4)
    twins[0].step(4)
    assert np.array_equal(members[0].copy_U(1), twins[0].copy_U(1))
    grp.close()
    # a state whose steps read counts back cannot join a group
    bad = fm.Trajectories(fm.make_params(256, batch=2, protocol=0, precision=1, gamma=0.5, seed=65))
    with pytest.raises(fm.FmError):
        fm.Group([bad])
