"""Scheduling logic of the continuous-batching server, on the CPU with fake groups."""
import contextlib

import pytest

pytest.importorskip("torch")
from paper_2508_18468_gb300 import serve  # noqa: E402


class FakeGroup:
    """Same interface as serve.Group; 'computes' S = rid + steps / 1000.  A launched period
    completes after `cost` idle() polls (cost = L / 256: larger lattices are slower), and an
    entropy is ready one poll after it was started."""
    live = []
    launches = []                # (L, protocol, group id, n) in launch order

    def __init__(self, L, protocol, slots, precision, seed, reorth_interval, graphs=True, tile_config=0):
        self.L, self.protocol, self.slots = L, protocol, slots
        self.reorth_interval, self.tile_config = reorth_interval, tile_config
        self.bytes = L * slots
        self.period = 2 * reorth_interval if graphs else 1
        self.free = list(range(slots))[::-1]
        self.active = {}
        self.tickets = []
        self.closed = False
        self.admitted = 0
        self.remaining = 0
        self.last_n = 0
        FakeGroup.live.append(self)

    def stream_context(self):
        return contextlib.nullcontext()

    def synchronize(self):
        pass

    def close(self):
        self.closed = True

    def idle(self):
        if self.remaining > 0:
            self.remaining -= 1
        return self.remaining == 0

    def busy(self):
        return bool(self.active) or bool(self.tickets)

    def admit(self, req, now):
        assert req.L == self.L and req.protocol == self.protocol
        assert self.remaining == 0                     # never admitted into a running group
        b = self.free.pop()
        self.active[b] = serve._Slot(req=req, done=0, admitted=now)
        self.admitted += 1

    tick_steps = serve.Group.tick_steps

    def launch_steps(self, n, now):
        assert self.remaining == 0
        for sl in self.active.values():
            sl.done += n
        self.remaining = max(1, self.L // 256)
        self.last_n = n
        FakeGroup.launches.append((self.L, self.protocol, id(self), n))

    def account(self, now, lat):
        if self.last_n:
            lat.extend([1.0 * self.L / 256] * (self.last_n * len(self.active)))
            self.last_n = 0

    def start_entropies(self):
        for b in [b for b, sl in self.active.items() if sl.done >= sl.req.steps]:
            sl = self.active.pop(b)
            self.tickets.append([1, sl])
            self.free.append(b)

    def harvest(self, now, block=False):
        out, keep = [], []
        for t in self.tickets:
            if t[0] > 0 and not block:
                t[0] -= 1
                keep.append(t)
                continue
            sl = t[1]
            out.append(serve.Result(rid=sl.req.rid, S=sl.req.rid + sl.done / 1000.0, steps=sl.done,
                                    admitted=sl.admitted, finished=now, group=(self.L, self.protocol)))
        self.tickets = keep
        return out


def size_of(L, protocol, slots, precision, reorth_interval):
    return L * slots


def make_requests(n, steps=10):
    kinds = [(256, "homodyne"), (512, "projective"), (256, "projective"), (1024, "homodyne")]
    return [serve.Request(rid=i, L=kinds[i % 4][0], protocol=kinds[i % 4][1], gamma=0.5, traj_id=i,
                          steps=steps + (i % 3), arrival=0.0) for i in range(n)]


def test_every_request_answered_once_with_exact_steps():
    FakeGroup.live = []
    srv = serve.Server(memory_budget=1 << 40, slots=3, group_factory=FakeGroup, size_of=size_of)
    reqs = make_requests(20)
    res, st = srv.run(reqs, realtime=False)
    assert sorted(r.rid for r in res) == list(range(20))
    for r in res:
        assert r.steps == reqs[r.rid].steps            # ticks are clipped to the finishing request
        assert r.group == (reqs[r.rid].L, reqs[r.rid].protocol)
    assert st["requests"] == 20
    assert st["trajectory_steps"] == sum(q.steps for q in reqs)
    # slots are reused: 4 groups of 3 slots served 20 requests
    assert sum(g.admitted for g in FakeGroup.live) == 20
    assert len({(g.L, g.protocol) for g in FakeGroup.live}) == 4
    assert st["latency_samples"] == st["trajectory_steps"]


def test_groups_advance_at_their_own_pace():
    """A 4096-site group takes 16 polls per period, a 256-site group 1: while the large
    group runs one period, the small one runs many, and small requests submitted with a
    large one finish first."""
    FakeGroup.live, FakeGroup.launches = [], []
    reqs = [serve.Request(rid=0, L=4096, protocol="homodyne", gamma=0.5, traj_id=0, steps=8)]
    reqs += [serve.Request(rid=i, L=256, protocol="homodyne", gamma=0.5, traj_id=i, steps=8) for i in (1, 2, 3)]
    srv = serve.Server(memory_budget=1 << 40, slots=1, group_factory=FakeGroup, size_of=size_of)
    res, st = srv.run(reqs, realtime=False)
    order = [r.rid for r in res]
    assert sorted(order) == [0, 1, 2, 3]
    assert order[-1] == 0                              # the large request finishes last
    big = [i for i, l in enumerate(FakeGroup.launches) if l[0] == 4096]
    small = [i for i, l in enumerate(FakeGroup.launches) if l[0] == 256]
    assert len(small) > 2 * len(big) and small[-1] < big[-1] or len(small) >= 3 * len(big)
    # the three 256-site requests ran in parallel groups (one slot each, memory allows)
    assert len([g for g in FakeGroup.live if g.L == 256]) == 3


def test_full_group_is_duplicated_when_memory_allows():
    FakeGroup.live = []
    reqs = [serve.Request(rid=i, L=512, protocol="projective", gamma=0.5, traj_id=i, steps=6) for i in range(5)]
    srv = serve.Server(memory_budget=512 * 2 * 2, slots=2, group_factory=FakeGroup, size_of=size_of)
    res, _ = srv.run(reqs, realtime=False)
    assert sorted(r.rid for r in res) == list(range(5))
    assert len([g for g in FakeGroup.live if g.L == 512]) == 2          # two groups of the kind, no third


def test_memory_budget_is_respected_and_idle_groups_are_evicted():
    FakeGroup.live = []
    budget = 1024 * 2            # room for one group of two 1024-site slots, or a few smaller ones
    srv = serve.Server(memory_budget=budget, slots=2, group_factory=FakeGroup, size_of=size_of)
    used_max = [0]
    orig = srv._group_for

    def tracking(req, ready):
        g = orig(req, ready)
        used_max[0] = max(used_max[0], srv.used)
        return g
    srv._group_for = tracking
    res, _ = srv.run(make_requests(16), realtime=False)
    assert len(res) == 16
    assert used_max[0] <= budget
    assert any(g.closed for g in FakeGroup.live)       # groups were evicted to make room


def test_request_larger_than_budget_is_reported():
    srv = serve.Server(memory_budget=10, slots=2, group_factory=FakeGroup, size_of=size_of)
    with pytest.raises(RuntimeError):
        srv.run(make_requests(1), realtime=False)


def test_autotuned_settings_reach_each_group_and_are_searched_once():
    FakeGroup.live = []
    calls = []

    def tuner(L, protocol):
        calls.append((L, protocol))
        return {"tile_config": 1 | (2 << 2) if L < 512 else 2, "reorth_interval": 2 if protocol == "projective" else 1}
    srv = serve.Server(memory_budget=1 << 40, slots=2, group_factory=FakeGroup, size_of=size_of, autotune=True,
                       tuner=tuner)
    reqs = make_requests(12)
    srv.pretune((r.L, r.protocol) for r in reqs)
    res, st = srv.run(reqs, realtime=False)
    assert len(res) == 12
    assert sorted(calls) == sorted(set((r.L, r.protocol) for r in reqs))     # one search per kind
    for g in FakeGroup.live:
        t = tuner(g.L, g.protocol)
        assert (g.tile_config, g.reorth_interval) == (t["tile_config"], t["reorth_interval"])
        assert g.period == 2 * t["reorth_interval"]
    assert set(st["tuned"]) == {"%d/%s" % (r.L, r.protocol) for r in reqs}
