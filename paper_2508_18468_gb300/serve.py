"""Continuous-batching server for monitored-trajectory jobs on one GPU.

A request asks for one trajectory: lattice size L (ring), protocol, monitoring
rate gamma, trajectory id and a number of steps; the answer is the half-chain
entanglement entropy at the end.  Requests of equal (L, protocol) share an
``fm_state`` whose batch slots are reused as requests finish
(``fm_reset_trajectory``); when every state of a kind is full and the memory
budget allows, another state of that kind is opened.  Each state (a group)
steps on its own CUDA stream, replaying a CUDA graph of its step period, and
advances at its own pace: the serving loop polls each group's completion event
and, as soon as a group is idle, starts the entropies of the requests that just
finished (``fm_entropy_async``, eigen-solved by library threads), admits
waiting requests into free slots and launches the group's next period -- no
group waits for another, so a ring of 256 sites is not held to the pace of a
ring of 4096.  A new group is created only if its workspace fits the memory
budget (admission by HBM footprint); otherwise the request waits for a slot.

Latency is recorded per request step: each period a request takes part in
contributes (completion - launch) / steps for each of its steps.

Per-trajectory results do not depend on the company a request keeps: every
slot's computation is independent of the others (tests check this).  With
``reorth_interval > 1`` the second re-orthonormalisation pass follows the
group's step count, so results then agree only within the mixed-precision
tolerance rather than bitwise.

With ``autotune=True`` each (L, protocol) group takes the tile configuration
and re-orthonormalisation interval that ``fm_autotune`` measures fastest for
its slot count under the orthonormality bar; ``pretune`` runs those searches
before serving so that no request waits for one.
"""
import collections
import time
from dataclasses import dataclass, field

import numpy as np

from . import fm, workloads


@dataclass
class Request:
    rid: int
    L: int
    protocol: str           # "projective" or "homodyne"
    gamma: float
    traj_id: int
    steps: int
    arrival: float = 0.0    # seconds after the server starts


@dataclass
class Result:
    rid: int
    S: float
    steps: int
    admitted: float
    finished: float
    group: tuple


@dataclass
class _Slot:
    req: Request
    done: int = 0
    admitted: float = 0.0


def workspace_bytes(L, protocol, slots, precision, reorth_interval):
    prot = fm.FM_HOMODYNE if protocol == "homodyne" else fm.FM_PROJECTIVE
    return fm.fm_workspace_bytes(fm.make_params(L, batch=slots, protocol=prot, precision=precision,
                                                reorth_interval=reorth_interval))


class Group:
    """One fm_state of `slots` trajectories of the same (L, protocol), on its own stream."""

    def __init__(self, L, protocol, slots, precision, seed, reorth_interval, graphs=True, tile_config=0):
        import torch
        self.L, self.protocol, self.slots = L, protocol, slots
        prot = fm.FM_HOMODYNE if protocol == "homodyne" else fm.FM_PROJECTIVE
        self.params = fm.make_params(L, batch=slots, protocol=prot, precision=precision,
                                     reorth_interval=reorth_interval, gamma=0.0, seed=seed,
                                     tile_config=tile_config)
        self.bytes = fm.fm_workspace_bytes(self.params)
        self.period = 2 * reorth_interval if graphs else 1
        self.stream = torch.cuda.Stream()
        with torch.cuda.stream(self.stream):
            self.traj = fm.Trajectories(self.params, stream=self.stream)
        if graphs:
            self.traj.set_graphs(True)
        self.free = list(range(slots))[::-1]
        self.active = {}
        self.tickets = []            # (ticket, slot record) of entropies in flight
        self.half = workloads.half_chain(L)
        self.done_event = None       # completion of the last launched period
        self.launched_at = 0.0
        self.last_n = 0

    def stream_context(self):
        import torch
        return torch.cuda.stream(self.stream)

    def synchronize(self):
        self.stream.synchronize()

    def close(self):
        self.traj.close()

    def idle(self):
        """True when the last launched period has completed (never blocks)."""
        return self.done_event is None or self.done_event.query()

    def busy(self):
        return bool(self.active) or bool(self.tickets)

    def admit(self, req, now):
        b = self.free.pop()
        self.traj.reset_trajectory(b, req.traj_id, req.gamma)
        self.active[b] = _Slot(req=req, done=0, admitted=now)

    def tick_steps(self):
        """Steps for the next launch: one graph period, clipped to the nearest finishing request."""
        rem = min(sl.req.steps - sl.done for sl in self.active.values())
        return max(1, min(self.period, rem))

    def launch_steps(self, n, now):
        import torch
        with self.stream_context():
            self.traj.step(n)
            self.done_event = torch.cuda.Event()
            self.done_event.record(self.stream)
        self.launched_at = now
        self.last_n = n
        for sl in self.active.values():
            sl.done += n

    def account(self, now, lat):
        """After a launched period completed: per-step latency of every request in it."""
        if self.last_n:
            per = (now - self.launched_at) * 1e3 / self.last_n
            lat.extend([per] * (self.last_n * len(self.active)))
            self.last_n = 0

    def start_entropies(self):
        """Finished requests: their entropies start (library threads) and their slots free up."""
        for b in [b for b, sl in self.active.items() if sl.done >= sl.req.steps]:
            sl = self.active.pop(b)
            self.tickets.append((self.traj.entropy_async(self.half, b), sl))
            self.free.append(b)

    def harvest(self, now, block=False):
        out, keep = [], []
        for t, sl in self.tickets:
            if block or self.traj.entropy_ready(t):
                out.append(Result(rid=sl.req.rid, S=self.traj.entropy_wait(t), steps=sl.done,
                                  admitted=sl.admitted, finished=now, group=(self.L, self.protocol)))
            else:
                keep.append((t, sl))
        self.tickets = keep
        return out


class Server:
    """Admit, step and retire requests until all are answered."""

    def __init__(self, memory_budget=64 << 30, slots=8, precision=fm.FM_MIXED, seed=None, reorth_interval=1,
                 graphs=True, group_factory=Group, size_of=workspace_bytes, autotune=False, tuner=None):
        self.budget = memory_budget
        self.slots = slots
        self.precision = precision
        self.seed = workloads.seed_of("served_mix") if seed is None else seed
        self.reorth = reorth_interval
        self.graphs = graphs
        self.factory = group_factory
        self.size_of = size_of
        self.groups = {}
        self.used = 0
        self.autotune = autotune
        self.tuner = tuner if tuner is not None else self._fm_tuner
        self.tuned = {}           # (L, protocol) -> {"tile_config", "reorth_interval", ...}

    def _fm_tuner(self, L, protocol):
        prot = fm.FM_HOMODYNE if protocol == "homodyne" else fm.FM_PROJECTIVE
        p = fm.make_params(L, batch=self.slots, protocol=prot, precision=self.precision, gamma=1.0, seed=self.seed)
        return fm.autotune(p, steps=4, max_reorth=4, ortho_tol=1e-6, use_graphs=self.graphs)

    def pretune(self, kinds):
        """Run the tile / reorth search for every (L, protocol) in `kinds` now."""
        for key in sorted(set(kinds)):
            if key not in self.tuned:
                self.tuned[key] = self.tuner(*key)
        return dict(self.tuned)

    def _settings(self, key):
        if not self.autotune:
            return 0, self.reorth
        if key not in self.tuned:
            self.tuned[key] = self.tuner(*key)
        t = self.tuned[key]
        return t["tile_config"], t["reorth_interval"]

    def _group_for(self, req, ready):
        """A group of the request's kind with a free slot that may take it now (`ready`: ids of
        the groups whose last period completed and was processed), a new group if every group
        of the kind is full and the memory budget allows, else None (the request waits)."""
        key = (req.L, req.protocol)
        gs = self.groups.get(key, [])
        for g in gs:
            if g.free and id(g) in ready:
                return g
        if any(g.free for g in gs):
            return None                  # a slot frees up when that group's period ends
        tile_config, reorth = self._settings(key)
        need = self.size_of(req.L, req.protocol, self.slots, self.precision, reorth)
        if self.used + need > self.budget:
            # free the memory of groups with nothing in flight
            for k in list(self.groups):
                for gg in [gg for gg in self.groups[k] if not gg.busy() and gg.idle()]:
                    self.used -= gg.bytes
                    self.groups[k].remove(gg)
                    gg.close()
                if not self.groups[k]:
                    del self.groups[k]
            if self.used + need > self.budget:
                return None
        g = self.factory(req.L, req.protocol, self.slots, self.precision, self.seed, reorth, self.graphs,
                         tile_config)
        self.groups.setdefault(key, []).append(g)
        self.used += g.bytes
        ready.add(id(g))
        return g

    def _all_groups(self):
        return [g for gs in self.groups.values() for g in gs]

    def run(self, requests, realtime=True):
        """Serve `requests`; returns (results, stats)."""
        pending = collections.deque(sorted(requests, key=lambda r: r.arrival))
        waiting = collections.deque()
        results = []
        lat = []                      # per request step, ms
        steps_done = 0
        t0 = time.perf_counter()
        while pending or waiting or any(g.busy() for g in self._all_groups()):
            now = time.perf_counter() - t0
            while pending and (pending[0].arrival <= now or not realtime):
                waiting.append(pending.popleft())
            progressed = False
            # groups whose last period completed: account, start the entropies of finished
            # requests; collect finished entropies
            ready = set()
            for g in self._all_groups():
                if g.idle():
                    g.account(now, lat)
                    g.start_entropies()
                    ready.add(id(g))
                if g.tickets:
                    got = g.harvest(now)
                    results.extend(got)
                    progressed |= bool(got)
            # admission: first come first served, by free slot (of a ready group) and memory budget
            still = collections.deque()
            while waiting:
                req = waiting.popleft()
                g = self._group_for(req, ready)
                if g is None:
                    still.append(req)
                else:
                    g.admit(req, now)
                    progressed = True
            waiting = still
            # launch the next period of every ready group with work
            for g in self._all_groups():
                if g.active and id(g) in ready:
                    n = g.tick_steps()
                    steps_done += n * len(g.active)
                    g.launch_steps(n, time.perf_counter() - t0)
                    progressed = True
            if not progressed:
                live = [g for g in self._all_groups() if g.busy()]
                if not live and waiting and not pending:
                    raise RuntimeError("request (L=%d, %s) does not fit the memory budget"
                                       % (waiting[0].L, waiting[0].protocol))
                if not live and pending and realtime:
                    time.sleep(max(0.0, min(0.01, pending[0].arrival - now)))
                else:
                    time.sleep(0.0002)
        wall = time.perf_counter() - t0
        lat_a = np.array(lat) if lat else np.zeros(1)
        stats = {"requests": len(results), "trajectory_steps": steps_done, "wall_s": wall,
                 "steps_per_s": steps_done / wall if wall > 0 else 0.0,
                 "step_latency_ms_p50": float(np.percentile(lat_a, 50)),
                 "step_latency_ms_p99": float(np.percentile(lat_a, 99)),
                 "latency_samples": int(lat_a.size),
                 "groups": {"%d/%s" % k: [g.slots for g in gs] for k, gs in self.groups.items()},
                 "workspace_gb": self.used / 1e9,
                 "tuned": {"%d/%s" % k: v for k, v in self.tuned.items()}}
        return results, stats


def served_mix_requests(n=256, steps=500, rate=None, seed=None):
    """The served-mix workload: Poisson arrivals of ring trajectories, L in {256 .. 4096}."""
    reqs = workloads.served_requests(n=n, rate=rate, seed=seed)
    return [Request(rid=i, L=L, protocol=p, gamma=g, traj_id=tid, steps=steps, arrival=t)
            for (t, L, p, g, tid), i in zip(reqs, range(n))]


if __name__ == "__main__":
    import argparse
    import json

    import torch
    ap = argparse.ArgumentParser(description="serve the mixed trajectory workload and report latency")
    ap.add_argument("--requests", type=int, default=256)
    ap.add_argument("--steps", type=int, default=500)
    ap.add_argument("--slots", type=int, default=16)
    ap.add_argument("--rate", type=float, default=None, help="arrivals per second (default: workload's)")
    ap.add_argument("--no-autotune", action="store_true", help="default tiles, reorth_interval 1")
    args = ap.parse_args()
    torch.cuda.set_device(0)
    srv = Server(slots=args.slots, autotune=not args.no_autotune)
    reqs = served_mix_requests(args.requests, args.steps, rate=args.rate)
    t0 = time.perf_counter()
    if srv.autotune:
        srv.pretune((r.L, r.protocol) for r in reqs)
    tune_s = time.perf_counter() - t0
    res, st = srv.run(reqs)
    st["autotune_s"] = tune_s
    print(json.dumps(st))
