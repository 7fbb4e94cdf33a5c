"""Continuous-batching server for monitored-trajectory jobs on one GPU.

A request asks for one trajectory: lattice size L (ring), protocol, monitoring
rate gamma, trajectory id and a number of steps; the answer is the half-chain
entanglement entropy at the end.  Requests of equal (L, protocol) share one
``fm_state`` whose batch slots are reused as requests finish
(``fm_reset_trajectory``); each group steps on its own CUDA stream, replaying
a CUDA graph of its step, so groups of different sizes run side by side on the
device.  A new group is created only if its workspace fits the memory budget
(admission by HBM footprint); otherwise the request waits for a free slot.

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
        self.half = workloads.half_chain(L)

    def stream_context(self):
        import torch
        return torch.cuda.stream(self.stream)

    def synchronize(self):
        self.stream.synchronize()

    def close(self):
        self.traj.close()

    def admit(self, req, now):
        b = self.free.pop()
        self.traj.reset_trajectory(b, req.traj_id, req.gamma)
        self.active[b] = _Slot(req=req, done=0, admitted=now)

    def tick_steps(self):
        """Steps for the next tick: one graph period, clipped to the nearest finishing request."""
        rem = min(sl.req.steps - sl.done for sl in self.active.values())
        return max(1, min(self.period, rem))

    def launch_steps(self, n):
        self.traj.step(n)
        for sl in self.active.values():
            sl.done += n

    def harvest(self, now):
        out = []
        for b in [b for b, sl in self.active.items() if sl.done >= sl.req.steps]:
            sl = self.active.pop(b)
            S = self.traj.entropy(self.half, b)
            out.append(Result(rid=sl.req.rid, S=S, steps=sl.done, admitted=sl.admitted, finished=now,
                              group=(self.L, self.protocol)))
            self.free.append(b)
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

    def _group_for(self, req):
        key = (req.L, req.protocol)
        g = self.groups.get(key)
        if g is not None:
            return g if g.free else None
        tile_config, reorth = self._settings(key)
        need = self.size_of(req.L, req.protocol, self.slots, self.precision, reorth)
        if self.used + need > self.budget:
            # free the memory of groups with nothing in flight
            for k in [k for k, gg in self.groups.items() if not gg.active]:
                self.used -= self.groups[k].bytes
                self.groups.pop(k).close()
            if self.used + need > self.budget:
                return None
        g = self.factory(req.L, req.protocol, self.slots, self.precision, self.seed, reorth, self.graphs,
                         tile_config)
        self.groups[key] = g
        self.used += g.bytes
        return g

    def run(self, requests, realtime=True):
        """Serve `requests`; returns (results, stats)."""
        pending = collections.deque(sorted(requests, key=lambda r: r.arrival))
        waiting = collections.deque()
        results = []
        tick_ms = []
        steps_done = 0
        t0 = time.perf_counter()
        while pending or waiting or any(g.active for g in self.groups.values()):
            now = time.perf_counter() - t0
            while pending and (pending[0].arrival <= now or not realtime):
                waiting.append(pending.popleft())
            # admission: first come first served, by free slot and memory budget
            still = collections.deque()
            while waiting:
                req = waiting.popleft()
                g = self._group_for(req)
                if g is None:
                    still.append(req)
                else:
                    g.admit(req, now)
            waiting = still
            busy = [g for g in self.groups.values() if g.active]
            if not busy:
                if waiting and not pending:
                    raise RuntimeError("request (L=%d, %s) does not fit the memory budget"
                                       % (waiting[0].L, waiting[0].protocol))
                if pending:
                    time.sleep(max(0.0, min(0.01, pending[0].arrival - now)))
                continue
            t1 = time.perf_counter()
            nsteps = {}
            for g in busy:                       # each group on its own stream: work overlaps on the GPU
                nsteps[id(g)] = g.tick_steps()
                with g.stream_context():
                    g.launch_steps(nsteps[id(g)])
            for g in busy:
                g.synchronize()
            dt = (time.perf_counter() - t1) * 1e3
            tick_ms.append(dt / max(nsteps.values()))          # per-step latency of this tick
            steps_done += sum(len(g.active) * nsteps[id(g)] for g in busy)
            now = time.perf_counter() - t0
            for g in busy:
                results.extend(g.harvest(now))
        wall = time.perf_counter() - t0
        lat = np.array(tick_ms) if tick_ms else np.zeros(1)
        stats = {"requests": len(results), "trajectory_steps": steps_done, "wall_s": wall,
                 "steps_per_s": steps_done / wall if wall > 0 else 0.0,
                 "step_latency_ms_p50": float(np.percentile(lat, 50)),
                 "step_latency_ms_p99": float(np.percentile(lat, 99)),
                 "groups": {"%d/%s" % k: g.slots for k, g in self.groups.items()},
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
