"""Profiling helpers: workloads to run under ncu, and a launch-list summary.

    python -m paper_2508_18468_gb300.profiling steps L B K [protocol] [propagation] [reorth] [tile_config]
        L-site ring (or Lx x Ly torus written "LxxLy"), B trajectories, mixed precision:
        warm-up steps up to a whole step period, then K steps inside the NVTX range "steps"
        (capture them with ncu --nvtx --nvtx-include "steps/").  protocol: homodyne (default),
        projective, poisson, rk4; propagation: dense (default) or banded; reorth: the
        reorth_interval (default 1); tile_config (default 0).  Prints one JSON line.
    python -m paper_2508_18468_gb300.profiling entropy L [full|sketch] [steps]
        `steps` steps (default 1) of a single homodyne trajectory, then the half-chain
        entropy by the given method (default full) inside the NVTX range "entropy".
    python -m paper_2508_18468_gb300.profiling summary <launches.csv>
        launches, total time and share of every kernel of an ncu launch list
        (--metrics gpu__time_duration.sum --csv), largest first.
"""
import collections
import csv
import json
import re
import sys
import time

SCALE = {"ns": 1e-6, "nsecond": 1e-6, "us": 1e-3, "usecond": 1e-3, "ms": 1.0, "msecond": 1.0, "s": 1e3,
         "second": 1e3}


def summary(path):
    rows = list(csv.reader(open(path)))
    hi = next(i for i, r in enumerate(rows) if "Kernel Name" in r)
    hdr = rows[hi]
    ki, mi, vi, ui = (hdr.index(x) for x in ("Kernel Name", "Metric Name", "Metric Value", "Metric Unit"))
    tot, cnt = collections.defaultdict(float), collections.Counter()
    for r in rows[hi + 1:]:
        if len(r) <= vi or r[mi] != "gpu__time_duration.sum":
            continue
        name = re.sub(r"\(CUtensorMap.*|\((const |int|long|float|double|cplx|__half|unsigned).*", "", r[ki]).strip()
        tot[name] += float(r[vi].replace(",", "")) * SCALE[r[ui]]
        cnt[name] += 1
    T = sum(tot.values())
    print("launches %d, total %.1f ms" % (sum(cnt.values()), T))
    print("%8s %12s %7s  %s" % ("launches", "total ms", "share", "kernel"))
    for k, v in sorted(tot.items(), key=lambda x: -x[1]):
        print("%8d %12.2f %6.1f%%  %s" % (cnt[k], v, 100 * v / T, k))


def _lattice(spec):
    if "x" in spec:
        a, b = spec.split("x")
        return int(a), int(b)
    return int(spec), 1


def steps(spec, B, K, protocol="homodyne", propagation="dense", reorth=1, tile_config=0):
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from . import fm, workloads
    Lx, Ly = _lattice(spec)
    prot = {"homodyne": fm.FM_HOMODYNE, "projective": fm.FM_PROJECTIVE, "poisson": fm.FM_PROJECTIVE_POISSON,
            "rk4": fm.FM_HOMODYNE_RK4}[protocol]
    reorth = int(reorth)
    g = fm.Trajectories(fm.make_params(Lx, Ly, batch=B, protocol=prot, precision=fm.FM_MIXED, gamma=1.0,
                                       seed=workloads.seed_of("ring16384_homodyne"), reorth_interval=reorth,
                                       tile_config=int(tile_config)))
    g.set_gammas(([0.3, 0.3, 1.0, 1.0] * B)[:B])
    if propagation == "banded":
        g.set_propagation(fm.FM_PROP_BANDED)
    g.step(3 if reorth == 1 else reorth)
    torch.cuda.synchronize()
    l0 = g.kernel_launches
    torch.cuda.nvtx.range_push("steps")
    t0 = time.perf_counter()
    g.step(K)
    torch.cuda.synchronize()
    t = time.perf_counter() - t0
    torch.cuda.nvtx.range_pop()
    print(json.dumps({"Lx": Lx, "Ly": Ly, "B": B, "steps": K, "protocol": protocol, "propagation": propagation,
                      "reorth_interval": reorth, "tile_config": int(tile_config), "s_per_step": t / K,
                      "launches_per_step": (g.kernel_launches - l0) / K}))


def entropy(L, method="full", nsteps=1):
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from . import fm
    g = fm.Trajectories(fm.make_params(L, batch=1, protocol=fm.FM_HOMODYNE, precision=fm.FM_MIXED, gamma=1.0,
                                       seed=1))
    g.step(nsteps)
    if method == "sketch":
        g.set_entropy_method(fm.FM_EE_SKETCH)
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_push("entropy")
    t0 = time.perf_counter()
    S = g.entropy(list(range(L // 2)))
    t = time.perf_counter() - t0
    torch.cuda.nvtx.range_pop()
    info = g.entropy_sketch_info() if method == "sketch" else None
    print(json.dumps({"L": L, "steps": nsteps, "method": method, "S": S, "entropy_s": t, "sketch_info": info}))


if __name__ == "__main__":
    cmd = sys.argv[1]
    if cmd == "steps":
        steps(sys.argv[2], int(sys.argv[3]), int(sys.argv[4]), *sys.argv[5:9])
    elif cmd == "entropy":
        entropy(int(sys.argv[2]), *(sys.argv[3:4]), *[int(x) for x in sys.argv[4:5]])
    elif cmd == "summary":
        summary(sys.argv[2])
    else:
        summary(cmd)
