#!/usr/bin/env python
"""Throughput of the monitored free-fermion trajectory step on GB300.

One step = the whole hot path for every trajectory of the batch: dense
propagation U <- exp(-i H dt) U, the homodyne weight, CholeskyQR2
re-orthonormalisation, and -- on the workload's schedule -- the half-chain
entanglement entropy (FP64 eigenvalues).  Default workload: 1d ring
L = 16384 (N = 8192), homodyne protocol, 4 trajectories (gamma 0.3, 0.3,
1.0, 1.0), dt = 0.05, half-chain EE every 100 steps, mixed precision
(split-fp16 tensor-core GEMMs, FP64 Cholesky / eigenvalues).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Multi-GPU: trajectories are independent, so N ranks run N independent
batches (replicas, weak scaling); the only collective is the timing barrier.
--impl reference times the FP64 CPU oracle on this host's cores (bounded
sample, scaled by the step's L^3 flop count).
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "trajectory steps/s at L=16384 (mixed precision, EE err <= 1e-3)"
UNIT = "trajectory-steps/s"
WORKLOAD = "ring16384_homodyne"
ORACLE_SAMPLE_L = 4096
# The paper's own rate for the same workload, from its wall time (App. A): about 130 h
# for one homodyne trajectory at L = 16384 over t in [0, L] with dt = 0.05 (327,680
# steps) on one A100 -> 0.70 trajectory-steps/s.  Other hardware: context only.
PAPER_RATE = {"ring16384_homodyne": 327680 / (130 * 3600.0)}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default=WORKLOAD)
    ap.add_argument("--precision", choices=["mixed", "fp64"], default="mixed")
    ap.add_argument("--propagation", choices=["dense", "banded"], default="dense",
                    help="dense L x L GEMM (the method as defined) or stencils of the circulant propagator")
    ap.add_argument("--ee-method", choices=["auto", "sketch", "full"], default="auto",
                    help="entropy method of the in-window entropies (mixed precision): auto (the "
                         "cross-block sketch for subsystems of 1024 sites or more, else the full "
                         "method), the sketch, or the full eigen-decomposition of C_A")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-others", action="store_true",
                    help="skip the short measurements of the other workloads (ring64, ring1024 x 256, torus "
                         "160 x 160, served mix) added to the line")
    ap.add_argument("--fp64-steps", type=int, default=2,
                    help="steps of the all-FP64 GPU path (one trajectory, beside the mixed path on the same "
                         "trajectory) for the speedup and the accuracy of the mixed path; 0 skips it")
    return ap.parse_args()


# ---------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index):
        self.idx = device_index
        self.rows = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.idx), "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) == 7:
                self.rows.append(parts)

    def stop(self):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
        rows = self.rows
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(r[0]) for r in rows if r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[3 + i].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


# ---------------------------------------------------------------- oracle timing (CPU)
def oracle_sample(wl, cap=None):
    """The oracle's bounded sample of a workload: (Lx, Ly, protocol, gamma) of the lattice it times.
    The workload's own lattice when L <= cap (default ORACLE_SAMPLE_L), else a ring of cap sites or a
    square torus of that many; the workload's protocol (homodyne for the torus workload that runs
    both, and for the served mix) at its mean rate."""
    cap = ORACLE_SAMPLE_L if cap is None else cap
    if "Lx" not in wl:                                   # the served mix: its largest ring
        Lx, Ly, prot, gam = max(wl["sizes"]), 1, "homodyne", sum(wl["gamma_range"]) / 2
    else:
        Lx, Ly = wl["Lx"], wl["Ly"]
        prot = "projective" if wl["protocol"] == "projective" else "homodyne"
        gam = sum(wl["gammas"]) / len(wl["gammas"])
    if Lx * Ly > cap:
        if Ly == 1:
            Lx = cap
        else:
            Lx = Ly = int(round(cap ** 0.5))
    return Lx, Ly, prot, gam


def oracle_step_seconds(sample, nsteps, seed):
    """Wall time per oracle step of one trajectory on the sample lattice (FP64, numpy on all host cores)."""
    import numpy as np  # noqa: F401
    from oracle import lattice, trajectory
    Lx, Ly, prot, gam = sample
    prm = trajectory.Params(Lx=Lx, Ly=Ly, gamma=gam, seed=seed,
                            protocol=trajectory.PROJECTIVE if prot == "projective" else trajectory.HOMODYNE)
    P = lattice.propagator(Lx, Ly, prm.J, prm.dt)
    U = lattice.initial_orbitals(Lx, Ly)
    U, _ = trajectory.step(U, P, prm, 0)       # one untimed step (first touch)
    t0 = time.perf_counter()
    for s in range(1, 1 + nsteps):
        U, _ = trajectory.step(U, P, prm, s)
    return (time.perf_counter() - t0) / nsteps


def cpu_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count()


def workload_sites(wl):
    return wl["Lx"] * wl["Ly"] if "Lx" in wl else max(wl["sizes"])


def describe_sample(sample, nsteps, L_target, per):
    Lx, Ly, prot, gam = sample
    lat = "L=%d" % Lx if Ly == 1 else "%dx%d torus" % (Lx, Ly)
    text = "%d %s oracle steps (gamma %.2f) at %s (numpy FP64, %.3g s/step)" % (nsteps, prot, gam, lat, per)
    if Lx * Ly != L_target:
        text += ", scaled by (%d/%d)^3" % (L_target, Lx * Ly)
    return text


SINGLE_CORE_SAMPLE_L = 1024


def oracle_single_core(wl, seed, nsteps=2):
    """The oracle held to one thread (BLAS and OpenMP pools of size 1, in a child process so the
    setting takes effect before numpy loads), on at most SINGLE_CORE_SAMPLE_L sites, scaled by the
    cube of the site ratio like the multi-core figure.  Returns a dict; on any failure its value is
    None and it says why."""
    sample = oracle_sample(wl, SINGLE_CORE_SAMPLE_L)
    L_target = workload_sites(wl)
    code = ("import json, sys; sys.path.insert(0, %r); import bench; "
            "print(json.dumps(bench.oracle_step_seconds(%r, %d, %d)))" % (ROOT, tuple(sample), nsteps, seed))
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1",
               CUDA_VISIBLE_DEVICES="")
    try:
        out = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=120)
        if out.returncode != 0:
            raise RuntimeError(out.stderr.strip().splitlines()[-1] if out.stderr.strip() else "exit %d" % out.returncode)
        per = float(out.stdout.strip().splitlines()[-1])
    except Exception as e:  # the bench line is printed either way
        return {"value": None, "threads": 1, "error": str(e)[:200]}
    scale = (L_target / (sample[0] * sample[1])) ** 3
    return {"value": 1.0 / (per * scale), "unit": UNIT, "threads": 1,
            "sample": describe_sample(sample, nsteps, L_target, per)}


def cpu_baseline_line(wl, seed, nsteps=3):
    """The oracle timed on a bounded sample of the workload (one trajectory-step costs ~L^3 for the
    dense propagation and CholeskyQR, so a smaller lattice is scaled by the cube of the site ratio)."""
    sample = oracle_sample(wl)
    L_target = workload_sites(wl)
    t = oracle_step_seconds(sample, nsteps, seed)
    scale = (L_target / (sample[0] * sample[1])) ** 3
    return {"value": 1.0 / (t * scale), "unit": UNIT, "cores": cpu_cores(), "kind": "oracle",
            "sample": describe_sample(sample, nsteps, L_target, t),
            "single_core": oracle_single_core(wl, seed)}


# ---------------------------------------------------------------- helpers
def load_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return d, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


def profiled_traffic(L, B):
    """DRAM bytes (read + write) of one propagation launch at ring L with B trajectories, from the
    ncu capture at ring L = 4096, B = 4 (profiles/prop_gemm_ring4096.md, line
    'dram_bytes_per_launch_propagation: X'), scaled by (L / 4096)^3 (B / 4): the operand re-reads
    grow with the number of tile waves (~L^2 B) times the operand bytes of a wave (~L).  Returns
    (bytes, source) or (None, why)."""
    path = os.path.join(ROOT, "profiles", "prop_gemm_ring4096.md")
    if not os.path.exists(path):
        return None, "no capture"
    for line in open(path):
        if line.strip().startswith("dram_bytes_per_launch_propagation:"):
            try:
                x = float(line.split(":", 1)[1].split()[0])
            except ValueError:
                return None, "unreadable capture line"
            scale = (L / 4096.0) ** 3 * (B / 4.0)
            return x * scale, ("ncu dram__bytes_read.sum + dram__bytes_write.sum of tc_gemm_kernel<128,0,1> "
                               "(the benchmark's tile configuration) at ring L=4096, B=4 "
                               "(profiles/prop_gemm_ring4096.md) x (L/4096)^3 (B/4) = x %.0f" % scale)
    return None, "no propagation line in the capture summary"


def setup_distributed(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x, world):
    """The largest x over the ranks (the timing reduction; NCCL on GPUs, gloo on CPU)."""
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_traj_id(rank, batch):
    """Replicas: rank r advances trajectories r * batch .. (r + 1) * batch - 1 of the workload."""
    return rank * batch


def fp64_side_by_side(fm, wl, seed, traj, gamma, nsteps, ee_sites, ee_method):
    """The all-FP64 GPU path (complex128 state, FP64 GEMMs and Cholesky, the workload's reorth
    interval) on one trajectory of the workload, timed with CUDA events over nsteps steps from the
    Neel start, and the mixed path on the same trajectory (same Philox draws) for the same steps;
    then the half-chain entropy of both (FP64: the full eigen-decomposition; mixed: the bench's
    entropy method), max|C_mixed - C_fp64| on the first 512 rows and the orthonormality of both."""
    import numpy as np
    import torch
    Lx, Ly = wl["Lx"], wl["Ly"]
    protocol = fm.FM_HOMODYNE if wl["protocol"] == "homodyne" else fm.FM_PROJECTIVE
    kw = dict(batch=1, protocol=protocol, reorth_interval=wl["reorth_interval"], gamma=gamma, seed=seed,
              traj_id=traj)
    stream = torch.cuda.current_stream()
    gd = fm.Trajectories(fm.make_params(Lx, Ly, precision=fm.FM_FP64, **kw))
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    gd.step(nsteps)
    e1.record(stream)
    torch.cuda.synchronize()
    t = e0.elapsed_time(e1) / 1e3
    gm = fm.Trajectories(fm.make_params(Lx, Ly, precision=fm.FM_MIXED, tile_config=wl.get("tile_config", 0), **kw))
    if ee_method != "full":
        gm.set_entropy_method(fm.FM_EE_SKETCH if ee_method == "sketch" else fm.FM_EE_AUTO)
    gm.step(nsteps)
    Sd, Sm = gd.entropy(ee_sites), gm.entropy(ee_sites)
    rows = 512
    Ud, Um = gd.copy_U()[:rows], gm.copy_U()[:rows]
    dc = float(np.max(np.abs(Um @ Um.conj().T - Ud @ Ud.conj().T)))
    cols = list(range(0, gd.N, max(1, gd.N // 64)))[:64]
    od, om = gd.orthonormality_error(cols), gm.orthonormality_error(cols)
    gd.close()
    gm.close()
    del gd, gm
    torch.cuda.empty_cache()
    return {"fp64_gpu": {"value": nsteps / t, "unit": UNIT, "steps": nsteps, "trajectories": 1,
                         "ms_per_step": t * 1e3 / nsteps, "gamma": gamma, "traj_id": traj,
                         "what": "complex128 state, FP64 dense propagation GEMM, FP64 CholeskyQR2 "
                                 "(reorth interval %d), CUDA events" % wl["reorth_interval"]},
            "accuracy": {"steps": nsteps, "S_fp64": Sd, "S_mixed": Sm,
                         "ee_rel_err": abs(Sm - Sd) / max(abs(Sd), 1.0),
                         "max_abs_dC_512_rows": dc, "ortho_fp64": od, "ortho_mixed": om,
                         "ee_method_mixed": ee_method}}


def timed_steps(fm, g, nsteps, stream):
    """Device time (s) of nsteps steps of g with CUDA events, and its phase split."""
    import torch
    g.step(1)                                       # warm-up (and first-use set-up)
    torch.cuda.synchronize()
    g.phase_times()
    g.set_timing(True)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    g.step(nsteps)
    e1.record(stream)
    torch.cuda.synchronize()
    ph = g.phase_times()
    g.set_timing(False)
    return e0.elapsed_time(e1) / 1e3, ph


def prop_roofline(ph, L, N, B, peaks):
    ms, n = ph["propagate"]
    if n == 0:
        return None
    peak = peaks.get("bf16_tflops_sustained", peaks["bf16_tflops"]) / 3.0
    ach = 8.0 * L * L * N * B / (ms / n / 1e3) / 1e12
    return {"bound": "tensor", "achieved": ach, "peak": peak, "unit": "TFLOP/s", "frac": ach / peak,
            "kernel": "tc_gemm_kernel (propagation)", "ms_per_launch": ms / n}


def other_workloads(fm, peaks):
    """Short measurements of the other workloads, one GPU, CUDA events on the stepping stream:
    ring L = 64 projective (FP64, 200 steps, half-chain entropy every 10 steps); ring L = 1024
    projective, 256 trajectories (mixed, 20 steps); the 160 x 160 torus, 8 trajectories of each
    protocol (mixed, 2 steps); a bounded served mix (64 Poisson requests of 100 steps, L in
    {256 .. 4096}, arrivals at the workload's rate)."""
    import torch
    from paper_2508_18468_gb300 import serve, workloads
    stream = torch.cuda.current_stream()
    out = {}
    # c1: ring 64, FP64, 200 steps with 20 half-chain entropies
    wl = workloads.WORKLOADS["ring64_projective"]
    g = fm.Trajectories(fm.make_params(64, protocol=fm.FM_PROJECTIVE, precision=fm.FM_FP64, gamma=0.5,
                                       seed=workloads.seed_of("ring64_projective")))
    g.step(1)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(20):
        g.step(10)
        g.entropy(workloads.half_chain(64))
    torch.cuda.synchronize()
    t = time.perf_counter() - t0
    out["ring64_projective"] = {"value": 200 / t, "unit": UNIT, "steps": 200, "trajectories": 1,
                                "precision": "fp64", "what": "200 steps and 20 half-chain entropies, wall "
                                "time (launch-latency bound)"}
    g.close()
    # c2: ring 1024 x 256 projective, mixed
    wl = workloads.WORKLOADS["ring1024_projective_batch"]
    gam = wl["gammas"]
    g = fm.Trajectories(fm.make_params(1024, batch=len(gam), protocol=fm.FM_PROJECTIVE, precision=fm.FM_MIXED,
                                       seed=workloads.seed_of("ring1024_projective_batch")))
    g.set_gammas(gam)
    t, ph = timed_steps(fm, g, 20, stream)
    out["ring1024_projective_batch"] = {"value": len(gam) * 20 / t, "unit": UNIT, "steps": 20,
                                        "trajectories": len(gam), "precision": "mixed",
                                        "ms_per_step": t * 1e3 / 20,
                                        "phases_ms": {k: round(v[0], 3) for k, v in ph.items()},
                                        "roofline": prop_roofline(ph, 1024, 512, len(gam), peaks)}
    g.close()
    del g
    torch.cuda.empty_cache()
    # c4: torus 160 x 160, 8 trajectories per protocol
    wl = workloads.WORKLOADS["torus160_both"]
    gam = wl["gammas"]
    for name, prot in (("homodyne", fm.FM_HOMODYNE), ("projective", fm.FM_PROJECTIVE)):
        g = fm.Trajectories(fm.make_params(160, 160, batch=len(gam), protocol=prot, precision=fm.FM_MIXED,
                                           seed=workloads.seed_of("torus160_both")))
        g.set_gammas(gam)
        t, ph = timed_steps(fm, g, 2, stream)
        out["torus160_" + name] = {"value": len(gam) * 2 / t, "unit": UNIT, "steps": 2,
                                   "trajectories": len(gam), "precision": "mixed", "ms_per_step": t * 1e3 / 2,
                                   "phases_ms": {k: round(v[0], 3) for k, v in ph.items()},
                                   "roofline": prop_roofline(ph, 25600, 12800, len(gam), peaks)}
        g.close()
        del g
        torch.cuda.empty_cache()
    # c5 as one batch: the served mix's lattice sizes, 8 homodyne trajectories each, advanced by one
    # CUDA graph per period (fm_group: the batches' kernels overlap) against stepping the batches in turn
    sizes = workloads.WORKLOADS["served_mix"]["sizes"]
    states = [fm.Trajectories(fm.make_params(Lm, batch=8, protocol=fm.FM_HOMODYNE, precision=fm.FM_MIXED,
                                             gamma=1.0, seed=workloads.seed_of("served_mix"), traj_id=8 * i))
              for i, Lm in enumerate(sizes)]
    grp = fm.Group(states)
    nst = 10 * grp.period
    grp.step(grp.period)                           # capture and warm-up
    times = {}
    for mode in ("one_graph", "batches_in_turn"):
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        if mode == "one_graph":
            grp.step(nst)
        else:
            for g in states:
                g.step(nst)
        e1.record(stream)
        torch.cuda.synchronize()
        times[mode] = e0.elapsed_time(e1) / 1e3
    ntraj = 8 * len(sizes)
    out["batched_mix_one_graph"] = {"value": ntraj * nst / times["one_graph"], "unit": UNIT, "steps": nst,
                                    "trajectories": ntraj, "lattices": sizes,
                                    "batches_in_turn_value": ntraj * nst / times["batches_in_turn"],
                                    "what": "8 homodyne trajectories of each L, one fm_group graph launch per "
                                            "period vs each batch's own eager steps, CUDA events"}
    grp.close()
    for g in states:
        g.close()
    del states
    torch.cuda.empty_cache()
    # c5: a bounded served mix in real time
    reqs = serve.served_mix_requests(64, 100)
    srv = serve.Server(slots=8)
    res, st = srv.run(reqs, realtime=True)
    for gs in srv.groups.values():
        for gg in gs:
            gg.close()
    torch.cuda.empty_cache()
    out["served_mix"] = {"value": st["steps_per_s"], "unit": UNIT, "requests": st["requests"],
                         "steps_per_request": 100, "arrivals": "Poisson, 50/s",
                         "step_latency_ms_p50": st["step_latency_ms_p50"],
                         "step_latency_ms_p99": st["step_latency_ms_p99"], "wall_s": st["wall_s"],
                         "groups": st["groups"], "what": "64 of the workload's 256 requests, 100 of its 500 "
                         "steps each; latency per request step"}
    return out


# ---------------------------------------------------------------- reference arm
def run_reference(args, world, rank):
    from paper_2508_18468_gb300 import workloads
    if rank != 0:
        return
    wl = workloads.WORKLOADS[args.workload]
    L = workload_sites(wl)
    seed = workloads.seed_of(args.workload)
    sample = oracle_sample(wl)
    for s in range(args.warmup):
        oracle_step_seconds(sample, 1, seed + s)
    per = oracle_step_seconds(sample, args.steps, seed)
    scale = (L / (sample[0] * sample[1])) ** 3
    value = 1.0 / (per * scale)
    metric = METRIC if args.workload == WORKLOAD else "trajectory steps/s (%s)" % args.workload
    config = {"workload": args.workload, "L": L, "N": L // 2}
    if "protocol" in wl:
        config["protocol"] = wl["protocol"]
    line = {"metric": metric, "value": value, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": per * scale * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference", "config": config,
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cpu_cores(), "kind": "oracle",
                             "sample": describe_sample(sample, args.steps, L, per)},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------- our arm
def run_ours(args, world, rank, local):
    import numpy as np
    import torch
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", init_method="env://")
    else:
        torch.cuda.set_device(0)
    import __graft_entry__
    __graft_entry__.build()
    from paper_2508_18468_gb300 import fm, workloads

    wl = workloads.WORKLOADS[args.workload]
    Lx, Ly = wl["Lx"], wl["Ly"]
    L = Lx * Ly
    N = L // 2
    gam = list(wl["gammas"])
    B = len(gam)
    seed = workloads.seed_of(args.workload)
    precision = fm.FM_MIXED if args.precision == "mixed" else fm.FM_FP64
    protocol = fm.FM_HOMODYNE if wl["protocol"] == "homodyne" else fm.FM_PROJECTIVE
    prm = fm.make_params(Lx, Ly, batch=B, protocol=protocol, precision=precision,
                         reorth_interval=wl["reorth_interval"], gamma=gam[0], seed=seed,
                         traj_id=replica_traj_id(rank, B),
                         tile_config=wl.get("tile_config", 0) if precision == fm.FM_MIXED else 0)
    g = fm.Trajectories(prm)
    g.set_gammas(gam)
    if args.propagation == "banded":
        g.set_propagation(fm.FM_PROP_BANDED)
    ee_method = args.ee_method if precision == fm.FM_MIXED else "full"
    if ee_method != "full":
        g.set_entropy_method(fm.FM_EE_SKETCH if ee_method == "sketch" else fm.FM_EE_AUTO)
    ee_sites = workloads.half_chain(L)
    ee_every = wl["ee_every"]

    def window(nsteps, per_step=None):
        """nsteps steps; every ee_every steps (from the window start) the half-chain
        entropy of every trajectory is started asynchronously and overlaps the
        following steps; the window ends when all of them are back (at most 48
        are left outstanding: the library keeps 64 results)."""
        pending, results = [], []
        for i in range(nsteps):
            if i % ee_every == 0:
                for b in range(B):
                    if len(pending) >= 48:
                        results.append(g.entropy_wait(pending.pop(0)))
                    pending.append(g.entropy_async(ee_sites, b))
            if per_step:
                per_step()
            g.step(1)
        return results + [g.entropy_wait(t) for t in pending]

    for _ in range(args.warmup):
        g.step(1)
    g.entropy_wait(g.entropy_async([0, 1], 0))          # warm the eigen-solver path
    torch.cuda.synchronize()
    g.phase_times()
    g.set_timing(True)
    stream = torch.cuda.current_stream()
    sampler = ClockSampler(torch.cuda.current_device()) if rank == 0 else None
    launches0 = g.kernel_launches
    barrier(world)
    torch.cuda.synchronize()
    if sampler:
        sampler.start()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    w0 = time.perf_counter()
    e0.record(stream)
    entropies = window(args.steps)
    e1.record(stream)
    torch.cuda.synchronize()
    wall = time.perf_counter() - w0
    barrier(world)
    clocks = sampler.stop() if sampler else None
    launches = g.kernel_launches - launches0
    phases = g.phase_times()
    g.set_timing(False)
    t_dev = max(e0.elapsed_time(e1) / 1e3, wall)          # the window ends when the last entropy is back
    t = max_over_ranks(t_dev, world)
    value = world * B * args.steps / t

    # end to end through the public API: per step, upload the rates (pinned host),
    # advance, read every trajectory's occupations back to the host
    e2e = None
    if not args.no_e2e:
        gam_host = torch.tensor(gam, dtype=torch.float64).pin_memory().numpy()
        occ_host = [torch.empty(L, dtype=torch.float64).pin_memory().numpy() for _ in range(B)]

        def io():
            g.set_gammas(gam_host)
            for b in range(B):
                g.occupations(b, out=occ_host[b])
        barrier(world)
        torch.cuda.synchronize()
        w1 = time.perf_counter()
        window(args.steps, per_step=io)
        torch.cuda.synchronize()
        t_e2e = max_over_ranks(time.perf_counter() - w1, world)
        e2e = {"value": world * B * args.steps / t_e2e, "unit": UNIT, "h2d_bytes_per_step": 8 * B,
               "d2h_bytes_per_step": 8 * B * L + 8 * B // ee_every}

    guard = g.reorth_stats() if precision == fm.FM_MIXED else None
    # the batch's workspace is no longer needed: free it before the side measurements
    g.close()
    del g
    torch.cuda.empty_cache()
    side = None
    if args.fp64_steps > 0 and precision == fm.FM_MIXED and world == 1:
        hard = max(range(B), key=lambda b: gam[b])        # the trajectory with the largest rate
        side = fp64_side_by_side(fm, wl, seed, replica_traj_id(rank, B) + hard, gam[hard], args.fp64_steps,
                                 ee_sites, ee_method)

    peaks, peak_src = load_peaks()
    others = None
    if not args.no_others and world == 1 and args.workload == WORKLOAD:
        others = other_workloads(fm, peaks)

    if rank != 0:
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()
        return

    prop_ms, prop_n = phases["propagate"]
    prop_flops = 8.0 * L * L * N * B                        # algorithmic complex GEMM flops per launch
    if precision == fm.FM_MIXED:
        peak = peaks.get("bf16_tflops_sustained", peaks["bf16_tflops"]) / 3.0
        peak_note = ("%s sustained dense bf16/fp16 tensor rate / 3 (three fp16 products per "
                     "split-precision product)" % peak_src)
        dtype = "f32 state, split-fp16 tensor products, f64 Cholesky/eigenvalues"
    else:
        peak = 1.05
        peak_note = "cuBLAS DGEMM measured on this pool (FP64)"
        dtype = "f64"
    roof = None
    if prop_n > 0 and args.propagation == "banded":
        # stencil passes: each reads and writes the state once (algorithmic bytes)
        passes = 2 if Ly > 1 else 1
        elem = 8 if precision == fm.FM_MIXED else 16
        nbytes = passes * 2.0 * B * L * N * elem
        achieved = nbytes / (prop_ms / prop_n / 1e3) / 1e9
        roof = {"bound": "hbm", "achieved": achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                "frac": achieved / peaks["hbm_gbs"], "traffic": None, "kernel": "band_x4_kernel (stencil propagation)",
                "ms_per_launch": prop_ms / prop_n, "peak_note": "%s copy bandwidth" % peak_src}
    elif prop_n > 0:
        achieved = prop_flops / (prop_ms / prop_n / 1e3) / 1e12
        traffic, tsrc = profiled_traffic(L, B) if (precision == fm.FM_MIXED and Ly == 1) else (None, "not captured")
        roof = {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                "traffic": traffic, "traffic_source": tsrc,
                "kernel": "tc_gemm_kernel (propagation, split-fp16 tcgen05)",
                "ms_per_launch": prop_ms / prop_n, "peak_note": peak_note}
    line = {
        "metric": METRIC if args.workload == WORKLOAD else "trajectory steps/s (%s)" % args.workload,
        "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t * 1e3 / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": (value / PAPER_RATE[args.workload]) if args.workload in PAPER_RATE else None,
        "dtype": dtype, "data": "synthetic",
        "config": {"workload": args.workload, "L": L, "N": N, "batch_per_gpu": B, "gammas": gam,
                   "protocol": wl["protocol"], "dt": 0.05, "ee_every": ee_every,
                   "ee_sites": "half chain (%d sites), FP64, started every %d steps and overlapped" % (L // 2, ee_every),
                   "ee_method": ee_method,
                   "precision": args.precision, "propagation": args.propagation,
                   "reorth_interval": wl["reorth_interval"], "tile_config": wl.get("tile_config", 0),
                   "l2": "inputs larger than L2 (state %.1f GB, propagator %.1f GB per GPU)" % (
                       B * 2 * L * N * 4 / 1e9, 4 * L * L * 4 / 1e9),
                   "parallelism": "replicas x%d" % world},
        "roofline": roof,
        "phases_ms": {k: round(v[0], 3) for k, v in phases.items()},
        "entropies": [round(x, 6) for x in entropies],
        "gpu_launches": int(launches),
        "wall_s": wall,
        "clocks": clocks,
        "e2e": e2e,
    }
    if guard is not None:
        line["reorth_guard"] = {"second_passes": guard[0], "extra_passes": guard[1],
                                "max_diag_E": guard[2][0], "max_offdiag_E": guard[2][1],
                                "note": "E = U^dag U - 1 measured by each second CholeskyQR pass"}
    if others is not None:
        line["other_workloads"] = others
    if side is not None:
        line["fp64_gpu"] = side["fp64_gpu"]
        line["speedup_vs_fp64"] = value / side["fp64_gpu"]["value"]
        line["ee_rel_err_vs_fp64"] = side["accuracy"]["ee_rel_err"]
        line["accuracy_vs_fp64"] = side["accuracy"]
    if not args.no_cpu_baseline and world == 1:
        line["cpu_baseline"] = cpu_baseline_line(wl, seed)
    print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def main():
    args = parse()
    world, rank, local = setup_distributed(args)
    if args.impl == "reference":
        run_reference(args, world, rank)
    else:
        run_ours(args, world, rank, local)


if __name__ == "__main__":
    main()
