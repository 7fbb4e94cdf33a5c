"""The reference arm of bench.py (the oracle on the host cores) and its workload sampling (CPU only)."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def test_oracle_sample_follows_the_workload():
    import bench
    from paper_2508_18468_gb300 import workloads
    W = workloads.WORKLOADS
    assert bench.oracle_sample(W["ring64_projective"]) == (64, 1, "projective", 0.5)
    Lx, Ly, prot, gam = bench.oracle_sample(W["ring1024_projective_batch"])
    assert (Lx, Ly, prot) == (1024, 1, "projective") and gam == pytest.approx(0.9)
    assert bench.oracle_sample(W["ring16384_homodyne"]) == (bench.ORACLE_SAMPLE_L, 1, "homodyne", 0.65)
    Lx, Ly, prot, _ = bench.oracle_sample(W["torus160_both"])
    assert Lx == Ly and Lx * Ly <= bench.ORACLE_SAMPLE_L and prot == "homodyne"
    assert bench.oracle_sample(W["served_mix"])[:3] == (4096, 1, "homodyne")
    assert bench.workload_sites(W["torus160_both"]) == 25600


def test_reference_arm_prints_one_contract_line():
    env = dict(os.environ, CUDA_VISIBLE_DEVICES="")
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--workload",
                          "ring64_projective", "--steps", "2", "--warmup", "3"], cwd=ROOT, env=env,
                         capture_output=True, text=True, timeout=300)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["value"] > 0 and d["higher_is_better"] is True
    assert d["steps"] == 2 and d["warmup"] == 3 and d["n_gpus"] == 1
    assert d["config"]["workload"] == "ring64_projective" and d["config"]["L"] == 64
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"]
    assert "projective" in cb["sample"] and "scaled" not in cb["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}


def test_reference_arm_under_torchrun_prints_once():
    """Launched as the driver launches N > 1 (one process per rank): rank 0 alone times the oracle and
    prints; the other rank exits 0 without work."""
    import socket
    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        port = sk.getsockname()[1]
    env = dict(os.environ, CUDA_VISIBLE_DEVICES="")
    out = subprocess.run([sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
                          "--master-addr", "127.0.0.1", "--master-port", str(port), os.path.join(ROOT, "bench.py"),
                          "--impl", "reference", "--workload", "ring64_projective", "--gpus", "2", "--steps", "1",
                          "--warmup", "3"], cwd=ROOT, env=env, capture_output=True, text=True, timeout=300)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0


def test_single_core_oracle_figure():
    """cpu_baseline carries the oracle held to one thread as well (a child process with every
    thread pool of size 1), on the same kind of sample, capped at 1024 sites."""
    import bench
    from paper_2508_18468_gb300 import workloads
    W = workloads.WORKLOADS
    assert bench.oracle_sample(W["ring16384_homodyne"], bench.SINGLE_CORE_SAMPLE_L)[:2] == (1024, 1)
    assert bench.oracle_sample(W["torus160_both"], bench.SINGLE_CORE_SAMPLE_L)[:2] == (32, 32)
    cb = bench.cpu_baseline_line(W["ring64_projective"], 1, nsteps=1)
    sc = cb["single_core"]
    assert sc["threads"] == 1 and sc.get("value") and sc["value"] > 0, sc
    assert "projective" in sc["sample"] and "scaled" not in sc["sample"]
