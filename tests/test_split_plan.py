"""The plan of a trajectory split over ranks by orbitals (split.py), on CPU with gloo.

Two and three ranks each hold a column block of U; the test does the local arithmetic in
numpy FP64 (what each GPU's kernels would do on its block) and the plan does every
exchange.  After a homodyne step (propagation, occupations, weight, CholeskyQR2), a
projective step (every measured site: Born weight and v = U x^dag summed over ranks) and an
entropy of a subsystem (C_A summed over ranks), C = U U^dag and S_A equal the oracle's
unsplit step.  The multi-GPU path itself is not built: these are its exchanges only."""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

WORKER = r"""
import json, os, sys
sys.path.insert(0, os.environ["FM_ROOT"])
import numpy as np
import torch
import torch.distributed as dist
dist.init_process_group("gloo", init_method="env://")
from oracle import lattice, observables, philox, trajectory
from paper_2508_18468_gb300.split import SplitPlan, column_shards

L, N = 48, 24
out = {}
for protocol in (trajectory.HOMODYNE, trajectory.PROJECTIVE):
    prm = trajectory.Params(Lx=L, gamma=1.3, protocol=protocol, seed=17, traj_id=3)
    P = lattice.propagator(L, 1, prm.J, prm.dt)
    U = lattice.initial_orbitals(L, 1)
    for s in range(4):                               # a developed state, the same on every rank
        U, _ = trajectory.step(U, P, prm, s)
    s = 4
    ref, _ = trajectory.step(U, P, prm, s)
    plan = SplitPlan(L, N)
    Ur = P @ U[:, plan.lo:plan.hi]                   # propagation: local
    if protocol == trajectory.HOMODYNE:
        part = torch.from_numpy(np.real(np.sum(Ur * np.conj(Ur), axis=1)).copy())
        n = plan.allreduce_occupations(part).numpy()
        xi = philox.noise_normals(prm.seed, prm.traj_id, s, L)
        w = np.exp(np.sqrt(prm.gamma * prm.dt) * xi + (2.0 * n - 1.0) * prm.gamma * prm.dt)
        Ur = w[:, None] * Ur                         # weight: local
    else:
        u_sel, u_out = philox.measure_draws(prm.seed, prm.traj_id, s, L)
        p_meas = 1.0 - np.exp(-prm.gamma * prm.dt)
        for j in np.nonzero(u_sel < p_meas)[0]:
            x = Ur[j, :].copy()
            pj = plan.allreduce_sum(torch.tensor([float(np.real(np.vdot(x, x)))], dtype=torch.float64)).item()
            pj = min(max(pj, 0.0), 1.0)
            o = 1 if u_out[j] < pj else 0
            if pj < 1e-300:
                continue
            sp = np.sqrt(pj)
            v = plan.allreduce_sum(torch.from_numpy(Ur @ np.conj(x))).numpy() / sp
            ej = np.zeros(L, dtype=complex)
            ej[j] = 1.0
            vn = ej if o == 1 else (v - sp * ej) / np.sqrt(1.0 - pj)
            Ur = Ur + np.outer(vn - v, x) / sp       # rank-1 update: local
    for _ in range(2):                               # CholeskyQR2
        Uf = plan.gather_columns(torch.from_numpy(Ur)).numpy()
        G = plan.allreduce_gram(torch.from_numpy(Uf.conj().T @ Ur)).numpy()
        R = np.linalg.cholesky(G).conj().T           # replicated factor
        T = np.linalg.inv(R)
        Ur = Uf @ T[:, plan.lo:plan.hi]
    Uf = plan.gather_columns(torch.from_numpy(Ur)).numpy()
    A = list(range(0, L, 3))
    CA = plan.allreduce_sum(torch.from_numpy(Ur[A] @ Ur[A].conj().T)).numpy()
    lam = np.clip(np.linalg.eigvalsh(CA), 0.0, 1.0)
    S = float(-np.sum(observables.binary_entropy_terms(lam)))
    key = "homodyne" if protocol == trajectory.HOMODYNE else "projective"
    out[key] = {"dC": float(np.max(np.abs(observables.correlation(Uf) - observables.correlation(ref)))),
                "dS": abs(S - observables.entanglement_entropy(ref, A)),
                "ortho": float(np.max(np.abs(Uf.conj().T @ Uf - np.eye(N)))),
                "cols": [plan.lo, plan.hi]}
out["rank"] = dist.get_rank()
out["bytes"] = SplitPlan(16384, 8192, world=dist.get_world_size(), rank=0).bytes_per_step()
print(json.dumps(out))
dist.destroy_process_group()
"""


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_column_shards():
    pytest.importorskip("torch")
    from paper_2508_18468_gb300.split import column_shards
    assert column_shards(8192, 4) == [(0, 2048), (2048, 4096), (4096, 6144), (6144, 8192)]
    assert column_shards(8192, 3) == [(0, 2816), (2816, 5504), (5504, 8192)]     # 128-wide boundaries
    assert column_shards(24, 3) == [(0, 8), (8, 16), (16, 24)]
    for N, R in ((24, 2), (100, 7), (12800, 8)):
        sh = column_shards(N, R)
        assert sh[0][0] == 0 and sh[-1][1] == N and all(a[1] == b[0] for a, b in zip(sh, sh[1:]))
        assert max(h - l for l, h in sh) - min(h - l for l, h in sh) <= (128 if N % 128 == 0 else 1)
    with pytest.raises(ValueError):
        column_shards(3, 4)


@pytest.mark.parametrize("world", [2, 3])
def test_split_step_equals_the_unsplit_oracle_step(world):
    pytest.importorskip("torch")
    port = _free_port()
    procs = []
    for r in range(world):
        env = dict(os.environ, MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(r),
                   WORLD_SIZE=str(world), LOCAL_RANK=str(r), FM_ROOT=ROOT, CUDA_VISIBLE_DEVICES="")
        procs.append(subprocess.Popen([sys.executable, "-c", WORKER], env=env, stdout=subprocess.PIPE,
                                      stderr=subprocess.PIPE, text=True))
    outs = []
    for p in procs:
        out, err = p.communicate(timeout=180)
        assert p.returncode == 0, err
        outs.append(json.loads(out.strip().splitlines()[-1]))
    outs.sort(key=lambda d: d["rank"])
    for d in outs:
        for key in ("homodyne", "projective"):
            assert d[key]["dC"] <= 1e-12, (key, d[key])
            assert d[key]["dS"] <= 1e-11, (key, d[key])
            assert d[key]["ortho"] <= 1e-13, (key, d[key])
    cols = [d["homodyne"]["cols"] for d in outs]
    assert cols[0][0] == 0 and cols[-1][1] == 24 and all(a[1] == b[0] for a, b in zip(cols, cols[1:]))
    assert outs[0]["bytes"] > 0
