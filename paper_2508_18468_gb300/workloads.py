"""Seeded synthetic workloads shaped like the paper's runs (parameters only).

Nothing here computes any part of the method; these are the inputs that both
the CUDA library and the oracle receive.  The paper's lattices are 1d rings
up to L = 16384 (Sec. III, App. B) and 2d tori up to 160 x 160 (Sec. IV) at
half filling from the Neel / checkerboard state, dt = 0.05 (App. A); the
monitoring rates span the ranges the paper scans.  The seed of workload k is
0x2508184680 + k; trajectory ids run 0, 1, ... within a workload.
"""

SEED_BASE = 0x2508184680


def _gammas(values, per):
    out = []
    for g in values:
        out += [g] * per
    return out


WORKLOADS = {
    # 1d ring L = 64, projective, gamma = 0.5, 200 steps, QR every step, half-chain EE every 10 steps
    "ring64_projective": dict(index=0, Lx=64, Ly=1, protocol="projective", gammas=[0.5], steps=200,
                              ee_every=10, ee_sizes=[32], reorth_interval=1, precision="fp64"),
    # 1d ring L = 1024, projective, gamma in {0.1, 0.5, 1, 2} x 64 trajectories, 2000 steps,
    # EE of l = L/8, L/4, L/2
    "ring1024_projective_batch": dict(index=1, Lx=1024, Ly=1, protocol="projective",
                                      gammas=_gammas([0.1, 0.5, 1.0, 2.0], 64), steps=2000, ee_every=100,
                                      ee_sizes=[128, 256, 512], reorth_interval=1, precision="mixed"),
    # 1d ring L = 16384, homodyne, gamma in {0.3, 1.0} x 2 trajectories, 1000 steps,
    # half-chain EE every 100 steps.  reorth_interval and tile_config: what fm_autotune picks for
    # this batch (max_reorth 8, orthonormality bar 1e-6): the second CholeskyQR pass every 8
    # steps; tile_config 77 = 128-wide tiles in raster groups of 16 row tiles, the first-pass
    # product drained every 8 K-blocks between second passes
    "ring16384_homodyne": dict(index=2, Lx=16384, Ly=1, protocol="homodyne", gammas=[0.3, 0.3, 1.0, 1.0],
                               steps=1000, ee_every=100, ee_sizes=[8192], reorth_interval=8, tile_config=77,
                               precision="mixed"),
    # profiling size of the same step (a few GB on the device): 1d ring L = 4096, homodyne, 4 trajectories
    "ring4096_homodyne": dict(index=5, Lx=4096, Ly=1, protocol="homodyne", gammas=[0.3, 0.3, 1.0, 1.0],
                              steps=1000, ee_every=100, ee_sizes=[2048], reorth_interval=1, precision="mixed"),
    # 2d torus 160 x 160, both protocols, gamma in {0.5, 1, 1.5, 2} x 2 trajectories, 500 steps,
    # MI of two 40 x 40 blocks 40 apart and EE of the half-torus strip
    "torus160_both": dict(index=3, Lx=160, Ly=160, protocol="both", gammas=_gammas([0.5, 1.0, 1.5, 2.0], 2),
                          steps=500, ee_every=100, reorth_interval=1, precision="mixed"),
    # served mix: 256 1d trajectories, L uniform in {256, ..., 4096}, random protocol,
    # gamma ~ U[0.1, 2.0], 500 steps each, Poisson arrivals
    "served_mix": dict(index=4, sizes=[256, 512, 1024, 2048, 4096], n_requests=256, gamma_range=(0.1, 2.0),
                       steps=500, precision="mixed"),
}


def seed_of(name):
    return SEED_BASE + WORKLOADS[name]["index"]


def half_chain(L):
    return list(range(L // 2))


def torus_blocks(Lx=160, Ly=160, side=40, gap=40):
    """Two side x side blocks separated by `gap` sites along x, and the half-torus strip."""
    A = [x + Lx * y for y in range(side) for x in range(side)]
    B = [x + Lx * y for y in range(side) for x in range(side + gap, 2 * side + gap)]
    strip = [x + Lx * y for y in range(Ly) for x in range(Lx // 2)]
    return A, B, strip


def served_requests(n=256, sizes=(256, 512, 1024, 2048, 4096), gamma_range=(0.1, 2.0), rate=None, seed=None):
    """Poisson stream of (arrival_time, L, protocol, gamma, traj_id) requests."""
    import numpy as np
    rng = np.random.default_rng(seed_of("served_mix") if seed is None else seed)
    rate = 50.0 if rate is None else rate
    t = np.cumsum(rng.exponential(1.0 / rate, size=n))
    Ls = rng.choice(list(sizes), size=n)
    prot = rng.choice(["projective", "homodyne"], size=n)
    gam = rng.uniform(gamma_range[0], gamma_range[1], size=n)
    return [(float(t[i]), int(Ls[i]), str(prot[i]), float(gam[i]), i) for i in range(n)]
