"""Lattice, propagator and initial orbitals (oracle side).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Sec. II: H = J sum_i (c_i^dag c_{i+1} + h.c.) on a ring of L sites with
periodic boundary conditions, so the single-particle matrix of App. A is
H~_ij = J (delta_{j,i+1} + delta_{j,i-1}) (indices mod L).  Sec. IV uses the
same Hamiltonian on an Lx x Ly square lattice; periodic boundaries are taken
in both directions and site (x, y) has index i = x + Lx*y.

The propagator exp(-i H~ dt) of App. A is built from the plane-wave
eigenvectors of H~: on a ring, H~ e^{ika} = 2J cos(k) e^{ika} with
k = 2 pi m / L, so

    P_ab = (1/L) sum_m exp(i k (a-b)) exp(-2 i J dt cos k),

a circulant matrix.  On the torus H~ = H~_x (+) H~_y commute, so
P = P_y (x) P_x in the index x + Lx*y.
"""
import numpy as np


def n_sites(Lx, Ly=1):
    return int(Lx) * int(Ly)


def hopping_matrix(Lx, Ly=1, J=1.0):
    """H~ (L x L, real): J on every nearest-neighbour bond, periodic."""
    L = n_sites(Lx, Ly)
    H = np.zeros((L, L))
    for y in range(Ly):
        for x in range(Lx):
            i = x + Lx * y
            nbrs = [((x + 1) % Lx) + Lx * y] if Lx > 1 else []
            if Ly > 1:
                nbrs.append(x + Lx * ((y + 1) % Ly))
            for j in nbrs:
                # one bond term c_i^dag c_j + c_j^dag c_i per neighbour pair
                H[i, j] += J
                H[j, i] += J
    return H


def ring_propagator_row(L, J, dt):
    """p[r] = (1/L) sum_m exp(2 pi i m r / L) exp(-2 i J dt cos(2 pi m / L)).

    The angle m*r is reduced mod L in integers before scaling, so every term
    is accurate to a few ulp at any L.
    """
    m = np.arange(L, dtype=np.int64)
    phase = np.exp(-2j * J * dt * np.cos(2.0 * np.pi * m / L))
    p = np.empty(L, dtype=np.complex128)
    chunk = max(1, (1 << 22) // max(L, 1))
    for r0 in range(0, L, chunk):
        r = np.arange(r0, min(L, r0 + chunk), dtype=np.int64)
        ang = 2.0 * np.pi * ((r[:, None] * m[None, :]) % L) / L
        p[r0:r0 + len(r)] = (np.exp(1j * ang) @ phase) / L
    return p


def ring_propagator(L, J, dt):
    """exp(-i H~ dt) on a ring (L x L complex128): P_ab = p[(a - b) mod L]."""
    p = ring_propagator_row(L, J, dt)
    a = np.arange(L)
    return p[(a[:, None] - a[None, :]) % L]


def propagator(Lx, Ly, J, dt):
    """exp(-i H~ dt) for the ring (Ly == 1) or the Lx x Ly torus."""
    Px = ring_propagator(Lx, J, dt) if Lx > 1 else np.ones((1, 1), complex)
    if Ly == 1:
        return Px
    Py = ring_propagator(Ly, J, dt)
    return np.kron(Py, Px)


def occupied_sites(Lx, Ly=1):
    """Neel start of App. A, |1010...>: even sites occupied (site 0 first).

    On the torus the analogous checkerboard: (x + y) even.
    """
    if Ly == 1:
        return np.arange(0, Lx, 2)
    return np.array([x + Lx * y for y in range(Ly) for x in range(Lx) if (x + y) % 2 == 0])


def initial_orbitals(Lx, Ly=1):
    """U0 (L x N): column k is the unit vector on the k-th occupied site."""
    L = n_sites(Lx, Ly)
    occ = occupied_sites(Lx, Ly)
    U = np.zeros((L, len(occ)), dtype=np.complex128)
    U[occ, np.arange(len(occ))] = 1.0
    return U
