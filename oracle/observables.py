"""Observables of a Slater determinant (oracle side).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Sec. II: the entanglement entropy of a subsystem A is
S_A = - sum_i [lambda_i ln lambda_i + (1 - lambda_i) ln(1 - lambda_i)] over the
eigenvalues lambda_i of the correlation matrix restricted to A.  (The density
matrix form printed beside it lacks the overall minus sign; the eigenvalue
form fixes it.)  Natural logarithm; eigenvalues are clamped to [0, 1] and
0 ln 0 = 0.

Sec. IV: the mutual information I_2 = S_A + S_B - S_{A u B}.

Eq. (2): C_ij = -D_ij D_ji (= -|C_ij|^2), i != j, averaged over pairs at
distance r.
"""
import numpy as np


def correlation(U):
    """C = U U^dag (L x L); D_ij = <c_i^dag c_j> = conj(C_ij)."""
    return U @ np.conj(U).T


def binary_entropy_terms(lam):
    """f(lam) = lam ln lam + (1 - lam) ln(1 - lam), with f(0) = f(1) = 0."""
    lam = np.clip(np.asarray(lam, dtype=np.float64), 0.0, 1.0)
    out = np.zeros_like(lam)
    inner = (lam > 0.0) & (lam < 1.0)
    x = lam[inner]
    out[inner] = x * np.log(x) + (1.0 - x) * np.log1p(-x)
    return out


def subsystem_eigenvalues(U, sites):
    """Eigenvalues of C_A = U_A U_A^dag, A = ``sites``."""
    UA = U[np.asarray(sites, dtype=np.int64), :]
    CA = UA @ np.conj(UA).T
    return np.linalg.eigvalsh(CA)


def entanglement_entropy(U, sites):
    """S_A (nats) of the subsystem A = ``sites`` (Sec. II)."""
    if len(sites) == 0:
        return 0.0
    return float(-np.sum(binary_entropy_terms(subsystem_eigenvalues(U, sites))))


def mutual_information(U, A, B):
    """I_2 = S_A + S_B - S_{A u B} (Sec. IV); A and B must be disjoint."""
    A = list(A)
    B = list(B)
    if set(A) & set(B):
        raise ValueError("A and B overlap")
    return (entanglement_entropy(U, A) + entanglement_entropy(U, B)
            - entanglement_entropy(U, sorted(A + B)))


def displacement_correlation(U, Lx, Ly=1):
    """Eq. (2) per displacement class: c[d] = (1/L) sum_i C_{i, i+d}, C_ij = -D_ij D_ji = -|C_ij|^2,
    the partner site i + d taken with periodic wrap in x and in y, d = dx + Lx dy.

    c[0] = 0 (the paper uses i != j only).  On the ring C(r) = c[r] for r = 1 .. L/2, and
    c[d] = c[L - d].  Returns an array of L floats.
    """
    L = Lx * Ly
    C2 = np.abs(correlation(U)) ** 2
    site = np.arange(L)
    x, y = site % Lx, site // Lx
    out = np.zeros(L)
    for dy in range(Ly):
        for dx in range(Lx):
            d = dx + Lx * dy
            if d == 0:
                continue
            j = (x + dx) % Lx + Lx * ((y + dy) % Ly)
            out[d] = -float(np.mean(C2[site, j]))
    return out


def particle_covariance(U, A, B):
    """G_AB of Eq. (GAB) for one trajectory, the integral read as the lattice sum:
    G_AB = -sum_{i in A, j in B} C_ij = sum_{i in A, j in B} |C_ij|^2 (A, B disjoint)."""
    A = np.asarray(list(A), dtype=np.int64)
    B = np.asarray(list(B), dtype=np.int64)
    if set(A.tolist()) & set(B.tolist()):
        raise ValueError("A and B overlap")
    M = U[A, :] @ np.conj(U[B, :]).T
    return float(np.sum(np.abs(M) ** 2))
