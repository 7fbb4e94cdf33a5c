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


def density_correlation(U, Lx, Ly=1):
    """C(r) of Eq. (2) on a ring: mean of -|C_ij|^2 over pairs with ring distance r.

    Returns an array indexed by r = 1 .. L//2 (entry 0 unused, set to 0).
    """
    if Ly != 1:
        raise ValueError("density_correlation: ring only")
    L = Lx
    C2 = np.abs(correlation(U)) ** 2
    out = np.zeros(L // 2 + 1)
    i = np.arange(L)
    for r in range(1, L // 2 + 1):
        # each unordered pair at distance r once (r = L/2 pairs are met twice)
        vals = C2[i, (i + r) % L]
        out[r] = -float(np.mean(vals))
    return out
