"""Brute-force many-body state vector for small lattices (test-only checker).

Written independently of ``oracle/``: it never forms the orbital matrix U after
the start, it works with the full N-particle wave function in the occupation
basis.  Used to pin the oracle's propagation, measurement updates and
entropies (App. A, Sec. II).

Conventions.  A basis state is a bit string s, bit i = occupation of site i,
and |s> = c^dag_{a1} c^dag_{a2} ... c^dag_{aN} |vac> with a1 < a2 < ... .
Then c_j |s> = (-1)^{#occupied sites below j} |s - j>, and the amplitude of the
Slater determinant prod_k (sum_j U_jk c_j^dag)|vac> on |s> is det(U[S, :]).
"""
import itertools

import numpy as np
import scipy.linalg


def _popcount_below(s, i):
    return bin(s & ((1 << i) - 1)).count("1")


def ring_bonds(L):
    return [(i, (i + 1) % L) for i in range(L)]


def torus_bonds(Lx, Ly):
    bonds = []
    for y in range(Ly):
        for x in range(Lx):
            i = x + Lx * y
            bonds.append((i, (x + 1) % Lx + Lx * y))
            bonds.append((i, x + Lx * ((y + 1) % Ly)))
    return bonds


class Sector:
    """The fixed-N sector of L fermionic modes."""

    def __init__(self, L, N):
        self.L, self.N = L, N
        self.states = [sum(1 << i for i in c) for c in itertools.combinations(range(L), N)]
        self.index = {s: k for k, s in enumerate(self.states)}
        self.dim = len(self.states)
        self.occ = np.array([[(s >> i) & 1 for i in range(L)] for s in self.states], dtype=np.float64)
        self._hop = {}

    def hop(self, i, j):
        """Sparse c_i^dag c_j: (src, dst, sign) index arrays."""
        key = (i, j)
        if key not in self._hop:
            src, dst, sgn = [], [], []
            for k, s in enumerate(self.states):
                if i == j:
                    if (s >> i) & 1:
                        src.append(k); dst.append(k); sgn.append(1.0)
                    continue
                if not (s >> j) & 1 or (s >> i) & 1:
                    continue
                sign = (-1) ** _popcount_below(s, j)
                s1 = s ^ (1 << j)
                sign *= (-1) ** _popcount_below(s1, i)
                src.append(k); dst.append(self.index[s1 | (1 << i)]); sgn.append(float(sign))
            self._hop[key] = (np.array(src, dtype=np.int64), np.array(dst, dtype=np.int64),
                              np.array(sgn))
        return self._hop[key]

    def hamiltonian(self, bonds, J=1.0):
        H = np.zeros((self.dim, self.dim))
        for a, b in bonds:
            for (i, j) in ((a, b), (b, a)):
                src, dst, sgn = self.hop(i, j)
                np.add.at(H, (dst, src), J * sgn)
        return H

    def from_orbitals(self, U):
        psi = np.empty(self.dim, dtype=np.complex128)
        for k, s in enumerate(self.states):
            S = [i for i in range(self.L) if (s >> i) & 1]
            psi[k] = np.linalg.det(U[S, :])
        return psi

    def d_matrix(self, psi):
        """D_ij = <psi| c_i^dag c_j |psi>."""
        D = np.zeros((self.L, self.L), dtype=np.complex128)
        for i in range(self.L):
            for j in range(self.L):
                src, dst, sgn = self.hop(i, j)
                D[i, j] = np.sum(np.conj(psi[dst]) * sgn * psi[src])
        return D

    def occupation(self, psi):
        return self.occ.T @ (np.abs(psi) ** 2)

    def project(self, psi, j, outcome):
        """Apply n_j (outcome 1) or 1 - n_j (outcome 0) and normalise; also the Born weight."""
        keep = self.occ[:, j] == outcome
        out = np.where(keep, psi, 0.0)
        w = float(np.sum(np.abs(out) ** 2))
        return out / np.sqrt(w), w

    def weight(self, psi, m):
        """psi(s) <- exp(sum_i m_i n_i(s)) psi(s), normalised."""
        out = np.exp(self.occ @ m) * psi
        return out / np.linalg.norm(out)

    def entropy(self, psi, sites):
        """Von Neumann entropy of the fermionic reduced state of ``sites``.

        The modes are reordered so that ``sites`` come first (each basis
        amplitude picks up the sign of the permutation of its occupied
        modes); the first |A| modes then factor off as in a tensor product
        and the Schmidt values come from an SVD.
        """
        A = list(sites)
        rest = [i for i in range(self.L) if i not in A]
        order = A + rest
        nA = len(A)
        M = np.zeros((1 << nA, 1 << (self.L - nA)), dtype=np.complex128)
        for k, s in enumerate(self.states):
            occ_new = [p for p, site in enumerate(order) if (s >> site) & 1]
            old = [order[p] for p in occ_new]
            # sign of the permutation sorting `old` (new order) into ascending site order
            inv = sum(1 for a in range(len(old)) for b in range(a + 1, len(old)) if old[a] > old[b])
            sign = -1.0 if inv % 2 else 1.0
            ia = sum(1 << p for p in occ_new if p < nA)
            ib = sum(1 << (p - nA) for p in occ_new if p >= nA)
            M[ia, ib] += sign * psi[k]
        sv = np.linalg.svd(M, compute_uv=False)
        w = sv ** 2
        w = w[w > 1e-300]
        return float(-np.sum(w * np.log(w)))


def evolution_operator(sector, bonds, J, dt):
    return scipy.linalg.expm(-1j * dt * sector.hamiltonian(bonds, J))
