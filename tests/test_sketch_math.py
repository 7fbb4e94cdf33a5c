"""The mathematics of the entropy sketch, in numpy on oracle states (CPU).

The GPU sketch (FM_EE_SKETCH) computes S_A from the Rayleigh-Ritz values of the cross
block C_AB = U_A U_B^dag over a randomized subspace.  Written out here with the same
steps -- complex64 products, two shifted CholeskyQR passes, one power iteration -- it must
give the exact entropy of an orthonormal state, and on a complex64-rounded state
(orthonormal only to ~1e-7) it must still give the exact entropy to ~1e-8, because the
rounding enters sigma^2 at second order, while C_A's own eigenvalues move at first order.
"""
import numpy as np
import pytest

from oracle import observables, trajectory
from oracle.trajectory import HOMODYNE, Params


def c64(M):
    return M.astype(np.complex64).astype(np.complex128)


def orth(Y):
    n, r = Y.shape
    for _ in range(2):
        G = Y.conj().T @ Y
        G = G + 11 * (n * r + r * (r + 1)) * 2.0**-53 * np.trace(G).real * np.eye(r)
        R = np.linalg.cholesky(G).conj().T
        Y = Y @ np.linalg.inv(R)
    return Y


def entropy_of_sigma2(x):
    y = np.clip(x, 0.0, 0.25)
    lam = 2 * y / (1 + np.sqrt(1 - 4 * y))
    lam = lam[(lam > 0) & (lam < 1)]
    return float(-np.sum(lam * np.log(lam) + (1 - lam) * np.log1p(-lam)))


def sketch(U, A, r, rounded, seed=0):
    L = U.shape[0]
    B = [i for i in range(L) if i not in set(A)]
    XA, XB = U[A], U[B]
    f = c64 if rounded else (lambda M: M)
    rng = np.random.default_rng(seed)
    Om = (rng.choice([-1.0, 1.0], (len(B), r)) + 1j * rng.choice([-1.0, 1.0], (len(B), r))) / np.sqrt(2)
    Q = orth(f(XA @ f(XB.conj().T @ Om)))
    P = orth(f(XB @ f(XA.conj().T @ Q)))
    Q = orth(f(XA @ f(XB.conj().T @ P)))
    Bh = f(XB @ f(XA.conj().T @ Q))
    x = np.sort(np.linalg.eigvalsh(Bh.conj().T @ Bh))
    return entropy_of_sigma2(x), x[max(8, r // 8) - 1]


@pytest.mark.parametrize("L,steps,sites", [(512, 80, (200, 456)), (384, 40, (0, 192))])
def test_sketch_reproduces_the_exact_entropy(L, steps, sites):
    U = trajectory.run(Params(Lx=L, gamma=0.5, protocol=HOMODYNE, seed=3), steps)["U"]
    A = list(range(*sites))
    S = observables.entanglement_entropy(U, A)
    S_sk, chk = sketch(U, A, 64, rounded=False)
    assert chk < 1e-9                                   # converged: the sketch holds every mode
    assert abs(S_sk - S) <= 1e-9 * max(S, 1.0)
    # the complex64-rounded state, products in complex64
    Ur = c64(U)
    S_r, chk_r = sketch(Ur, A, 64, rounded=True)
    assert chk_r < 1e-9
    assert abs(S_r - S) <= 2e-7 * max(S, 1.0)
    # C_A of the same rounded state, without a projector correction, is biased at first order
    S_direct = observables.entanglement_entropy(Ur, A)
    assert abs(S_direct - S) > 10 * abs(S_r - S)
