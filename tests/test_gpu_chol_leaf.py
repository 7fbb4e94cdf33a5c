"""The Cholesky leaf of the mixed-precision CholeskyQR (128 x 128 blocks and
smaller, complex64, one CTA per block) against the float64 textbook Cholesky
(needs a GB300).

For G = X^dag X with X a 3n x n Gaussian matrix (condition number of R about
(sqrt(3) + 1) / (sqrt(3) - 1) ~ 4), the float32 factor satisfies
|R - R_ref| <= c n u |R| and |T R - 1| <= c n u with u = 2^-24; the bars below
(2e-5, i.e. ~2.5 n u at n = 128 including the condition number) leave room for
accumulation order only.
"""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2508_18468_gb300 import build
    build.build()
    from paper_2508_18468_gb300 import fm
    lib = fm.lib
    vp, i32 = ctypes.c_void_p, ctypes.c_int
    lib.fmx_chol_leaf.restype = i32
    lib.fmx_chol_leaf.argtypes = [vp, i32, i32, i32, vp, vp, vp, vp]
    return torch, lib


def run_leaf(torch, lib, Gs, n, ld):
    B = len(Gs)
    buf = np.zeros((B, n, ld), np.complex64)   # block b, column c, row r (column-major, ld rows)
    for b, G in enumerate(Gs):
        buf[b, :, :n] = G.T.astype(np.complex64)
        buf[b, :, n:] = np.nan                   # padding rows are never read
    dG = torch.from_numpy(buf.view(np.float32).copy()).cuda()
    dR = torch.full_like(dG, np.nan)
    dT = torch.full_like(dG, np.nan)
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    rc = lib.fmx_chol_leaf(dG.data_ptr(), n, ld, B, dR.data_ptr(), dT.data_ptr(), st.data_ptr(), None)
    assert rc == 0
    torch.cuda.synchronize()
    R = dR.cpu().numpy().view(np.complex64).reshape(B, n, ld)[:, :, :n].transpose(0, 2, 1)
    T = dT.cpu().numpy().view(np.complex64).reshape(B, n, ld)[:, :, :n].transpose(0, 2, 1)
    return R.astype(np.complex128), T.astype(np.complex128), int(st.item())


@pytest.mark.parametrize("n,ld", [(128, 128), (128, 200), (100, 128), (64, 64), (33, 40), (32, 32), (7, 7),
                                  (1, 1)])
def test_leaf_matches_float64_cholesky(env, n, ld):
    torch, lib = env
    rng = np.random.default_rng(n * 1000 + ld)
    Gs = []
    for _ in range(3):
        X = rng.standard_normal((3 * n, n)) + 1j * rng.standard_normal((3 * n, n))
        Gs.append(X.conj().T @ X)
    R, T, status = run_leaf(torch, lib, Gs, n, ld)
    assert status == 0
    for b in range(3):
        Rref = np.linalg.cholesky(Gs[b]).conj().T
        assert np.all(R[b][np.tril_indices(n, -1)] == 0) and np.all(T[b][np.tril_indices(n, -1)] == 0)
        assert np.all(np.diag(R[b]).imag == 0) and np.all(np.diag(R[b]).real > 0)
        err_r = np.abs(R[b] - Rref).max() / np.abs(Rref).max()
        err_t = np.abs(T[b] @ R[b] - np.eye(n)).max()
        print("n %d ld %d b %d: |R - R_ref| / |R| %.2e, |T R - 1| %.2e" % (n, ld, b, err_r, err_t))
        assert err_r <= 2e-5 and err_t <= 2e-5


def test_leaf_identity_and_diagonal_blocks(env):
    """G = diag(g): R = diag(sqrt g), T = diag(1 / sqrt g) up to rounding of sqrt."""
    torch, lib = env
    g = np.linspace(0.5, 4.0, 128)
    R, T, status = run_leaf(torch, lib, [np.diag(g), np.eye(128)], 128, 128)
    assert status == 0
    np.testing.assert_allclose(R[0], np.diag(np.sqrt(g)), rtol=1e-7, atol=0)
    np.testing.assert_allclose(T[0], np.diag(1 / np.sqrt(g)), rtol=2e-7, atol=0)
    assert np.array_equal(R[1], np.eye(128)) and np.array_equal(T[1], np.eye(128))


def test_leaf_flags_a_non_positive_pivot(env):
    """An indefinite block raises the pivot flag; the outputs stay finite."""
    torch, lib = env
    G = np.eye(64, dtype=np.complex128)
    G[40, 40] = -1.0
    R, T, status = run_leaf(torch, lib, [G], 64, 64)
    assert status & 1
    assert np.all(np.isfinite(R)) and np.all(np.isfinite(T))
