"""The split-fp16 tcgen05 GEMM on its own, against float64 products (needs a GB300).

The planes represent x = h + l 2^-11; the kernel drops only the l*l product
(~2^-22 relative) and accumulates in fp32 in TMEM.  The accumulator is updated
once per 16-deep MMA and each update may lose up to one fp32 ulp of the
running sum (measured: the loss is biased toward zero on positive sums), so
the bound used is (K/16) 2^-23 max|partial sum| + 2^-22 sum|a b| -- still
three orders below the ~4e-3 relative error of a single fp16 product.
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
    lib.fmx_tc_gemm.restype = i32
    lib.fmx_tc_gemm.argtypes = [vp, vp, vp, vp, i32, i32, i32, vp, i32, i32, i32, i32, vp, vp]
    lib.fmx_tc_gram.restype = i32
    lib.fmx_tc_gram.argtypes = [vp, vp, i32, i32, i32, vp, i32, vp, vp]
    return torch, lib


def split(torch, x):
    h = x.to(torch.float16)
    l = ((x - h.to(torch.float32)) * 2048.0).to(torch.float16)
    return h, l


def joined(torch, h, l):
    return h.to(torch.float64) + l.to(torch.float64) / 2048.0


@pytest.mark.parametrize("M,N,K,BN,grid,chunk,raster", [
    (128, 256, 64, 256, 0, 0, 0),        # one tile, one K-block
    (256, 512, 1024, 256, 0, 0, 0),      # several tiles and K-blocks
    (384, 384, 320, 128, 0, 0, 0),       # BN = 128, K not a power of two
    (1024, 1024, 512, 128, 8, 0, 0),     # persistent: 8 CTAs walk 64 tiles
    (512, 768, 192, 256, 3, 0, 1),       # ragged tile count per CTA, computed raster
    (2304, 384, 256, 128, 5, 0, 1),      # raster with a partial last m-group (18 m-tiles)
    (256, 384, 1024, 128, 0, 2, 0),      # chunked accumulation, 8 chunks
    (512, 512, 320, 128, 3, 2, 1),       # chunked, last chunk ragged (5 K-blocks), persistent
    (128, 128, 64, 128, 1, 4, 1),        # chunked, one partial chunk
])
def test_plain_gemm(env, M, N, K, BN, grid, chunk, raster):
    torch, lib = env
    g = torch.Generator(device="cuda").manual_seed(M * 7 + N + K)
    A = torch.randn(M, K, device="cuda", generator=g)
    B = torch.randn(N, K, device="cuda", generator=g)
    Ah, Al = split(torch, A)
    Bh, Bl = split(torch, B)
    D = torch.full((N, M), float("nan"), device="cuda")        # column-major M x N
    ntiles = (M // 128) * (N // BN)
    tiles = torch.empty(ntiles * 16, dtype=torch.uint8, device="cuda")
    st = torch.cuda.current_stream().cuda_stream
    rc = lib.fmx_tc_gemm(Ah.data_ptr(), Al.data_ptr(), Bh.data_ptr(), Bl.data_ptr(), M, N, K, D.data_ptr(), BN,
                         grid, chunk, raster, tiles.data_ptr(), st)
    assert rc == 0
    torch.cuda.synchronize()
    ref = joined(torch, Ah, Al) @ joined(torch, Bh, Bl).T
    err = (D.T.to(torch.float64) - ref).abs().max().item()
    assert np.isfinite(err)
    assert err < 2e-6 * np.sqrt(K) * 16, err
    assert not torch.isnan(D).any().item()
    # the low planes matter: the hi-only product is far off
    hi_only = Ah.to(torch.float64) @ Bh.to(torch.float64).T
    assert (hi_only - ref).abs().max().item() > 50 * err


@pytest.mark.parametrize("L,N,B,BN", [(128, 128, 1, 128), (256, 128, 2, 128), (512, 256, 1, 256),
                                      (512, 512, 2, 256)])
def test_complex_gram(env, L, N, B, BN):
    torch, lib = env
    rng = np.random.default_rng(L + N + B)
    U = (rng.standard_normal((B, L, N)) + 1j * rng.standard_normal((B, L, N))) / np.sqrt(2 * L)
    V = np.concatenate([U.real, U.imag], axis=1)               # B x 2L x N, column k = [Re; Im]
    Vt = torch.tensor(np.ascontiguousarray(np.transpose(V, (0, 2, 1))), dtype=torch.float32, device="cuda")
    Vh, Vl = split(torch, Vt)                                   # memory = column-major 2L x N per b
    G = torch.zeros(B, N, N, 2, dtype=torch.float32, device="cuda")   # G[b, k2, k1] = G_b(k1, k2)
    mt, nt = N // 128, N // BN
    tiles = torch.empty(B * 2 * mt * nt * 16, dtype=torch.uint8, device="cuda")
    rc = lib.fmx_tc_gram(Vh.data_ptr(), Vl.data_ptr(), L, N, B, G.data_ptr(), BN, tiles.data_ptr(),
                         torch.cuda.current_stream().cuda_stream)
    assert rc == 0
    torch.cuda.synchronize()
    Vj = joined(torch, Vh, Vl).cpu().numpy()                    # B x N x 2L
    Uj = np.transpose(Vj[:, :, :L] + 1j * Vj[:, :, L:], (0, 2, 1))
    Gc = G[..., 0].double().cpu().numpy() + 1j * G[..., 1].double().cpu().numpy()
    for b in range(B):
        ref = Uj[b].conj().T @ Uj[b]
        got = Gc[b].T
        iu = np.triu_indices(N)
        err = np.max(np.abs(got[iu] - ref[iu]))
        bound = (2 * L / 16) * 2.0 ** -23 * np.max(np.abs(ref)) + 2.0 ** -24 * np.max(np.abs(ref)) + 1e-7
        assert err < bound, (err, bound)


def test_chunked_accumulation_is_more_accurate_on_long_positive_sums(env):
    """Sums of K positive products: the chunked kernel keeps the fp32 rounding unbiased."""
    torch, lib = env
    M, N, K = 128, 128, 16384
    g = torch.Generator(device="cuda").manual_seed(5)
    A = torch.rand(M, K, device="cuda", generator=g) / np.sqrt(K)
    B = torch.rand(N, K, device="cuda", generator=g) / np.sqrt(K)
    Ah, Al = split(torch, A)
    Bh, Bl = split(torch, B)
    ref = joined(torch, Ah, Al) @ joined(torch, Bh, Bl).T
    errs = {}
    for chunk in (0, 2):
        D = torch.empty(N, M, device="cuda")
        tiles = torch.empty(16, dtype=torch.uint8, device="cuda")
        rc = lib.fmx_tc_gemm(Ah.data_ptr(), Al.data_ptr(), Bh.data_ptr(), Bl.data_ptr(), M, N, K, D.data_ptr(),
                             128, 1, chunk, 1, tiles.data_ptr(), torch.cuda.current_stream().cuda_stream)
        assert rc == 0
        torch.cuda.synchronize()
        errs[chunk] = ((D.T.to(torch.float64) - ref) / ref).abs().max().item()
    print("relative error, K=16384 positive sums: unchunked %.2e, chunked %.2e" % (errs[0], errs[2]))
    assert errs[2] < 2e-6
    assert errs[2] < errs[0]


def _digits(Z, e):
    """Five signed 7-bit digits of every row of Z (float64) scaled by 2^-e_r, toward zero."""
    x = np.ldexp(Z, (7 - e)[:, None])
    out = []
    for _ in range(5):
        q = np.trunc(x)
        out.append(q.astype(np.int64))
        x = (x - q) * 128.0
    return out


def exact_gram_reference(X):
    """The exact-product Gram of the float-valued block X (n x N complex), written from
    the digit definition: integer digit products by class (s + t <= 6) in int64, then
    M = 2^(e_i+e_j-28) H + 2^(e_i+e_j-56) Lo, H and Lo the classes 0-2 and 3-6."""
    n, N = X.shape
    Y = X if n <= N else X.T
    Z = np.concatenate([Y.real, Y.imag], axis=1)
    Zs = np.concatenate([Y.imag, -Y.real], axis=1)          # rows read at K + Kp, negated past the wrap
    mx = np.max(np.abs(Z), axis=1)
    e = np.where(mx > 0, np.frexp(mx)[1], 0).astype(np.int64)    # max < 2^e, exactly
    D = _digits(Z, e)
    Ds = _digits(Zs, e)
    out = []
    for B in (D, Ds):
        A = [sum(D[s] @ B[c - s].T for s in range(5) if 0 <= c - s < 5) for c in range(7)]
        H = (A[0] << 14) + (A[1] << 7) + A[2]
        Lo = (A[3] << 21) + (A[4] << 14) + (A[5] << 7) + A[6]
        ee = e[:, None] + e[None, :]
        out.append(np.ldexp(H.astype(np.float64), ee - 28) + np.ldexp(Lo.astype(np.float64), ee - 56))
    return out[0] - 1j * out[1]


@pytest.mark.parametrize("n,N", [(200, 384), (300, 256), (640, 512), (513, 768)])
def test_exact_gram_is_bit_exact_to_its_digit_definition(env, n, N):
    torch, lib = env
    lib.fmx_exact_gram.restype = ctypes.c_int
    lib.fmx_exact_gram.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p,
                                   ctypes.c_void_p]
    lib.fmx_exact_gram_scratch_bytes.restype = ctypes.c_ulonglong
    lib.fmx_exact_gram_scratch_bytes.argtypes = [ctypes.c_int, ctypes.c_int]
    rng = np.random.default_rng(n * 1000 + N)
    scale = np.ldexp(1.0, rng.integers(-12, 3, size=(n, 1)))
    X = ((rng.standard_normal((n, N)) + 1j * rng.standard_normal((n, N))) * scale)
    X = (X.real.astype(np.float32) + 1j * X.imag.astype(np.float32)).astype(np.complex128)
    X[3] = 0.0                                                  # a zero row
    X[:, 5] *= 1e-6                                             # entries far below their row maxima
    m = min(n, N)
    dX = torch.from_numpy(np.asfortranarray(X).T.copy().reshape(-1).view(np.float64)).cuda()
    dM = torch.zeros(2 * m * m, dtype=torch.float64, device="cuda")
    scratch = torch.empty(int(lib.fmx_exact_gram_scratch_bytes(n, N)), dtype=torch.uint8, device="cuda")
    rc = lib.fmx_exact_gram(dX.data_ptr(), n, N, dM.data_ptr(), scratch.data_ptr(),
                            torch.cuda.current_stream().cuda_stream)
    assert rc == 0
    torch.cuda.synchronize()
    M = dM.cpu().numpy().view(np.complex128).reshape(m, m).T     # column-major
    ref = exact_gram_reference(X)
    low = np.tril(np.ones((m, m), dtype=bool))
    assert np.array_equal(M[low], ref[low])
    # and it is the Gram of X to the truncation bound
    G = X @ X.conj().T if n <= N else X.T @ X.conj()
    Y = X if n <= N else X.T
    rowmax = np.max(np.maximum(np.abs(Y.real), np.abs(Y.imag)), axis=1)
    bound = 2.0 ** -24 * (rowmax[:, None] * np.sum(np.abs(Y), axis=1)[None, :] +
                          rowmax[None, :] * np.sum(np.abs(Y), axis=1)[:, None]) + 1e-300
    assert np.all(np.abs(M - G)[low] <= bound[low])
