"""fm_entropy_noalloc against fm_entropy (needs a GB300).

fm_entropy_noalloc is for callers that must not allocate device memory --
for instance an application whose own memory pool already holds almost all
of the GPU, or a loop that cannot afford the synchronisation that freeing
memory implies.  Its scratch is a fixed array in the library's static device
memory.  This test hands it a device copy of a trajectory's orbitals and
checks two calls in a row (and a third of the other eigenproblem shape)
against fm_entropy on the same state, at the FP64 tolerance of the other
entropy tests, then checks that oversized requests are refused.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

S_TOL = 1e-9


def test_noalloc_entropy_matches_fm_entropy():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2508_18468_gb300 import build
    build.build()
    from paper_2508_18468_gb300 import fm

    L, N = 96, 48
    g = fm.Trajectories(fm.make_params(L, protocol=fm.FM_HOMODYNE, precision=fm.FM_FP64, gamma=1.0, seed=13))
    g.step(25)
    U = g.copy_U()                                                   # L x N, column-major
    dU = torch.from_numpy(np.ascontiguousarray(U.T)).to("cuda")      # rows = columns of U
    dS = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream

    cases = [list(range(N)),                                          # half chain, n = N
             [0, 5, 7, 20, 33, 60, 61, 95] + list(range(70, 90)),     # scattered, n < N
             list(range(60))]                                         # n > N: the N x N eigenproblem
    for sites in cases:
        rc = fm.fm_entropy_noalloc(dU.data_ptr(), L, N, sites, dS.data_ptr(), stream)
        assert rc == fm.FM_OK
        torch.cuda.synchronize()
        got, ref = dS.item(), g.entropy(sites)
        assert abs(got - ref) <= S_TOL * max(1.0, abs(ref)), (sites[:4], got, ref)

    # the largest eigenproblem size takes the multi-kernel reduction path (m > 256)
    g2 = fm.Trajectories(fm.make_params(1024, protocol=fm.FM_PROJECTIVE, precision=fm.FM_FP64, gamma=1.0,
                                        seed=14))
    g2.step(6)
    dU2 = torch.from_numpy(np.ascontiguousarray(g2.copy_U().T)).to("cuda")
    sites2 = list(range(0, 1024, 3))[:300]
    rc = fm.fm_entropy_noalloc(dU2.data_ptr(), 1024, 512, sites2, dS.data_ptr(), stream)
    assert rc == fm.FM_OK
    torch.cuda.synchronize()
    got, ref = dS.item(), g2.entropy(sites2)
    assert abs(got - ref) <= S_TOL * max(1.0, abs(ref)), (got, ref)

    # sizes beyond the fixed scratch, and bad site lists, are refused up front
    assert fm.fm_entropy_noalloc(dU.data_ptr(), L, N, [0, 0], dS.data_ptr(), stream) == fm.FM_EINVAL
    assert fm.fm_entropy_noalloc(dU.data_ptr(), L, N, [L], dS.data_ptr(), stream) == fm.FM_EINVAL
    assert fm.fm_entropy_noalloc(dU.data_ptr(), 4096, 2048, [0], dS.data_ptr(), stream) == fm.FM_EINVAL
    big = list(range(1025))
    assert fm.fm_entropy_noalloc(dU.data_ptr(), 4096, 512, big, dS.data_ptr(), stream) == fm.FM_EINVAL
