"""fm_entropy_noalloc against the FP64 oracle and fm_entropy (needs a GB300).

fm_entropy_noalloc is for callers that must not allocate device memory -- for
instance an application whose own memory pool already holds almost all of the
GPU, or a loop that cannot afford the synchronisation that freeing memory
implies.  Its scratch is a fixed array in the library's static device memory.
This test hands it a device copy of a trajectory's orbitals and checks two calls
in a row (and a third of the other eigenproblem shape) against the oracle's
entropy of the same orbitals (numpy eigenvalues, no code shared with the library)
and against fm_entropy, at the FP64 tolerance of the other entropy tests; that the
device's free memory is the same before and after the calls; that an empty
subsystem gives S = 0; and that oversized requests are refused.
"""
import numpy as np
import pytest

from oracle import observables

pytestmark = pytest.mark.gpu

S_TOL = 1e-9


def test_noalloc_entropy_matches_oracle_and_fm_entropy():
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
    via_state = [g.entropy(sites) for sites in cases]                 # fm_entropy on the same state
    # warm-up call: the first call on a device looks up the scratch array's address
    assert fm.fm_entropy_noalloc(dU.data_ptr(), L, N, cases[0], dS.data_ptr(), stream) == fm.FM_OK
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for sites, S_state in zip(cases, via_state):
        rc = fm.fm_entropy_noalloc(dU.data_ptr(), L, N, sites, dS.data_ptr(), stream)
        assert rc == fm.FM_OK
        torch.cuda.synchronize()
        got = dS.item()
        ref = observables.entanglement_entropy(U, sites)
        assert abs(got - ref) <= S_TOL * max(1.0, abs(ref)), (sites[:4], got, ref)
        assert abs(got - S_state) <= S_TOL * max(1.0, abs(ref))
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0                      # nothing allocated on the device
    # an empty subsystem: S = 0
    dS.fill_(float("nan"))
    assert fm.fm_entropy_noalloc(dU.data_ptr(), L, N, [], dS.data_ptr(), stream) == fm.FM_OK
    torch.cuda.synchronize()
    assert dS.item() == 0.0
    # the largest eigenproblem size takes the multi-kernel reduction path (m > 256)
    g2 = fm.Trajectories(fm.make_params(1024, protocol=fm.FM_PROJECTIVE, precision=fm.FM_FP64, gamma=1.0,
                                        seed=14))
    g2.step(6)
    U2 = g2.copy_U()
    dU2 = torch.from_numpy(np.ascontiguousarray(U2.T)).to("cuda")
    sites2 = list(range(0, 1024, 3))[:300]
    torch.cuda.synchronize()
    free1 = torch.cuda.mem_get_info()[0]
    for _ in range(2):
        rc = fm.fm_entropy_noalloc(dU2.data_ptr(), 1024, 512, sites2, dS.data_ptr(), stream)
        assert rc == fm.FM_OK
        torch.cuda.synchronize()
        got, ref = dS.item(), observables.entanglement_entropy(U2, sites2)
        assert abs(got - ref) <= S_TOL * max(1.0, abs(ref)), (got, ref)
    torch.cuda.synchronize()
    # no device memory was taken by the calls
    assert torch.cuda.mem_get_info()[0] == free1

    # sizes beyond the fixed scratch, and bad site lists, are refused up front
    assert fm.fm_entropy_noalloc(dU.data_ptr(), L, N, [0, 0], dS.data_ptr(), stream) == fm.FM_EINVAL
    assert fm.fm_entropy_noalloc(dU.data_ptr(), L, N, [L], dS.data_ptr(), stream) == fm.FM_EINVAL
    assert fm.fm_entropy_noalloc(dU.data_ptr(), 4096, 2048, [0], dS.data_ptr(), stream) == fm.FM_EINVAL
    big = list(range(1025))
    assert fm.fm_entropy_noalloc(dU.data_ptr(), 4096, 512, big, dS.data_ptr(), stream) == fm.FM_EINVAL
