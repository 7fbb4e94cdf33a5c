// Blocked Cholesky G = R^dag R (upper R) and triangular inverse T = R^-1,
// batched over trajectories.  Diagonal 32 x 32 blocks are factored and
// inverted by one CTA each; panels and trailing updates are complex GEMMs.
#include <algorithm>

#include "kernels.h"

namespace fm {

template <typename TT>
cudaError_t cholesky_inverse(cudaStream_t st, cplx<TT>* G, cplx<TT>* R, cplx<TT>* T, cplx<TT>* Dinv, cplx<TT>* X,
                             int n, int ld, int64_t sNN, int alloc_n, int B, int* status, int64_t* launches) {
  const int nb = CHOL_NB;
  const int N = n;
  const int nblk = (N + nb - 1) / nb;
  const int64_t sD = (int64_t)((alloc_n + nb - 1) / nb) * nb * nb;
  const int64_t sX = (int64_t)alloc_n * nb;
  const cplx<TT> one = {(TT)1, (TT)0}, zero = {(TT)0, (TT)0}, mone = {(TT)-1, (TT)0};
  cudaError_t e;
  for (int k = 0; k < N; k += nb) {
    const int nbk = std::min(nb, N - k);
    if ((e = chol_diag_block(st, G, ld, sNN, R, ld, sNN, Dinv, sD, k, nb, nbk, B, status))) return e;
    ++*launches;
    const int rest = N - k - nbk;
    if (rest > 0) {
      cplx<TT>* Dk = Dinv + (int64_t)(k / nb) * nb * nb;
      // R12 = R11^-dag G12 ;  G22 -= R12^dag R12 (upper part)
      if ((e = zgemm<TT>(st, nbk, rest, nbk, OP_C, OP_N, one, Dk, nb, sD, G + k + (int64_t)(k + nbk) * ld, ld,
                             sNN, zero, R + k + (int64_t)(k + nbk) * ld, ld, sNN, B, 0)))
        return e;
      if ((e = zgemm<TT>(st, rest, rest, nbk, OP_C, OP_N, mone, R + k + (int64_t)(k + nbk) * ld, ld, sNN,
                             R + k + (int64_t)(k + nbk) * ld, ld, sNN, one, G + (k + nbk) + (int64_t)(k + nbk) * ld,
                             ld, sNN, B, GEMM_UPPER_ONLY)))
        return e;
      *launches += 2;
    }
  }
  if ((e = place_diag_blocks(st, Dinv, sD, T, ld, sNN, N, nb, B))) return e;
  ++*launches;
  for (int j = 1; j < nblk; ++j) {
    const int c0 = j * nb, nbj = std::min(nb, N - c0);
    // X = T[0:c0, 0:c0] R[0:c0, c0:c0+nbj] ;  T[0:c0, c0:c0+nbj] = -X Dinv_j
    if ((e = zgemm<TT>(st, c0, nbj, c0, OP_N, OP_N, one, T, ld, sNN, R + (int64_t)c0 * ld, ld, sNN, zero, X,
                           alloc_n, sX, B, GEMM_TRI_A_UPPER)))
      return e;
    if ((e = zgemm<TT>(st, c0, nbj, nbj, OP_N, OP_N, mone, X, alloc_n, sX, Dinv + (int64_t)j * nb * nb, nb, sD,
                           zero, T + (int64_t)c0 * ld, ld, sNN, B, 0)))
      return e;
    *launches += 2;
  }
  return cudaSuccess;
}

template cudaError_t cholesky_inverse<double>(cudaStream_t, z64*, z64*, z64*, z64*, z64*, int, int, int64_t, int, int,
                                              int*, int64_t*);
template cudaError_t cholesky_inverse<float>(cudaStream_t, c32*, c32*, c32*, c32*, c32*, int, int, int64_t, int, int,
                                             int*, int64_t*);

}  // namespace fm
