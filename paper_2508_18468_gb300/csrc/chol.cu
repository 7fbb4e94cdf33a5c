// Blocked FP64 Cholesky G = R^dag R (upper R) and triangular inverse T = R^-1,
// batched over trajectories.  Diagonal 32 x 32 blocks are factored and
// inverted by one CTA each; panels and trailing updates are complex GEMMs.
#include <algorithm>

#include "kernels.h"

namespace fm {

cudaError_t cholesky_inverse_f64(cudaStream_t st, z64* G, z64* R, z64* T, z64* Dinv, z64* X, int n, int ld,
                                 int64_t sNN, int alloc_n, int B, int* status, int64_t* launches) {
  const int nb = CHOL_NB;
  const int N = n;
  const int nblk = (N + nb - 1) / nb;
  const int64_t sD = (int64_t)((alloc_n + nb - 1) / nb) * nb * nb;
  const int64_t sX = (int64_t)alloc_n * nb;
  const z64 one = {1.0, 0.0}, zero = {0.0, 0.0}, mone = {-1.0, 0.0};
  cudaError_t e;
  for (int k = 0; k < N; k += nb) {
    const int nbk = std::min(nb, N - k);
    if ((e = chol_diag_block(st, G, ld, sNN, R, ld, sNN, Dinv, sD, k, nb, nbk, B, status))) return e;
    ++*launches;
    const int rest = N - k - nbk;
    if (rest > 0) {
      z64* Dk = Dinv + (int64_t)(k / nb) * nb * nb;
      // R12 = R11^-dag G12 ;  G22 -= R12^dag R12 (upper part)
      if ((e = zgemm<double>(st, nbk, rest, nbk, OP_C, OP_N, one, Dk, nb, sD, G + k + (int64_t)(k + nbk) * ld, ld,
                             sNN, zero, R + k + (int64_t)(k + nbk) * ld, ld, sNN, B, 0)))
        return e;
      if ((e = zgemm<double>(st, rest, rest, nbk, OP_C, OP_N, mone, R + k + (int64_t)(k + nbk) * ld, ld, sNN,
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
    if ((e = zgemm<double>(st, c0, nbj, c0, OP_N, OP_N, one, T, ld, sNN, R + (int64_t)c0 * ld, ld, sNN, zero, X,
                           alloc_n, sX, B, GEMM_TRI_A_UPPER)))
      return e;
    if ((e = zgemm<double>(st, c0, nbj, nbj, OP_N, OP_N, mone, X, alloc_n, sX, Dinv + (int64_t)j * nb * nb, nb, sD,
                           zero, T + (int64_t)c0 * ld, ld, sNN, B, 0)))
      return e;
    *launches += 2;
  }
  return cudaSuccess;
}

}  // namespace fm
