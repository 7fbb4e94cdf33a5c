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

// ------------------------------------------------------------------ one-CTA leaf
// G = R^dag R and T = R^-1 for an n x n block (n <= 128) of every trajectory,
// complex64, in shared memory: right-looking Cholesky on the upper triangle,
// then T by 32 x 32 blocks -- each diagonal block inverted by one warp (a
// column per lane), then T_IJ = -T_II sum_{I < K <= J} R_IK T_KJ by all
// threads, J ascending, I descending -- with T^T kept in the strict lower
// triangle of the same array.  R and T are written with zeros below the
// diagonal.  One CTA of 1024 threads per trajectory; a non-positive pivot
// raises FM_DEVERR_PIVOT and continues with pivot 1.
namespace fm {

constexpr int kLeafMax = 128;
constexpr int kLeafLd = kLeafMax + 1;
constexpr size_t kLeafSmem = ((size_t)kLeafMax * kLeafLd + kLeafMax + 32 * 33) * sizeof(c32);

__global__ void __launch_bounds__(1024) chol_inv_leaf_kernel(const c32* __restrict__ G, c32* R, c32* T, int n,
                                                             int64_t ld, int64_t sNN, int* status) {
  extern __shared__ c32 sm[];
  c32* A = sm;                                  // A[r * kLeafLd + c]
  c32* Td = sm + kLeafMax * kLeafLd;            // diagonal of T
  c32* Z = Td + kLeafMax;                       // 32 x 33 block scratch
  const int64_t b = blockIdx.x;
  G += b * sNN;
  R += b * sNN;
  T += b * sNN;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  for (int idx = tid; idx < n * n; idx += blockDim.x) {
    const int r = idx % n, c = idx / n;
    A[r * kLeafLd + c] = r <= c ? G[r + (int64_t)c * ld] : cmk(0.0f, 0.0f);
  }
  __syncthreads();
  for (int j = 0; j < n; ++j) {
    if (tid == 0) {
      float d = A[j * kLeafLd + j].re;
      if (!(d > 0.0f) || !isfinite(d)) {
        atomicOr(status, FM_DEVERR_PIVOT);
        d = 1.0f;
      }
      A[j * kLeafLd + j] = cmk(sqrtf(d), 0.0f);
    }
    __syncthreads();
    const float inv = 1.0f / A[j * kLeafLd + j].re;
    for (int c = j + 1 + tid; c < n; c += blockDim.x) A[j * kLeafLd + c] = cscale(A[j * kLeafLd + c], inv);
    __syncthreads();
    const int m = n - j - 1;                    // trailing upper triangle, rows/cols j+1 .. n-1
    for (int idx = tid; idx < m * m; idx += blockDim.x) {
      const int r = j + 1 + idx % m, c = j + 1 + idx / m;
      if (r <= c) A[r * kLeafLd + c] = csub(A[r * kLeafLd + c], cmul(cconj(A[j * kLeafLd + r]), A[j * kLeafLd + c]));
    }
    __syncthreads();
  }
  // T(k, c), k <= c: Td[c] on the diagonal, A[c][k] above it
  auto tget = [&](int k, int c) -> c32 {
    if (k > c) return cmk(0.0f, 0.0f);
    return k == c ? Td[c] : A[c * kLeafLd + k];
  };
  const int nbk = (n + 31) / 32;
  // diagonal blocks: warp w, lane = column within the block
  if (warp < nbk) {
    const int o = warp * 32, sw = min(32, n - o);
    if (lane < sw) {
      const int c = o + lane;
      Td[c] = cmk(1.0f / A[c * kLeafLd + c].re, 0.0f);
      for (int i = c - 1; i >= o; --i) {
        c32 acc = cmul(A[i * kLeafLd + c], Td[c]);
        for (int k = i + 1; k < c; ++k) acc = cadd(acc, cmul(A[i * kLeafLd + k], A[c * kLeafLd + k]));
        A[c * kLeafLd + i] = cscale(acc, -1.0f / A[i * kLeafLd + i].re);
      }
    }
  }
  __syncthreads();
  // off-diagonal blocks
  const int a = tid >> 5, q = tid & 31;         // element (a, q) of a 32 x 32 block
  for (int J = 1; J < nbk; ++J) {
    const int oj = J * 32, swj = min(32, n - oj);
    for (int I = J - 1; I >= 0; --I) {
      const int oi = I * 32;
      // Z = sum_{K = I+1 .. J} R_IK T_KJ
      c32 z = cmk(0.0f, 0.0f);
      if (q < swj) {
        for (int k = oi + 32; k <= oj + q; ++k) z = cadd(z, cmul(A[(oi + a) * kLeafLd + k], tget(k, oj + q)));
      }
      Z[a * 33 + q] = z;
      __syncthreads();
      // T_IJ = -T_II Z (T_II upper: rows a .. 31)
      c32 t = cmk(0.0f, 0.0f);
      if (q < swj)
        for (int p = a; p < 32; ++p) t = cadd(t, cmul(tget(oi + a, oi + p), Z[p * 33 + q]));
      __syncthreads();
      if (q < swj) A[(oj + q) * kLeafLd + (oi + a)] = cmk(-t.re, -t.im);
      __syncthreads();
    }
  }
  for (int idx = tid; idx < n * n; idx += blockDim.x) {
    const int r = idx % n, c = idx / n;
    const int64_t o = r + (int64_t)c * ld;
    if (r < c) {
      R[o] = A[r * kLeafLd + c];
      T[o] = A[c * kLeafLd + r];
    } else if (r == c) {
      R[o] = A[r * kLeafLd + r];
      T[o] = Td[r];
    } else {
      R[o] = cmk(0.0f, 0.0f);
      T[o] = cmk(0.0f, 0.0f);
    }
  }
}

cudaError_t chol_inv_leaf(cudaStream_t st, const c32* G, c32* R, c32* T, int n, int64_t ld, int64_t sNN, int B,
                          int* status) {
  if (n < 1 || n > kLeafMax) return cudaErrorInvalidValue;
  static cudaError_t attr = cudaErrorNotReady;
  if (attr == cudaErrorNotReady)
    attr = cudaFuncSetAttribute(chol_inv_leaf_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kLeafSmem);
  if (attr != cudaSuccess) return attr;
  chol_inv_leaf_kernel<<<B, 1024, kLeafSmem, st>>>(G, R, T, n, ld, sNN, status);
  return cudaGetLastError();
}

}  // namespace fm
