// Blocked Cholesky G = R^dag R (upper R) and triangular inverse T = R^-1,
// batched over trajectories.  Diagonal 32 x 32 blocks are factored and
// inverted by one CTA each; panels and trailing updates are complex GEMMs.
#include <mutex>
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
// complex64, one CTA of 1024 threads per trajectory.  Thread (warp w, lane l)
// keeps the elements (w + 32q, l + 32p), q, p = 0..3, of the upper triangle in
// registers.
//   Cholesky, right-looking with the rows left unscaled: step j reads the final
//   row j and its pivot d_j from shared memory and updates every element r, c
//   with j < r <= c by a_rc -= conj(a_jr) a_jc / d_j; the owners of row j + 1
//   then store it (now final), one barrier per step.  Afterwards
//   R_jc = a_jc / sqrt(d_j).
//   Inverse, by rows from the bottom: W = 1; row j of T is W_j / R_jj once every
//   row below it has been subtracted, W_i -= R_ij T_j (i < j).  T is kept
//   transposed in the strict lower triangle of the same array, its diagonal
//   apart; again one barrier per step.
// R and T are written with zeros below the diagonal.  A non-positive pivot
// raises FM_DEVERR_PIVOT and continues with pivot 1.
namespace fm {

constexpr int kLeafMax = 128;
constexpr int kLeafLd = kLeafMax + 1;
constexpr size_t kLeafSmem = ((size_t)kLeafMax * kLeafLd + 2 * kLeafMax) * sizeof(c32);

__global__ void __launch_bounds__(1024) chol_inv_leaf_kernel(const c32* __restrict__ G, c32* R, c32* T, int n,
                                                             int64_t ld, int64_t sNN, int* status) {
  extern __shared__ c32 sm[];
  c32* A = sm;                                  // A[r * kLeafLd + c]
  c32* Td = sm + kLeafMax * kLeafLd;            // diagonal of T
  float* Rd = (float*)(Td + kLeafMax);          // sqrt of the pivots
  const int64_t b = blockIdx.x;
  G += b * sNN;
  R += b * sNN;
  T += b * sNN;
  const int tid = threadIdx.x, l = tid & 31, w = tid >> 5;
  for (int idx = tid; idx < n * n; idx += blockDim.x) {
    const int r = idx % n, c = idx / n;
    if (r <= c) A[r * kLeafLd + c] = G[r + (int64_t)c * ld];
  }
  __syncthreads();
  c32 a[4][4];
#pragma unroll
  for (int q = 0; q < 4; ++q)
#pragma unroll
    for (int p = 0; p < 4; ++p) {
      const int r = w + 32 * q, c = l + 32 * p;
      a[q][p] = (r <= c && c < n) ? A[r * kLeafLd + c] : cmk(0.0f, 0.0f);
    }
  // ---- Cholesky (unscaled rows)
  for (int j = 0; j + 1 < n; ++j) {
    float d = A[j * kLeafLd + j].re;
    if (!(d > 0.0f) || !isfinite(d)) {
      if (tid == 0) atomicOr(status, FM_DEVERR_PIVOT);
      d = 1.0f;
    }
    const float inv = 1.0f / d;
    c32 pc[4];
#pragma unroll
    for (int p = 0; p < 4; ++p) {
      const int c = l + 32 * p;
      pc[p] = (c > j && c < n) ? cscale(A[j * kLeafLd + c], inv) : cmk(0.0f, 0.0f);
    }
    // rows r = w + 32 q and column groups p are warp-uniform: skip the finished ones
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int r = w + 32 * q;
      if (r > j && r < n) {
        const c32 prc = cconj(A[j * kLeafLd + r]);
#pragma unroll
        for (int p = 0; p < 4; ++p) {
          if (32 * p + 31 >= r) {
            const int c = l + 32 * p;
            if (c >= r && c < n) a[q][p] = csub(a[q][p], cmul(prc, pc[p]));
          }
        }
      }
    }
    // row j + 1 is final: its owners store it
    const int nr = j + 1;
    if (w == (nr & 31)) {
      const int q = nr >> 5;
#pragma unroll
      for (int qq = 0; qq < 4; ++qq)
        if (qq == q)
#pragma unroll
          for (int p = 0; p < 4; ++p) {
            const int c = l + 32 * p;
            if (c >= nr && c < n) A[nr * kLeafLd + c] = a[qq][p];
          }
    }
    __syncthreads();
  }
  // ---- R = rows scaled by 1 / sqrt(pivot)
  for (int j = tid; j < n; j += blockDim.x) {
    float d = A[j * kLeafLd + j].re;
    if (!(d > 0.0f) || !isfinite(d)) {
      atomicOr(status, FM_DEVERR_PIVOT);
      d = 1.0f;
    }
    Rd[j] = sqrtf(d);
  }
  __syncthreads();
  for (int idx = tid; idx < n * n; idx += blockDim.x) {
    const int c = idx % n, r = idx / n;
    if (r < c) A[r * kLeafLd + c] = cscale(A[r * kLeafLd + c], 1.0f / Rd[r]);
    else if (r == c) A[r * kLeafLd + r] = cmk(Rd[r], 0.0f);
  }
  __syncthreads();
  // ---- T = R^-1 by rows from the bottom; W in registers
#pragma unroll
  for (int q = 0; q < 4; ++q)
#pragma unroll
    for (int p = 0; p < 4; ++p) a[q][p] = cmk((w + 32 * q == l + 32 * p) ? 1.0f : 0.0f, 0.0f);
  if (tid == 0) Td[n - 1] = cmk(1.0f / Rd[n - 1], 0.0f);
  __syncthreads();
  for (int j = n - 1; j >= 1; --j) {
    // T_jc for the owned columns c >= j, R_rj for the owned rows r < j (warp-uniform rows)
    c32 t[4];
#pragma unroll
    for (int p = 0; p < 4; ++p) {
      const int c = l + 32 * p;
      t[p] = (c > j && c < n) ? A[c * kLeafLd + j] : (c == j ? Td[j] : cmk(0.0f, 0.0f));
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int r = w + 32 * q;
      if (r < j) {
        const c32 rr = A[r * kLeafLd + j];
#pragma unroll
        for (int p = 0; p < 4; ++p) {
          if (32 * p + 31 >= j) {
            const int c = l + 32 * p;
            if (c >= j && c < n) a[q][p] = csub(a[q][p], cmul(rr, t[p]));
          }
        }
      }
    }
    // row j - 1 of W is final: T_{j-1, c} = W_{j-1, c} / R_{j-1, j-1}
    const int nr = j - 1;
    if (w == (nr & 31)) {
      const int q = nr >> 5;
      const float s = 1.0f / Rd[nr];
#pragma unroll
      for (int qq = 0; qq < 4; ++qq)
        if (qq == q)
#pragma unroll
          for (int p = 0; p < 4; ++p) {
            const int c = l + 32 * p;
            if (c == nr) Td[nr] = cscale(a[qq][p], s);
            else if (c > nr && c < n) A[c * kLeafLd + nr] = cscale(a[qq][p], s);
          }
    }
    __syncthreads();
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
  static std::once_flag once;
  static cudaError_t attr = cudaSuccess;
  std::call_once(once, [] {
    attr = cudaFuncSetAttribute(chol_inv_leaf_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kLeafSmem);
  });
  if (attr != cudaSuccess) return attr;
  chol_inv_leaf_kernel<<<B, 1024, kLeafSmem, st>>>(G, R, T, n, ld, sNN, status);
  return cudaGetLastError();
}

}  // namespace fm
