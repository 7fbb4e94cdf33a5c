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
// complex64, one CTA of 256 threads per trajectory, blocked by 32:
//   for each diagonal block k: one warp factors it (lane c owns column c; step j
//   scales row j by 1 / sqrt(pivot) and every lane updates its column with it)
//   and inverts its triangle by columns; the
//   CTA then forms the panel R_k,> = T_kk^dag G_k,> and the trailing update
//   G_>,> -= R_k,>^dag R_k,> (upper triangle);
//   then each block column j of T above the diagonal:
//   T_<j,j = -(T_<j,<j R_<j,j) T_jj, the inner product kept in shared memory.
// R is kept in the upper triangle of a shared array, T transposed in its strict
// lower triangle and T's diagonal apart: 20 CTA barriers per 128 x 128 leaf
// instead of one per row.  R and T are written with zeros below the diagonal.
// A non-positive pivot raises FM_DEVERR_PIVOT and continues with pivot 1.
namespace fm {

constexpr int kLeafMax = 128;
constexpr int kLeafLd = kLeafMax + 1;
constexpr int kLeafThreads = 256;
constexpr int kLeafYLd = 33;
constexpr size_t kLeafSmem = ((size_t)kLeafMax * kLeafLd + kLeafMax + 96 * kLeafYLd) * sizeof(c32) +
                              kLeafMax * sizeof(float);

// Factor and invert the m x m (m <= 32) diagonal block at D (row stride kLeafLd),
// one warp, lane c owning column c: R into the upper triangle of D, T = R^-1
// transposed into its strict lower triangle (row c of the lower triangle holds
// column c of T), T's diagonal into Tdk, 1 / R_jj into Rinv.  Returns true after a
// bad pivot (which is then taken as 1).
//   Factor: lane c keeps the rest of its column of the Schur complement in registers,
//   rotated so that the pivot row is always col[0]; step j takes G_jj from lane j,
//   forms R_jc = G_jc / R_jj and subtracts conj(R_jr) R_jc from rows r = j + 1 .. c,
//   R_jr arriving by a shuffle from lane r.
//   Inverse: column c of T by back substitution, R t = e_c from row c up; the entries
//   t_{i+1} .. already found sit rotated in registers, row i of R comes from shared
//   memory (one address for the whole warp).
__device__ __forceinline__ bool leaf_diag_block(c32* D, c32* Tdk, float* Rinv, int m, int c) {
  bool bad = false;
  c32 col[32];
#pragma unroll
  for (int q = 0; q < 32; ++q) col[q] = (c < m && q <= c) ? D[q * kLeafLd + c] : cmk(0.0f, 0.0f);
  for (int j = 0; j < m; ++j) {
    float piv = __shfl_sync(0xffffffffu, col[0].re, j);
    if (!(piv > 0.0f) || !isfinite(piv)) {
      bad = true;
      piv = 1.0f;
    }
    const float rs = sqrtf(piv), ri = __frcp_rn(rs);
    const c32 rj = (c == j) ? cmk(rs, 0.0f) : cscale(col[0], ri);   // R_jc (lanes c >= j)
    if (c >= j && c < m) D[j * kLeafLd + c] = rj;
    if (c == 0) Rinv[j] = ri;
#pragma unroll
    for (int q = 1; q < 32; ++q) {
      const int lr = (j + q) & 31;
      const c32 x = cmk(__shfl_sync(0xffffffffu, rj.re, lr), __shfl_sync(0xffffffffu, rj.im, lr));   // R_{j, j+q}
      if (j + q <= c) col[q] = csub(col[q], cmul(cconj(x), rj));
    }
#pragma unroll
    for (int q = 0; q < 31; ++q) col[q] = col[q + 1];
    col[31] = cmk(0.0f, 0.0f);
  }
  __syncwarp();                                   // rows of R visible to the whole warp
  // s[q] = t_{i+1+q}, column c of T (zero beyond row c)
  c32 sv[32];
#pragma unroll
  for (int q = 0; q < 32; ++q) sv[q] = cmk(0.0f, 0.0f);
  for (int i = m - 1; i >= 0; --i) {
    // four partial sums (k = i + 1 + q, q mod 4), so that the multiply-adds do not wait on
    // one another, then added in a fixed order
    c32 acc[4];
#pragma unroll
    for (int a = 0; a < 4; ++a) acc[a] = cmk(0.0f, 0.0f);
    const c32* Ri = D + i * kLeafLd;
#pragma unroll
    for (int q = 0; q < 31; ++q) {
      const int k = i + 1 + q;
      if (k <= c && k < m) cfma(acc[q & 3], Ri[k], sv[q]);
    }
    const c32 sum = cadd(cadd(acc[0], acc[1]), cadd(acc[2], acc[3]));
    const c32 ti = cscale(cmk((c == i ? 1.0f : 0.0f) - sum.re, -sum.im), Rinv[i]);
    if (c < m) {
      if (i < c) D[c * kLeafLd + i] = ti;
      else if (i == c) Tdk[c] = ti;
    }
#pragma unroll
    for (int q = 31; q > 0; --q) sv[q] = sv[q - 1];
    sv[0] = ti;
  }
  __syncwarp();
  return bad;
}

__global__ void __launch_bounds__(kLeafThreads, 1) chol_inv_leaf_kernel(const c32* __restrict__ G, c32* R, c32* T,
                                                                        int n, int64_t ld, int64_t sNN, int* status) {
  extern __shared__ c32 sm[];
  c32* A = sm;                                  // A[r * kLeafLd + c]
  c32* Td = sm + kLeafMax * kLeafLd;            // diagonal of T
  c32* Y = Td + kLeafMax;                       // panel staging (32 x 96), products of the inverse (96 x 32)
  float* Rinv = (float*)(Y + 96 * kLeafYLd);    // 1 / R_jj
  const int64_t b = blockIdx.x;
  G += b * sNN;
  R += b * sNN;
  T += b * sNN;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  for (int base = tid; base < n * n; base += 8 * kLeafThreads) {   // 8 loads in flight per thread
    c32 v[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int idx = base + u * kLeafThreads, r = idx % n, c = idx / n;
      v[u] = (idx < n * n && r <= c) ? G[r + (int64_t)c * ld] : cmk(0.0f, 0.0f);
    }
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int idx = base + u * kLeafThreads, r = idx % n, c = idx / n;
      if (idx < n * n && r <= c) A[r * kLeafLd + c] = v[u];
    }
  }
  __syncthreads();
  const int nb = (n + 31) / 32;
  bool bad = false;
  for (int kb = 0; kb < nb; ++kb) {
    const int o = 32 * kb, m = min(32, n - o), rest = n - o - m;   // rest > 0 implies m == 32
    if (warp == 0) bad |= leaf_diag_block(A + o * kLeafLd + o, Td + o, Rinv + o, m, lane);
    __syncthreads();
    if (rest == 0) break;
    // panel R_{o+r, c} = sum_{i <= r} conj(T_{o+i, o+r}) G_{o+i, c}: items (8 rows, column),
    // staged in Y (32 x 96) until every item has read G
    const int items = 4 * rest;
    for (int e = tid; e < items; e += kLeafThreads) {
      const int cidx = e % rest, r0 = 8 * (e / rest), cp = o + 32 + cidx;
      c32 acc[8];
#pragma unroll
      for (int rr = 0; rr < 8; ++rr) acc[rr] = cmk(0.0f, 0.0f);
      for (int i = 0; i < r0; ++i) {            // rows r0 .. r0 + 7 all below i
        const c32 a = A[(o + i) * kLeafLd + cp];
#pragma unroll
        for (int rr = 0; rr < 8; ++rr) cfma(acc[rr], cconj(A[(o + r0 + rr) * kLeafLd + o + i]), a);
      }
      for (int i = r0; i < r0 + 8; ++i) {       // the 8 x 8 triangle
        const c32 a = A[(o + i) * kLeafLd + cp];
#pragma unroll
        for (int rr = 0; rr < 8; ++rr) {
          const int r = r0 + rr;
          if (r > i) cfma(acc[rr], cconj(A[(o + r) * kLeafLd + o + i]), a);
          else if (r == i) cfma(acc[rr], cconj(Td[o + i]), a);
        }
      }
#pragma unroll
      for (int rr = 0; rr < 8; ++rr) Y[(r0 + rr) * 96 + cidx] = acc[rr];
    }
    __syncthreads();
    for (int e = tid; e < 32 * rest; e += kLeafThreads) {
      const int r = e / rest, cidx = e % rest;
      A[(o + r) * kLeafLd + o + 32 + cidx] = Y[r * 96 + cidx];
    }
    __syncthreads();
    // trailing update of the upper triangle: items (8 rows, column), rows <= column
    int tot = 0;
    for (int q = 0; 8 * q < rest; ++q) tot += rest - 8 * q;
    for (int e = tid; e < tot; e += kLeafThreads) {
      int q = 0, base = 0;
      while (e >= base + rest - 8 * q) {
        base += rest - 8 * q;
        ++q;
      }
      const int ci = 8 * q + (e - base), c = o + 32 + ci, rb = o + 32 + 8 * q;
      c32 s8[8];
#pragma unroll
      for (int rr = 0; rr < 8; ++rr) s8[rr] = cmk(0.0f, 0.0f);
#pragma unroll 2
      for (int i = 0; i < 32; ++i) {
        const c32 a = A[(o + i) * kLeafLd + c];
#pragma unroll
        for (int rr = 0; rr < 8; ++rr) cfma(s8[rr], cconj(A[(o + i) * kLeafLd + rb + rr]), a);
      }
#pragma unroll
      for (int rr = 0; rr < 8; ++rr)
        if (8 * q + rr <= ci) A[(rb + rr) * kLeafLd + c] = csub(A[(rb + rr) * kLeafLd + c], s8[rr]);
    }
    __syncthreads();
  }
  // T above the diagonal blocks, block column j: Y = T_<j,<j R_<j,j, then T_<j,j = -Y T_jj
  for (int j = 1; j < nb; ++j) {
    const int c0 = 32 * j, mj = min(32, n - c0), items = 4 * j * mj;
    for (int e = tid; e < items; e += kLeafThreads) {
      const int rq = e / mj, cc = e % mj, c = c0 + cc, rb = 8 * rq;
      c32 acc[8];
#pragma unroll
      for (int rr = 0; rr < 8; ++rr) acc[rr] = cmk(0.0f, 0.0f);
      for (int s = rb; s < rb + 8; ++s) {       // the 8 x 8 triangle of T_rs, s >= r
        const c32 rsc = A[s * kLeafLd + c];
#pragma unroll
        for (int rr = 0; rr < 8; ++rr) {
          const int r = rb + rr;
          if (s > r) cfma(acc[rr], A[s * kLeafLd + r], rsc);
          else if (s == r) cfma(acc[rr], Td[r], rsc);
        }
      }
      for (int s = rb + 8; s < c0; ++s) {
        const c32 rsc = A[s * kLeafLd + c];
#pragma unroll
        for (int rr = 0; rr < 8; ++rr) cfma(acc[rr], A[s * kLeafLd + rb + rr], rsc);
      }
#pragma unroll
      for (int rr = 0; rr < 8; ++rr) Y[(rb + rr) * kLeafYLd + cc] = acc[rr];
    }
    __syncthreads();
    for (int e = tid; e < items; e += kLeafThreads) {
      const int rq = e / mj, cc = e % mj, c = c0 + cc, rb = 8 * rq;
      c32 acc[8];
      const c32 tcc = Td[c];
#pragma unroll
      for (int rr = 0; rr < 8; ++rr) acc[rr] = cmul(Y[(rb + rr) * kLeafYLd + cc], tcc);
      for (int s = c0; s < c; ++s) {
        const c32 tsc = A[c * kLeafLd + s];
#pragma unroll
        for (int rr = 0; rr < 8; ++rr) cfma(acc[rr], Y[(rb + rr) * kLeafYLd + s - c0], tsc);
      }
#pragma unroll
      for (int rr = 0; rr < 8; ++rr) A[c * kLeafLd + rb + rr] = cmk(-acc[rr].re, -acc[rr].im);
    }
    __syncthreads();
  }
  if (bad && lane == 0) atomicOr(status, FM_DEVERR_PIVOT);
  for (int idx = tid; idx < n * n; idx += kLeafThreads) {
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
  chol_inv_leaf_kernel<<<B, kLeafThreads, kLeafSmem, st>>>(G, R, T, n, ld, sNN, status);
  return cudaGetLastError();
}

}  // namespace fm

extern "C" int fmx_chol_leaf(const void* G, int n, int ld, int B, void* R, void* T, int* d_status, void* stream) {
  if (n < 1 || n > fm::kLeafMax || ld < n || B < 1 || !d_status) return (int)cudaErrorInvalidValue;
  return (int)fm::chol_inv_leaf((cudaStream_t)stream, (const c32*)G, (c32*)R, (c32*)T, n, ld,
                                (int64_t)ld * n, B, d_status);
}
