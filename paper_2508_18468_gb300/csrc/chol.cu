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
//   for each diagonal block k: one warp factors and inverts it in one sweep (lane c
//   owns column c; step j scales row j by 1 / sqrt(pivot) and every lane updates its
//   column and its column of the inverse with it); the
//   CTA then forms the panel R_k,> = T_kk^dag G_k,> and the trailing update
//   G_>,> -= R_k,>^dag R_k,> (upper triangle);
//   each block column j of T above the diagonal, T_<j,j = -(T_<j,<j R_<j,j) T_jj,
//   is formed by the other seven warps while warp 0 factors the next diagonal
//   blocks: the inner product beside block j, the product with T_jj beside block
//   j + 1 (the last block column's after the loop).
// R is kept in the upper triangle of a shared array, T transposed in its strict
// lower triangle and T's diagonal apart: 14 CTA barriers per 128 x 128 leaf
// instead of one per row.  R and T are written with zeros below the diagonal.
// A non-positive pivot raises FM_DEVERR_PIVOT and continues with pivot 1.
namespace fm {

constexpr int kLeafMax = 128;
constexpr int kLeafLd = kLeafMax + 1;
constexpr int kLeafThreads = 256;
constexpr int kLeafYLd = 33;
constexpr size_t kLeafSmem = ((size_t)kLeafMax * kLeafLd + kLeafMax + 2 * 96 * kLeafYLd) * sizeof(c32);

// Steps j0 .. j1 - 1 of the diagonal-block sweep below, with b[] holding rows j .. j + QN - 1
// of lane c's column (every row still live when j >= 32 - QN).  Rolled, with constant
// indices into b[]: the quarter-sized copies keep the code small enough to stay in the
// instruction cache, and shrink the updates and the rotation as the block is consumed.
template <int QN>
__device__ __forceinline__ void leaf_diag_steps(c32 (&b)[32], c32* D, c32* Tdk, int j0, int j1, int m, int c,
                                                bool& bad) {
  const c32 zero = cmk(0.0f, 0.0f);
  for (int j = j0; j < j1; ++j) {
    float piv = __shfl_sync(0xffffffffu, b[0].re, j);
    if (!(piv > 0.0f) || !isfinite(piv)) {
      bad = true;
      piv = 1.0f;
    }
    const float rs = sqrtf(piv), ri = __frcp_rn(rs);
    const c32 s = cscale(b[0], ri);
    const c32 rj = (c > j) ? s : (c == j ? cmk(rs, 0.0f) : zero);   // R_jc
    const c32 tj = (c < j) ? s : (c == j ? cmk(ri, 0.0f) : zero);   // (R^-dag)_jc
    if (c < m) D[j * kLeafLd + c] = (c < j) ? cconj(s) : rj;
    if (c == j) Tdk[j] = cmk(ri, 0.0f);
    __syncwarp();
    const c32* Dj = D + j * kLeafLd + j;
    // every lane runs every update (masked rather than branched: branches here cost more
    // than the multiply-adds they would skip)
#pragma unroll
    for (int q = 1; q < QN; ++q) {
      const c32 x = (j + q < m) ? Dj[q] : zero;                     // R_{j, j+q}
      const c32 f = (j + q <= c) ? rj : tj;
      b[q] = csub(b[q], cmul(cconj(x), f));
    }
#pragma unroll
    for (int q = 0; q < QN - 1; ++q) b[q] = b[q + 1];
    b[QN - 1] = zero;
  }
}

// Factor and invert the m x m (m <= 32) diagonal block at D (row stride kLeafLd) in one
// sweep, one warp, lane c owning column c: R into the upper triangle of D, T = R^-1
// transposed into its strict lower triangle (row j of the lower triangle holds column j
// of T), T's diagonal into Tdk.  Returns true after a bad pivot (which is then taken as 1).
//   The row operations that take G to R (step j: row j scaled by 1 / sqrt(pivot), then
//   conj(R_jr) times it subtracted from every row r > j) take the identity to R^-dag when
//   applied to it alongside.  Lane c keeps one array b[], rotated so that b[0] is row j:
//   rows <= c hold its column of the Schur complement, rows > c its column of the
//   transformed identity (whose row c is 1 until step c and whose rows above c stay 0,
//   so neither is stored).  Step j writes row j (R_jc for c >= j, T_cj = conj of
//   (R^-dag)_jc for c < j) to shared memory, and every lane takes R_jr, r > j, from there
//   (one address for the whole warp).
__device__ __forceinline__ bool leaf_diag_block(c32* D, c32* Tdk, int m, int c) {
  bool bad = false;
  c32 b[32];
#pragma unroll
  for (int q = 0; q < 32; ++q) b[q] = (c < m && q <= c) ? D[q * kLeafLd + c] : cmk(0.0f, 0.0f);
  leaf_diag_steps<32>(b, D, Tdk, 0, min(m, 8), m, c, bad);
  leaf_diag_steps<24>(b, D, Tdk, 8, min(m, 16), m, c, bad);
  leaf_diag_steps<16>(b, D, Tdk, 16, min(m, 24), m, c, bad);
  leaf_diag_steps<8>(b, D, Tdk, 24, m, m, c, bad);
  __syncwarp();
  return bad;
}

// Block column j of T above the diagonal, in two halves run by threads t0 .. t0 + nt - 1:
//   first:  Z = T_<j,<j R_<j,j   (needs T up to block column j - 1 and the panels above j;
//                                 not T_jj, so it can run beside the factorisation of block j)
//   second: T_<j,j = -Z T_jj     (needs block j factored)
// Z (96 x 33) is the inverse's own staging; items are (8 rows, one column).
__device__ __forceinline__ void leaf_tcol_first(const c32* A, const c32* Td, c32* Z, int n, int j, int t, int nt) {
  const int c0 = 32 * j, mj = min(32, n - c0), items = 4 * j * mj;
  for (int e = t; e < items; e += nt) {
    const int rq = e / mj, cc = e % mj, c = c0 + cc, rb = 8 * rq;
    c32 acc[8];
#pragma unroll
    for (int rr = 0; rr < 8; ++rr) acc[rr] = cmk(0.0f, 0.0f);
    for (int s = rb; s < rb + 8; ++s) {         // the 8 x 8 triangle of T_rs, s >= r
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
    for (int rr = 0; rr < 8; ++rr) Z[(rb + rr) * kLeafYLd + cc] = acc[rr];
  }
}

__device__ __forceinline__ void leaf_tcol_second(c32* A, const c32* Td, const c32* Z, int n, int j, int t, int nt) {
  const int c0 = 32 * j, mj = min(32, n - c0), items = 4 * j * mj;
  for (int e = t; e < items; e += nt) {
    const int rq = e / mj, cc = e % mj, c = c0 + cc, rb = 8 * rq;
    c32 acc[8];
    const c32 tcc = Td[c];
#pragma unroll
    for (int rr = 0; rr < 8; ++rr) acc[rr] = cmul(Z[(rb + rr) * kLeafYLd + cc], tcc);
    for (int s = c0; s < c; ++s) {
      const c32 tsc = A[c * kLeafLd + s];
#pragma unroll
      for (int rr = 0; rr < 8; ++rr) cfma(acc[rr], Z[(rb + rr) * kLeafYLd + s - c0], tsc);
    }
#pragma unroll
    for (int rr = 0; rr < 8; ++rr) A[c * kLeafLd + rb + rr] = cmk(-acc[rr].re, -acc[rr].im);
  }
}

__global__ void __launch_bounds__(kLeafThreads, 1) chol_inv_leaf_kernel(const c32* __restrict__ G, c32* R, c32* T,
                                                                        int n, int64_t ld, int64_t sNN, int* status) {
  extern __shared__ c32 sm[];
  c32* A = sm;                                  // A[r * kLeafLd + c]
  c32* Td = sm + kLeafMax * kLeafLd;            // diagonal of T
  c32* Y = Td + kLeafMax;                       // panel staging (32 x 96)
  c32* Z = Y + 96 * kLeafYLd;                   // products of the inverse (96 x 32)
  const int64_t b = blockIdx.x;
  G += b * sNN;
  R += b * sNN;
  T += b * sNN;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  // the upper triangle, a warp per column and a lane per row, 16 loads in flight per thread
  // (one SM alone: the bytes in flight set the rate)
  for (int c0 = warp; c0 < n; c0 += 4 * (kLeafThreads / 32)) {
    c32 v[16];
#pragma unroll
    for (int u = 0; u < 16; ++u) {
      const int c = c0 + (u >> 2) * (kLeafThreads / 32), r = lane + 32 * (u & 3);
      v[u] = (c < n && r <= c) ? G[r + (int64_t)c * ld] : cmk(0.0f, 0.0f);
    }
#pragma unroll
    for (int u = 0; u < 16; ++u) {
      const int c = c0 + (u >> 2) * (kLeafThreads / 32), r = lane + 32 * (u & 3);
      if (c < n && r <= c) A[r * kLeafLd + c] = v[u];
    }
  }
  __syncthreads();
  const int nb = (n + 31) / 32;
  bool bad = false;
  for (int kb = 0; kb < nb; ++kb) {
    const int o = 32 * kb, m = min(32, n - o), rest = n - o - m;   // rest > 0 implies m == 32
    if (warp == 0) {
      bad |= leaf_diag_block(A + o * kLeafLd + o, Td + o, m, lane);
    } else if (kb >= 1) {
      // meanwhile, the other warps: the second half of block column kb - 1 of T, then the
      // first half of block column kb (neither touches block kb, which warp 0 is factoring)
      const int t = tid - 32, nt = kLeafThreads - 32;
      if (kb >= 2) {
        leaf_tcol_second(A, Td, Z, n, kb - 1, t, nt);
        asm volatile("bar.sync 1, %0;" ::"n"(kLeafThreads - 32) : "memory");
      }
      leaf_tcol_first(A, Td, Z, n, kb, t, nt);
    }
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
  // the second half of the last block column of T (the others ran beside the factorisation)
  if (nb >= 2) {
    leaf_tcol_second(A, Td, Z, n, nb - 1, tid, kLeafThreads);
    __syncthreads();
  }
  if (bad && lane == 0) atomicOr(status, FM_DEVERR_PIVOT);
  // R and T with their zeros, a warp per column and a lane per row
  for (int c = warp; c < n; c += kLeafThreads / 32) {
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int r = lane + 32 * u;
      if (r < n) {
        const int64_t o = r + (int64_t)c * ld;
        const c32 zero = cmk(0.0f, 0.0f);
        R[o] = (r <= c) ? A[r * kLeafLd + c] : zero;
        T[o] = (r < c) ? A[c * kLeafLd + r] : (r == c ? Td[r] : zero);
      }
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
