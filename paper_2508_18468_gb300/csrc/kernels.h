// Host-side launchers of the fm kernels (internal to the library).
#pragma once

#include <cuda_runtime.h>
#include <cuda_fp16.h>
#include <stdint.h>

#include "common.cuh"

namespace fm {

// op codes for the CUDA-core complex GEMM
enum { OP_N = 0, OP_T = 1, OP_C = 2 };
// flags
enum { GEMM_UPPER_ONLY = 1, GEMM_TRI_A_UPPER = 2, GEMM_TRI_B_UPPER = 4, GEMM_LOWER_ONLY = 8 };

// C[b] = alpha op(A[b]) op(B[b]) + beta C[b], column-major complex, T = double or float.
// beta == 0 does not read C.
template <typename T>
cudaError_t zgemm(cudaStream_t st, int M, int N, int K, int opA, int opB, cplx<T> alpha,
                  const cplx<T>* A, int64_t lda, int64_t sA, const cplx<T>* B, int64_t ldb, int64_t sB,
                  cplx<T> beta, cplx<T>* C, int64_t ldc, int64_t sC, int batch, int flags);

// ---- bandwidth kernels, FP64 layout (U: L x N complex128 per trajectory, contiguous)
// partial[b][chunk][i] = sum_{k in chunk} |U_b(i,k)|^2 ; nchunks chunks of columns.
// column chunks for the occupation partial sums (fills the GPU, <= 64)
int occupation_chunks(int L, int N, int batch);
cudaError_t rownorm_partials_z(cudaStream_t st, const z64* U, int L, int N, int batch,
                               double* partial, int nchunks);
// mixed layout (V: 2L x N float per trajectory; rows i, L+i = Re, Im of site i)
cudaError_t rownorm_partials_v(cudaStream_t st, const float* V, int L, int N, int batch,
                               double* partial, int nchunks);
// n[b][i] = sum_chunk partial; if weights != null also the homodyne weight
// w[b][i] = exp(sqrt(gamma_b dt) xi + (2 n - 1) gamma_b dt).
cudaError_t reduce_occupations(cudaStream_t st, const double* partial, int nchunks, int L, int batch,
                               double* n, double* w, const double* gamma, double dt,
                               const uint64_t* traj, const int64_t* step, uint64_t seed);
// U_b(i,k) *= w_b(i)
cudaError_t scale_rows_z(cudaStream_t st, z64* U, int L, int N, int batch, const double* w);
// V_b rows i and L+i *= w_b(i); also writes the split-fp16 planes of V.
cudaError_t scale_rows_v(cudaStream_t st, float* V, __half* Vh, __half* Vl, int L, int N, int batch,
                         const double* w);
// split-fp16 planes of a float array: h = fp16(x), l = fp16((x - h) * 2^11)
cudaError_t split_planes(cudaStream_t st, const float* x, __half* h, __half* l, int64_t n);

// projective measurements of one step, one CTA per trajectory (layout: 0 = complex128 U, 1 = float V)
struct pm_args {
  void* U; int L; int N; int batch; int layout;
  const double* gamma; double dt; const uint64_t* traj; const int64_t* step; uint64_t seed;
  void* xbuf; void* vbuf;            // scratch: batch*N and batch*L complex (T of the layout)
  fm_event* log; int64_t* log_count; int log_capacity;
  int* dev_status;
};
cudaError_t pm_measure(cudaStream_t st, const pm_args& a);
// the same measurements as grid-wide kernels per event, all trajectories at once
// (reads the per-trajectory event counts back to the host: synchronises the stream)
cudaError_t pm_measure_wide(cudaStream_t st, const pm_args& a, void* scratch, int64_t* launches);
size_t pm_wide_scratch_bytes(int L, int B);
// which of the two projective paths suits this shape
bool pm_use_wide(int L, int N, int B);

// ---- Cholesky / triangular inverse (T = double or float)
constexpr int CHOL_NB = 32;
// T_b = R_b^-1 with G_b = R_b^dag R_b for the n x n blocks at G, R, Tm (leading
// dimension ld, batch stride sNN; upper part of G read, G overwritten).
// Scratch per trajectory: Dinv ceil(alloc_n/32) 32 x 32 blocks, X alloc_n x 32.
template <typename T>
cudaError_t cholesky_inverse(cudaStream_t st, cplx<T>* G, cplx<T>* R, cplx<T>* Tm, cplx<T>* Dinv, cplx<T>* X, int n,
                             int ld, int64_t sNN, int alloc_n, int B, int* status, int64_t* launches);
// factor the nb x nb diagonal block at (k,k) of every G_b into R_b (upper) and
// write its inverse into Dinv_b (nb x nb at block index k/nb); nbk = min(nb, n - k)
// rows are real, the rest padded with identity.
template <typename T>
cudaError_t chol_diag_block(cudaStream_t st, const cplx<T>* G, int64_t ldg, int64_t sG, cplx<T>* R, int64_t ldr,
                            int64_t sR, cplx<T>* Dinv, int64_t sD, int k, int nb, int nbk, int batch, int* status);
// Tm_b = block-diagonal of Dinv_b, zero elsewhere (N x N)
template <typename T>
cudaError_t place_diag_blocks(cudaStream_t st, const cplx<T>* Dinv, int64_t sD, cplx<T>* Tm, int64_t ldt, int64_t sT,
                              int N, int nb, int batch);
cudaError_t zero_lower(cudaStream_t st, z64* R, int64_t ldr, int64_t sR, int N, int batch);

// ---- misc
cudaError_t gather_rows_z(cudaStream_t st, const z64* U, int L, int N, const int* rows, int nrows, z64* out);
cudaError_t gather_rows_v(cudaStream_t st, const float* V, int L, int N, const int* rows, int nrows, z64* out);
cudaError_t v_to_z(cudaStream_t st, const float* V, int L, int N, z64* U);
cudaError_t z_to_v(cudaStream_t st, const z64* U, int L, int N, float* V, __half* Vh, __half* Vl);
// U_b = 0 except U_b(occ[k], k) = 1 (occ: device array of N occupied sites)
cudaError_t neel_init_z(cudaStream_t st, z64* U, int L, int N, int batch, const int* occ);
cudaError_t neel_init_v(cudaStream_t st, float* V, __half* Vh, __half* Vl, int L, int N, int batch,
                        const int* occ);
cudaError_t expand_propagator_z(cudaStream_t st, const z64* px, const z64* py, int Lx, int Ly, z64* P);
cudaError_t expand_propagator_planes(cudaStream_t st, const z64* px, const z64* py, int Lx, int Ly,
                                     __half* Ah, __half* Al);
cudaError_t bump_steps(cudaStream_t st, int64_t* step, int batch);
// max |G(k,l) - delta(cols[k], l)| over a ncols x N block
cudaError_t max_abs_minus_identity(cudaStream_t st, const z64* G, int ncols, int N, const int* cols,
                                   double* out);
cudaError_t check_finite_z(cudaStream_t st, const z64* X, int64_t n, int* dev_status);

// ---- eigenvalues / entropy (FP64)
// in: Hermitian m x m matrix M (column-major, overwritten; for m > 256 only its
// lower triangle is read); out: S = -sum f(lambda).  pbuf: 1 + 2 * ceil(m/64) * m + m
// complex entries of scratch.
cudaError_t hermitian_entropy(cudaStream_t st, z64* M, int m, z64* vbuf, z64* wbuf, z64* pbuf,
                              double* partial, double* d, double* e, double* lam, double* S_dev,
                              int* nlaunch);
// size of pbuf (complex entries) hermitian_entropy needs for an m x m matrix
constexpr int EIG_TILE = 32;
constexpr int64_t hermitian_entropy_pbuf(int m) {
  return 1 + 2 * (int64_t)((m + EIG_TILE - 1) / EIG_TILE) * m + m + m / 256 + 2;
}
// the lower triangle alone is enough for this m
inline bool hermitian_entropy_lower_only(int m) { return m > 256; }

// ---- exact-product Gram of a float-valued block on the tensor cores (gram_exact.cu)
// X: n x N complex128 block (column-major, ld = n) whose entries are floats.
// M (m x m, m = min(n, N), column-major): lower triangle of X X^dag (n <= N)
// or of X^T conj(X) (n > N), exact for the 28-bit truncation of every row of
// [Re | Im] relative to its largest entry.  scratch: exact_gram_scratch_bytes(nmax, N)
// device bytes, n <= nmax.  Five launches on st.
size_t exact_gram_scratch_bytes(int nmax, int N);
cudaError_t exact_gram(cudaStream_t st, const z64* X, int n, int N, z64* M, void* scratch, int* status,
                       int64_t* launches);

}  // namespace fm
