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
  const int4* force; int force_n;    // forced outcomes (fm_force_outcomes), sorted; n = 0: none
};
cudaError_t pm_measure(cudaStream_t st, const pm_args& a);
// the same measurements as grid-wide kernels per event, all trajectories at once
// (reads the per-trajectory event counts back to the host: synchronises the stream)
cudaError_t pm_measure_wide(cudaStream_t st, const pm_args& a, void* scratch, int64_t* launches);
size_t pm_wide_scratch_bytes(int L, int B);
// which of the two projective paths suits this shape
bool pm_use_wide(int L, int N, int B);

// ---- projective measurements of a step as a block (pm_block.cu; mixed precision)
struct PmbEvent {
  double sp, c, dsel;
  int outcome, active;
};
// K x K complex64 coefficient matrices of every trajectory (stride sM = Kc * Kc
// per trajectory; row-major TBr, CTB, TA, CTA, TE, column-major C, TBc), the
// per-event vectors (stride Kc), and the K x N blocks W (rows of U0 at the
// selected sites) and X = T_B^dag W (column-major, ld Kc, stride sW).
struct PmbMats {
  int Kc;
  int64_t sM, sW;
  c32 *C, *TBr, *TBc, *CTB, *TA, *CTA, *TE;
  c32 *rho, *y, *ys, *g;
  PmbEvent* ev;
  c32 *Wc, *X;
};
int pmb_capacity(int L);   // largest block (selected sites per step) the scratch holds
cudaError_t pmb_setup(cudaStream_t st, const int* list, const int* count, int L, int B, int nmax, int* pos);
cudaError_t pmb_gather_w(cudaStream_t st, const __half* urm_h, const __half* urm_l, int L, int N, const int* list,
                         const int* count, int B, int K, __half* wt_h, __half* wt_l);
cudaError_t pmb_gather_c(cudaStream_t st, const float* Dp, int64_t sD, int L, int K, int B, const int* list,
                         const int* count, const PmbMats& m);
// one event i of the step, all trajectories (four launches, each spread over the GPU)
cudaError_t pmb_event(cudaStream_t st, int i, int Kc, int L, int B, const int* count, const int* list,
                      const double* ulist, const int64_t* step, const PmbMats& m, fm_event* log,
                      unsigned long long* log_count, int log_capacity, int nmax);
// whether pmb_events suits B trajectories with at most kmax events each
bool pmb_events_fit(int B, int kmax);
// every event of the step in one launch (one CTA per trajectory, the events in order)
cudaError_t pmb_events(cudaStream_t st, int Kc, int L, int B, const int* count, const int* list, const double* ulist,
                       const int64_t* step, const PmbMats& m, fm_event* log, unsigned long long* log_count,
                       int log_capacity);
cudaError_t pmb_ttilde(cudaStream_t st, const PmbMats& m, int K, int B, __half* th, __half* tl);
cudaError_t pmb_split(cudaStream_t st, const float* x, int64_t n, __half* h, __half* l);
cudaError_t pmb_atilde(cudaStream_t st, const float* Ap, int L, int K, int B, const int* pos, const PmbMats& m,
                       __half* ah, __half* al);
cudaError_t pmb_gather_wc(cudaStream_t st, const float* V, int L, int N, int K, int B, const int* list,
                          const int* count, const PmbMats& m);
cudaError_t pmb_xtilde(cudaStream_t st, const PmbMats& m, int K, int B, int N, __half* xh, __half* xl);
// the selection step of the grid-wide path: per trajectory the measured sites
// (ascending) and their outcome draws; count per trajectory
cudaError_t pm_select(cudaStream_t st, const pm_args& a, int* list, double* ulist, int* count);

// ---- Cholesky / triangular inverse (T = double or float)
constexpr int CHOL_NB = 32;
// T_b = R_b^-1 with G_b = R_b^dag R_b for the n x n blocks at G, R, Tm (leading
// dimension ld, batch stride sNN; upper part of G read, G overwritten).
// Scratch per trajectory: Dinv ceil(alloc_n/32) 32 x 32 blocks, X alloc_n x 32.
// G = R^dag R and T = R^-1 of an n x n complex64 block (n <= 128) per trajectory
// in one CTA each (shared memory); R, T written with zeros below the diagonal.
cudaError_t chol_inv_leaf(cudaStream_t st, const c32* G, c32* R, c32* T, int n, int64_t ld, int64_t sNN, int B,
                          int* status);
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
// lower triangle is read); out: S = -sum f(lambda).  pbuf: hermitian_entropy_pbuf(m)
// complex entries of scratch.
// cross != 0: M's eigenvalues are sigma^2 = lambda (1 - lambda) (the cross-block form
// of the entropy sketch); each gives the term of its root lambda <= 1/2.
// lam: the eigenvalues, ascending.
cudaError_t hermitian_entropy(cudaStream_t st, z64* M, int m, z64* vbuf, z64* wbuf, z64* pbuf,
                              double* partial, double* d, double* e, double* lam, double* S_dev,
                              int* nlaunch, int cross = 0);
// size of pbuf (complex entries) hermitian_entropy needs for an m x m matrix
constexpr int EIG_TILE = 32;
constexpr int64_t hermitian_entropy_pbuf(int m) {
  return 1 + 2 * (int64_t)((m + EIG_TILE - 1) / EIG_TILE) * m + m + m / 256 + 2 + 2 * (int64_t)m;
}
// the lower triangle alone is enough for this m
inline bool hermitian_entropy_lower_only(int m) { return m > 256; }

// ---- structured propagation: stencils of the circulant propagator (banded.cu)
constexpr int kBandMaxTaps = 41;   // half-width <= 20
// column chunks (blockIdx.y) of a stencil pass along dir, and of a thread-per-site pass
int band_chunks(int Lx, int Ly, int N, int B, int dir, int layout);
int site_chunks(int L, int N, int B);
// layout 0: complex128 U (L x N per trajectory); 1: float V (2L x N).  dir 0 along x,
// 1 along y.  partial (may be NULL): row sums of |out|^2 per column chunk, nch chunks.
// off: consecutive offsets; tap_stride > 0: trajectory b uses taps + b tap_stride.
cudaError_t band_propagate(cudaStream_t st, int layout, const void* in, void* out, int L, int N, int B, int Lx,
                           int Ly, int dir, const z64* taps, const int* off, int ntap, double* partial, int nch,
                           int tap_stride = 0);
// the projective event e of the grid-wide path (row and outcome, v = U x^dag / sqrt(p),
// rank-1 update) for every trajectory with e < count[b]; list / ulist hold the sites and
// Born draws of trajectory b at b ld_list + e.  scratch: pm_wide_scratch_bytes(L, B).
cudaError_t pm_wide_event(cudaStream_t st, const pm_args& a, int e, const int* list, const double* ulist,
                          int ld_list, const int* count, void* scratch);

// one Horner stage out = U0 + c (A dt) Y of the Runge-Kutta step of Eq. (QSD_evo):
// A dt = -i dt J (nearest-neighbour sum) + diag(ln w); layout as band_propagate
cudaError_t rk4_stage(cudaStream_t st, int layout, const void* U0, const void* Y, void* out, int L, int N, int B,
                      int Lx, int Ly, const double* w, double dtJ, double c);

// ---- density correlations and particle covariance (observables.cu)
cudaError_t v_to_c32(cudaStream_t st, const float* V, int L, int N, c32* U);
cudaError_t gather_rows_c32(cudaStream_t st, const float* V, int L, int N, const int* sites, int n, c32* out);
// bins[d] += sum over the stripe columns j0 .. j0+S-1 of |X(j - d, j - j0)|^2 (periodic in x, y; d != 0)
template <typename T>
cudaError_t displacement_bins(cudaStream_t st, const cplx<T>* X, int L, int Lx, int Ly, int j0, int S, double* bins);
int abs2_partials();   // doubles of `part` sum_abs2 uses
template <typename T>
cudaError_t sum_abs2(cudaStream_t st, const cplx<T>* M, int64_t n, double* part, double* out);

// ---- exact-product Gram of a float-valued block on the tensor cores (gram_exact.cu)
// X: n x N complex128 block (column-major, ld = n) whose entries are floats.
// M (m x m, m = min(n, N), column-major): lower triangle of X X^dag (n <= N)
// or of X^T conj(X) (n > N), exact for the 28-bit truncation of every row of
// [Re | Im] relative to its largest entry.  scratch: exact_gram_scratch_bytes(nmax, N)
// device bytes, n <= nmax.  Five launches on st.
size_t exact_gram_scratch_bytes(int nmax, int N);
cudaError_t exact_gram(cudaStream_t st, const z64* X, int n, int N, z64* M, void* scratch, int* status,
                       int64_t* launches);
// the same for a complex64 block with leading dimension ld >= n
cudaError_t exact_gram_c32(cudaStream_t st, const c32* X, int64_t ld, int n, int N, z64* M, void* scratch,
                           int* status, int64_t* launches);
// First-order correction of M (the lower triangle exact_gram wrote for the block XA
// of n gathered rows) from C = U U^dag to the projector onto span(U): Gx is the
// exact_gram of all L rows of U (= conj(U^dag U), lower triangle, N x N).
// scratch: projector_scratch_bytes(N).
size_t projector_scratch_bytes(int N);
cudaError_t projector_correct(cudaStream_t st, const z64* Gx, const z64* XA, int n, int N, z64* M, void* scratch,
                              int64_t* launches);

// ---- entanglement entropy from a sketch of the cross block C_AB = U_A U_B^dag (ee_sketch.cu)
constexpr int kSketchPartials = 17;   // partial-Gram capacity, in rmax x rmax matrices
struct SketchScratch {
  int nmax, N, rmax;
  c32 *Om, *Yc, *Z;           // nmax x rmax, nmax x rmax, N x rmax
  z64 *Yz, *Yz2;              // nmax x rmax (float64 orthonormalisation)
  z64 *G, *R, *T, *Dinv, *Xc; // rmax x rmax Cholesky factors and their scratch
  z64* H;                     // rmax x rmax Rayleigh-Ritz matrix
  z64* Gp;                    // kSketchPartials x rmax x rmax partial Grams
  z64 *vb, *wb, *pb;
  double *d, *e, *lam, *S;
  int* status;
  void* xg;                   // exact-Gram scratch
  size_t bytes;
};
// carve the scratch of a sketch (subsystem and complement of at most nmax sites, rank
// at most rmax) out of `base` (NULL: sizes only)
SketchScratch sketch_layout(void* base, int nmax, int N, int rmax);
// out (n x N, ld n) = the rows of the complex64 block X (column-major, ld) as complex128
cudaError_t rows_c32_to_z64(cudaStream_t st, const c32* X, int64_t ld, int n, int N, z64* out);
size_t sketch_scratch_bytes(int nmax, int N, int rmax);
// U: L x N complex64 rows, A's nA rows first, then B's nB rows (column-major, ld);
// r: sketch rank (multiple of 32, r < nA, nB), q: power iterations.  Writes S (entropy
// of A, nats) to S_out and the (max(8, r/8))-th smallest Ritz value to chk_out (the
// sketch has converged when it is below ~1e-9); w.status gets Cholesky pivot flags.
cudaError_t sketch_entropy(cudaStream_t st, const c32* U, int64_t ld, int nA, int nB, int N, int r, int q,
                           uint64_t seed, const SketchScratch& w, double* S_out, double* chk_out, int64_t* launches);

}  // namespace fm
