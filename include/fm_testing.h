/*
 * fm_testing.h -- test hooks of libfm.so that expose the tensor-core products
 * on their own (the split-fp16 GEMM and the exact-product Gram of the
 * entropy), so they can be checked against reference products.  They are not
 * part of the trajectory API (include/fm.h); the paper has no counterpart of
 * them.
 *
 * Operand planes: a float x is passed as two fp16 arrays h, l with
 * x ~= h + l * 2^-11.  All pointers are device pointers; work is issued on
 * `stream` (cudaStream_t or NULL) and not synchronised.  Return value: 0 on
 * success, otherwise a cudaError_t code (invalid sizes give
 * cudaErrorInvalidValue).  d_tiles: caller-owned device scratch of at least
 * 16 bytes per output tile.
 */
#ifndef FM_TESTING_H
#define FM_TESTING_H

#ifdef __cplusplus
extern "C" {
#endif

/* D (M x N, column-major, ld M, float) = A B^T, A: M x K and B: N x K, both
 * row-major (K contiguous) planes.  M % 128 == 0, N % BN == 0 (BN 128 or
 * 256), K % 64 == 0.  grid: CTAs (<= 0: one per tile).  chunk_kb > 0 (BN 128
 * only): move the TMEM accumulators into fp32 registers every chunk_kb
 * 64-deep K-blocks.  raster != 0: tiles in computed grouped order (d_tiles
 * unused) instead of an uploaded tile list. */
int fmx_tc_gemm(const void* Ah, const void* Al, const void* Bh, const void* Bl, int M, int N, int K,
                float* D, int BN, int grid, int chunk_kb, int raster, void* d_tiles, void* stream);

/* Complex Gram G_b = U_b^dag U_b (complex64, N x N column-major, upper 128 x BN
 * tiles written) of B trajectories whose orbitals are stored as V_b (2L x N,
 * column-major planes, column k = [Re U_{:,k}; Im U_{:,k}]). */
int fmx_tc_gram(const void* Vh, const void* Vl, int L, int N, int B, float* G, int BN, void* d_tiles,
                void* stream);

/* Device scratch bytes fmx_exact_gram needs for blocks with up to nmax rows. */
unsigned long long fmx_exact_gram_scratch_bytes(int nmax, int N);

/* M (m x m complex128, column-major, m = min(n, N); lower triangle written)
 * = X X^dag (n <= N) or X^T conj(X) (n > N) for the n x N complex128 block X
 * (column-major, ld n) whose entries are floats; exact for the 28-bit
 * truncation of every row of [Re | Im] relative to its largest entry.  The
 * same routine the mixed-precision entropy uses for m > 256. */
int fmx_exact_gram(const void* X, int n, int N, void* M, void* d_scratch, void* stream);

/* Cholesky factor and inverse of B Hermitian blocks on the CUDA cores, the leaf
 * of the mixed-precision CholeskyQR's recursive factorisation (Sec. III,
 * CholeskyQR2): G_b = R_b^dag R_b, R_b upper triangular with a real positive
 * diagonal, T_b = R_b^-1.  G, R, T: complex64 (re, im float pairs), n x n
 * column-major with leading dimension ld, block b at offset b * ld * n; only
 * the upper triangle of G is read; R and T are written in full (zeros below
 * the diagonal).  1 <= n <= 128.  A non-positive or non-finite pivot ORs 1
 * into *d_status (device int) and the factorisation continues with pivot 1. */
int fmx_chol_leaf(const void* G, int n, int ld, int B, void* R, void* T, int* d_status, void* stream);

/* Host-only hooks of the continuous-time projective protocol (no device
 * needed).  fmx_poisson_draw: the draws of event e of trajectory traj under
 * seed, out[0] = u_wait, out[1] = site, out[2] = Born draw.  fmx_poisson_taps:
 * the stencil of exp(-i H~ tau) along a direction of length n (half-width w:
 * 2w + 1 taps at the offsets -w .. w; w < 0: n taps at 0 .. n-1), out as
 * (re, im) pairs.  fmx_poisson_width: the half-width used for every tau <= dt
 * (-1: every offset).  Return 0, or -1 on invalid arguments. */
int fmx_poisson_draw(unsigned long long seed, unsigned long long traj, long long e, int L, double* out);
int fmx_poisson_taps(int n, int w, double J, double tau, double* out);
int fmx_poisson_width(int n, double J, double dt);

/* Host-only hook of the tensor-core GEMM's tile orders (no device needed): the
 * tiles (row tile, column tile, batch item) of one launch in the order its
 * persistent loop takes them, CTA i taking positions i, i + G, i + 2G, ... of
 * a grid of G = min(grid, tiles) CTAs.  The launch has `batch` items of
 * 2 mt_mod row tiles (the real and imaginary halves of a complex product's
 * rows, mt_mod tiles each) by ntiles_n column tiles.  order: 0 grouped raster
 * (16 row tiles sweep the columns); 1 the row blocks r and mt_mod - 1 - r of a
 * triangular A paired in consecutive rounds (lower != 0: A lower triangular,
 * else upper; mt_mod even); 2 the column tiles c and ntiles_n - 1 - c of a
 * triangular B paired (ntiles_n even); 3 only the tiles on or above the
 * diagonal of a Hermitian product (ntiles_n == mt_mod).  out[3 t .. 3 t + 2]
 * for each position t; cap: entries of out / 3.  Returns the number of tiles,
 * or -1 on invalid arguments. */
int fmx_tile_order(int order, int mt_mod, int ntiles_n, int batch, int lower, int grid, int* out, int cap);

#ifdef __cplusplus
}
#endif
#endif /* FM_TESTING_H */
