// Entanglement entropy from a sketch of the cross-correlation block (mixed precision).
//
// For orthonormal orbitals U (L x N) the correlation matrix C = U U^dag is a
// projector (Sec. II), so for a subsystem A with complement B the eigenvalues of
// C_A obey lambda (1 - lambda) = sigma^2, sigma the singular values of the cross
// block X = C_AB = U_A U_B^dag (C_A - C_A^2 = C_AB C_BA).  The entropy terms
// f(lambda) = lambda ln lambda + (1 - lambda) ln(1 - lambda) are symmetric under
// lambda <-> 1 - lambda, so S_A = -sum f(lambda) depends on sigma^2 alone, and a
// sigma below 1e-5 adds less than 3e-9.  Entanglement spectra fall off
// exponentially, so X has a low numerical rank: randomized subspace iteration
// (Halko, Martinsson and Tropp, SIAM Review 53, 217 (2011)) finds its range with
// r ~ 10^2 vectors, and the eigenvalues of the r x r Rayleigh-Ritz matrix
// H = B B^dag, B = Q^dag X, are the sigma^2, in float64.
//
// Precision.  The products with U are complex64 GEMMs.  An error delta in X moves
// each sigma by at most delta, so lambda ~ sigma^2 moves by ~2 sigma delta: the
// eigenvalues near 0 and 1, whose terms decide the entropy's accuracy, move far
// less than an error delta in C_A itself would move them (by delta).  The
// orthonormal bases are made in float64 (two shifted CholeskyQR passes, the shift
// of Fukaya, Kannan, Nakatsukasa, Yamamoto and Yanagisawa, SIAM J. Sci. Comput. 42
// (2020)), and H is the exact-product Gram of the float-valued B^dag.  The sketch
// needs no projector correction: the departure of the float U from orthonormality
// (~1e-7) enters sigma^2 at second order.
#include <algorithm>

#include "kernels.h"

namespace fm {

namespace {

// Om (n x r, column-major): (+-1 +- i) / sqrt(2), Philox counter (i, j, 0, 5) under `seed`
__global__ void sketch_random_kernel(c32* Om, int n, int r, uint64_t seed) {
  const int64_t tot = (int64_t)n * r;
  const float a = 0.70710678118654752f;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < tot; idx += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(idx % n), j = (int)(idx / n);
    const philox_out o = philox4x32_10((uint32_t)i, (uint32_t)j, 0u, 5u, (uint32_t)(seed & 0xFFFFFFFFu),
                                       (uint32_t)(seed >> 32));
    Om[idx] = cmk((o.w[0] & 1u) ? a : -a, (o.w[1] & 1u) ? a : -a);
  }
}

__global__ void c32_to_z64_kernel(const c32* __restrict__ a, int64_t n, z64* b) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    b[i] = cmk((double)a[i].re, (double)a[i].im);
}

__global__ void z64_to_c32_kernel(const z64* __restrict__ a, int64_t n, c32* b) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    b[i] = cmk((float)a[i].re, (float)a[i].im);
}

// G += s I with s = c * trace(G) (one CTA): the shift of the first CholeskyQR pass
__global__ void __launch_bounds__(256) shift_diag_kernel(z64* G, int r, double c) {
  __shared__ double red[8];
  double t = 0.0;
  for (int i = threadIdx.x; i < r; i += blockDim.x) t += G[i + (int64_t)i * r].re;
  for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = t;
  __syncthreads();
  double tr = 0.0;
  for (int w = 0; w < 8; ++w) tr += red[w];
  const double s = c * tr + 1e-300;
  for (int i = threadIdx.x; i < r; i += blockDim.x) G[i + (int64_t)i * r].re += s;
}

// upper triangle of H from its lower triangle (the small eigen-solver reads both)
__global__ void mirror_lower_kernel(z64* H, int r) {
  const int64_t tot = (int64_t)r * r;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < tot; idx += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(idx % r), j = (int)(idx / r);
    if (i < j) H[idx] = cconj(H[j + (int64_t)i * r]);
  }
}

__global__ void copy_value_kernel(const double* src, double* dst) { *dst = *src; }

// G = sum_p Gp[p] over the upper triangle (r x r each), in order of p
__global__ void sum_partials_upper_kernel(const z64* __restrict__ Gp, int P, int r, z64* G) {
  const int64_t tot = (int64_t)r * r;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < tot; idx += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(idx % r), j = (int)(idx / r);
    if (i > j) continue;
    z64 a = Gp[idx];
    for (int q = 1; q < P; ++q) a = cadd(a, Gp[(int64_t)q * tot + idx]);
    G[idx] = a;
  }
}

// out (n x N, ld n) = rows of X (column-major, ld) as complex128
__global__ void rows_c32_to_z64_kernel(const c32* __restrict__ X, int64_t ld, int n, int N, z64* out) {
  const int64_t tot = (int64_t)n * N;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < tot; idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = idx % n, k = idx / n;
    const c32 v = X[i + k * ld];
    out[idx] = cmk((double)v.re, (double)v.im);
  }
}

size_t al256(size_t x) { return (x + 255) & ~(size_t)255; }

}  // namespace

cudaError_t rows_c32_to_z64(cudaStream_t st, const c32* X, int64_t ld, int n, int N, z64* out) {
  rows_c32_to_z64_kernel<<<152 * 8, 256, 0, st>>>(X, ld, n, N, out);
  return cudaGetLastError();
}

SketchScratch sketch_layout(void* base, int nmax, int N, int rmax) {
  SketchScratch w;
  char* p = (char*)base;
  auto take = [&](size_t bytes) { char* q = p; p += al256(bytes); return (void*)q; };
  const int64_t nr = (int64_t)nmax * rmax, rr = (int64_t)rmax * rmax;
  w.nmax = nmax; w.N = N; w.rmax = rmax;
  w.Om = (c32*)take(nr * sizeof(c32));
  w.Yc = (c32*)take(nr * sizeof(c32));
  w.Z = (c32*)take((int64_t)N * rmax * sizeof(c32));
  w.Yz = (z64*)take(nr * sizeof(z64));
  w.Yz2 = (z64*)take(nr * sizeof(z64));
  w.G = (z64*)take(rr * sizeof(z64));
  w.R = (z64*)take(rr * sizeof(z64));
  w.T = (z64*)take(rr * sizeof(z64));
  w.Dinv = (z64*)take((int64_t)FM_CEIL_DIV(rmax, CHOL_NB) * CHOL_NB * CHOL_NB * sizeof(z64));
  w.Xc = (z64*)take((int64_t)rmax * CHOL_NB * sizeof(z64));
  w.H = (z64*)take(rr * sizeof(z64));
  w.Gp = (z64*)take((int64_t)kSketchPartials * rr * sizeof(z64));
  w.vb = (z64*)take((int64_t)rmax * sizeof(z64));
  w.wb = (z64*)take((int64_t)rmax * sizeof(z64));
  w.pb = (z64*)take(std::max<int64_t>(hermitian_entropy_pbuf(rmax), 1 + 32 * (int64_t)rmax) * sizeof(z64));
  w.d = (double*)take((int64_t)rmax * 8);
  w.e = (double*)take((int64_t)rmax * 8);
  w.lam = (double*)take((int64_t)rmax * 8);
  w.S = (double*)take(16);
  w.status = (int*)take(16);
  w.xg = take(exact_gram_scratch_bytes(nmax, rmax));
  w.bytes = (size_t)(p - (char*)base);
  return w;
}

size_t sketch_scratch_bytes(int nmax, int N, int rmax) { return sketch_layout(nullptr, nmax, N, rmax).bytes + 256; }

namespace {

// G (r x r, upper triangle) = Y^dag Y for Y (n x r, ld n), split over row chunks so that
// the short, deep product fills the GPU: P chunks of c rows as one batched product plus
// the remaining rows, the partial Grams summed in a fixed order.
cudaError_t gram_split(cudaStream_t st, const z64* Y, int n, int r, const SketchScratch& w, int64_t* launches) {
  const z64 one = {1.0, 0.0}, zero = {0.0, 0.0};
  const int64_t rr = (int64_t)r * r;
  const int64_t cap = (int64_t)kSketchPartials * w.rmax * w.rmax / rr;      // partials that fit
  const int64_t pmax = std::min<int64_t>(std::min<int64_t>(64, cap - 1), n / 64);
  const int P = (int)std::max<int64_t>(1, pmax);
  const int c = n / P, rest = n - P * c;
  cudaError_t e;
  if ((e = zgemm<double>(st, r, r, c, OP_C, OP_N, one, Y, n, c, Y, n, c, zero, w.Gp, r, rr, P, GEMM_UPPER_ONLY)))
    return e;
  ++*launches;
  int np = P;
  if (rest > 0) {
    const z64* Yr = Y + (int64_t)P * c;
    if ((e = zgemm<double>(st, r, r, rest, OP_C, OP_N, one, Yr, n, 0, Yr, n, 0, zero, w.Gp + (int64_t)P * rr, r, 0, 1,
                           GEMM_UPPER_ONLY)))
      return e;
    ++*launches;
    ++np;
  }
  sum_partials_upper_kernel<<<FM_CEIL_DIV(rr, 256), 256, 0, st>>>(w.Gp, np, r, w.G);
  ++*launches;
  return cudaGetLastError();
}

// Y (n x r, complex64, in place) <- an orthonormal basis of its numerical range, in
// float64: two CholeskyQR passes on G + s I, s = 11 (n r + r (r + 1)) 2^-53 trace(G).
cudaError_t orth(cudaStream_t st, c32* Yc, int n, int r, const SketchScratch& w, int64_t* launches) {
  const z64 one = {1.0, 0.0}, zero = {0.0, 0.0};
  const int64_t nr = (int64_t)n * r;
  cudaError_t e;
  c32_to_z64_kernel<<<152 * 4, 256, 0, st>>>(Yc, nr, w.Yz);
  ++*launches;
  z64* a = w.Yz;
  z64* b = w.Yz2;
  for (int pass = 0; pass < 2; ++pass) {
    if ((e = gram_split(st, a, n, r, w, launches))) return e;
    // both passes shifted: Y may be numerically rank deficient (the sketch rank exceeds
    // the rank of C_AB), and the shift only perturbs the directions below it
    const double c = 11.0 * ((double)n * r + (double)r * (r + 1)) * 1.1102230246251565e-16;
    shift_diag_kernel<<<1, 256, 0, st>>>(w.G, r, c);
    ++*launches;
    if ((e = cholesky_inverse<double>(st, w.G, w.R, w.T, w.Dinv, w.Xc, r, r, 0, r, 1, w.status, launches))) return e;
    if ((e = zgemm<double>(st, n, r, r, OP_N, OP_N, one, a, n, 0, w.T, r, 0, zero, b, n, 0, 1, GEMM_TRI_B_UPPER)))
      return e;
    ++*launches;
    std::swap(a, b);
  }
  z64_to_c32_kernel<<<152 * 4, 256, 0, st>>>(a, nr, Yc);
  ++*launches;
  return cudaGetLastError();
}

}  // namespace

cudaError_t sketch_entropy(cudaStream_t st, const c32* U, int64_t ld, int nA, int nB, int N, int r, int q,
                           uint64_t seed, const SketchScratch& w, double* S_out, double* chk_out, int64_t* launches) {
  if (r < 32 || r % 32 || r > w.rmax || nA <= r || nB <= r || std::max(nA, nB) > w.nmax || N != w.N)
    return cudaErrorInvalidValue;
  const c32 one = {1.0f, 0.0f}, zero = {0.0f, 0.0f};
  const c32* XA = U;
  const c32* XB = U + nA;
  cudaError_t e;
  if ((e = cudaMemsetAsync(w.status, 0, sizeof(int), st))) return e;
  // Q = orth(X Om), X = XA XB^dag
  sketch_random_kernel<<<152 * 4, 256, 0, st>>>(w.Om, nB, r, seed);
  ++*launches;
  if ((e = zgemm<float>(st, N, r, nB, OP_C, OP_N, one, XB, ld, 0, w.Om, nB, 0, zero, w.Z, N, 0, 1, 0))) return e;
  if ((e = zgemm<float>(st, nA, r, N, OP_N, OP_N, one, XA, ld, 0, w.Z, N, 0, zero, w.Yc, nA, 0, 1, 0))) return e;
  *launches += 2;
  if ((e = orth(st, w.Yc, nA, r, w, launches))) return e;
  for (int it = 0; it < q; ++it) {
    // P = orth(X^dag Q), Q = orth(X P)
    if ((e = zgemm<float>(st, N, r, nA, OP_C, OP_N, one, XA, ld, 0, w.Yc, nA, 0, zero, w.Z, N, 0, 1, 0))) return e;
    if ((e = zgemm<float>(st, nB, r, N, OP_N, OP_N, one, XB, ld, 0, w.Z, N, 0, zero, w.Om, nB, 0, 1, 0))) return e;
    *launches += 2;
    if ((e = orth(st, w.Om, nB, r, w, launches))) return e;
    if ((e = zgemm<float>(st, N, r, nB, OP_C, OP_N, one, XB, ld, 0, w.Om, nB, 0, zero, w.Z, N, 0, 1, 0))) return e;
    if ((e = zgemm<float>(st, nA, r, N, OP_N, OP_N, one, XA, ld, 0, w.Z, N, 0, zero, w.Yc, nA, 0, 1, 0))) return e;
    *launches += 2;
    if ((e = orth(st, w.Yc, nA, r, w, launches))) return e;
  }
  // B^dag = X^dag Q (nB x r); H = conj(B B^dag) = (B^dag)^T conj(B^dag), exact products
  if ((e = zgemm<float>(st, N, r, nA, OP_C, OP_N, one, XA, ld, 0, w.Yc, nA, 0, zero, w.Z, N, 0, 1, 0))) return e;
  if ((e = zgemm<float>(st, nB, r, N, OP_N, OP_N, one, XB, ld, 0, w.Z, N, 0, zero, w.Om, nB, 0, 1, 0))) return e;
  *launches += 2;
  if ((e = exact_gram_c32(st, w.Om, nB, nB, r, w.H, w.xg, w.status, launches))) return e;
  if (!hermitian_entropy_lower_only(r)) {
    mirror_lower_kernel<<<FM_CEIL_DIV((int64_t)r * r, 256), 256, 0, st>>>(w.H, r);
    ++*launches;
  }
  int nl = 0;
  if ((e = hermitian_entropy(st, w.H, r, w.vb, w.wb, w.pb, nullptr, w.d, w.e, w.lam, S_out, &nl, 1))) return e;
  *launches += nl;
  // convergence: the p-th smallest Ritz value (ascending order), p = max(8, r / 8)
  const int p = std::max(8, r / 8);
  copy_value_kernel<<<1, 1, 0, st>>>(w.lam + (p - 1), chk_out);
  ++*launches;
  return cudaGetLastError();
}

}  // namespace fm
