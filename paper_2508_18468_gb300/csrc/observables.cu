// Density-density correlations of a Slater determinant (Eq. (2)) and the
// particle-number covariance of two regions (Eq. (GAB)), from C = U U^dag.
//
//   C_ij = -D_ij D_ji = -|C_ij|^2 (i != j);  c[d] = (1/L) sum_i C_{i, i+d} per
//   displacement class d = dx + Lx dy (periodic in x and y);
//   G_AB = -sum_{i in A, j in B} C_ij = sum |(U_A U_B^dag)_ij|^2.
//
// C is formed in column stripes by the complex GEMM of the state's precision
// (float64 for the FP64 state, complex64 for the mixed one) and reduced into
// the displacement bins stripe by stripe: one thread per bin, a fixed order of
// summation, so the result is deterministic.
#include "kernels.h"

namespace fm {

// complex64 copy of trajectory b's U (L x N, column-major) from the float state V_b
__global__ void v_to_c32_kernel(const float* __restrict__ V, int L, int N, c32* U) {
  const int64_t n = (int64_t)L * N;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < n; idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = idx % L, k = idx / L;
    U[idx] = cmk(V[i + k * 2 * L], V[L + i + k * 2 * L]);
  }
}

// rows `sites` of trajectory b's U as complex64 (n x N, column-major, ld n) from V_b
__global__ void gather_rows_c32_kernel(const float* __restrict__ V, int L, int N, const int* sites, int n, c32* out) {
  const int64_t tot = (int64_t)n * N;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < tot; idx += (int64_t)gridDim.x * blockDim.x) {
    const int r = (int)(idx % n);
    const int64_t k = idx / n;
    const int j = sites[r];
    out[idx] = cmk(V[j + k * 2 * L], V[L + j + k * 2 * L]);
  }
}

// bins[d] += sum_k |X[i + k L]|^2 over the stripe columns j = j0 + k (k < S),
// i = j - d with periodic wrap in x and y, skipping i == j; one thread per bin
template <typename T>
__global__ void displacement_bins_kernel(const cplx<T>* __restrict__ X, int L, int Lx, int Ly, int j0, int S,
                                         double* bins) {
  const int d = blockIdx.x * blockDim.x + threadIdx.x;
  if (d >= L || d == 0) return;
  const int dx = d % Lx, dy = d / Lx;
  double acc = 0.0;
  for (int k = 0; k < S; ++k) {
    const int j = j0 + k;
    const int jx = j % Lx, jy = j / Lx;
    const int ix = jx - dx < 0 ? jx - dx + Lx : jx - dx;
    const int iy = jy - dy < 0 ? jy - dy + Ly : jy - dy;
    const cplx<T> v = X[(ix + Lx * iy) + (int64_t)k * L];
    acc += (double)v.re * v.re + (double)v.im * v.im;
  }
  bins[d] += acc;
}

// per-block sums of |M|^2 over n entries (fixed order), then their sum
template <typename T>
__global__ void __launch_bounds__(256) abs2_partial_kernel(const cplx<T>* __restrict__ M, int64_t n, double* part) {
  __shared__ double red[8];
  double acc = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const cplx<T> v = M[i];
    acc += (double)v.re * v.re + (double)v.im * v.im;
  }
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < 8; ++w) s += red[w];
    part[blockIdx.x] = s;
  }
}

__global__ void sum_partials_kernel(const double* part, int np, double* out) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    double s = 0.0;
    for (int i = 0; i < np; ++i) s += part[i];
    *out = s;
  }
}

// ------------------------------------------------------------------ launchers
cudaError_t v_to_c32(cudaStream_t st, const float* V, int L, int N, c32* U) {
  v_to_c32_kernel<<<152 * 8, 256, 0, st>>>(V, L, N, U);
  return cudaGetLastError();
}

cudaError_t gather_rows_c32(cudaStream_t st, const float* V, int L, int N, const int* sites, int n, c32* out) {
  if (n <= 0) return cudaSuccess;
  gather_rows_c32_kernel<<<152 * 8, 256, 0, st>>>(V, L, N, sites, n, out);
  return cudaGetLastError();
}

template <typename T>
cudaError_t displacement_bins(cudaStream_t st, const cplx<T>* X, int L, int Lx, int Ly, int j0, int S, double* bins) {
  displacement_bins_kernel<T><<<FM_CEIL_DIV(L, 128), 128, 0, st>>>(X, L, Lx, Ly, j0, S, bins);
  return cudaGetLastError();
}
template cudaError_t displacement_bins<double>(cudaStream_t, const z64*, int, int, int, int, int, double*);
template cudaError_t displacement_bins<float>(cudaStream_t, const c32*, int, int, int, int, int, double*);

constexpr int kAbs2Blocks = 152 * 4;
int abs2_partials() { return kAbs2Blocks; }

template <typename T>
cudaError_t sum_abs2(cudaStream_t st, const cplx<T>* M, int64_t n, double* part, double* out) {
  abs2_partial_kernel<T><<<kAbs2Blocks, 256, 0, st>>>(M, n, part);
  sum_partials_kernel<<<1, 32, 0, st>>>(part, kAbs2Blocks, out);
  return cudaGetLastError();
}
template cudaError_t sum_abs2<double>(cudaStream_t, const z64*, int64_t, double*, double*);
template cudaError_t sum_abs2<float>(cudaStream_t, const c32*, int64_t, double*, double*);

}  // namespace fm
