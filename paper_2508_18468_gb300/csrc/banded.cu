// Structured propagation: U <- exp(-i H~ dt) U as a stencil.
//
// The ring's propagator is circulant, P_ab = p_{(a - b) mod L} with
// p_r = (1/L) sum_k e^{i k r} e^{-2 i J dt cos k} (App. A), and its entries fall
// off like Bessel functions, |p_r| ~ |J_r(2 J dt)|: below 1e-15 beyond r = 8 at
// dt = 0.05.  The torus propagator is P_x (x) P_y.  So P U is a stencil along
// x (then along y) over the taps above 1e-15 -- the same product as the dense
// GEMM up to those dropped entries, for one read and one write of U per
// direction instead of L^2 N multiply-adds.  Offsets and taps come from the
// host; tiny lattices keep every tap.
#include "kernels.h"

namespace fm {

template <typename T, int LAYOUT>
struct band_io;
template <typename T>
struct band_io<T, 0> {  // complex128 U, L x N per trajectory
  FM_DEVFN static cplx<T> ld(const void* base, int64_t b, int L, int N, int i, int k) {
    const z64 z = ((const z64*)base)[b * L * (int64_t)N + i + (int64_t)k * L];
    return cmk<T>((T)z.re, (T)z.im);
  }
  FM_DEVFN static void st(void* base, int64_t b, int L, int N, int i, int k, cplx<T> v) {
    ((z64*)base)[b * L * (int64_t)N + i + (int64_t)k * L] = cmk((double)v.re, (double)v.im);
  }
};
template <typename T>
struct band_io<T, 1> {  // float V, 2L x N per trajectory (column k = [Re; Im])
  FM_DEVFN static cplx<T> ld(const void* base, int64_t b, int L, int N, int i, int k) {
    const float* V = (const float*)base + b * 2 * L * (int64_t)N + (int64_t)k * 2 * L;
    return cmk<T>((T)V[i], (T)V[L + i]);
  }
  FM_DEVFN static void st(void* base, int64_t b, int L, int N, int i, int k, cplx<T> v) {
    float* V = (float*)base + b * 2 * L * (int64_t)N + (int64_t)k * 2 * L;
    V[i] = (float)v.re;
    V[L + i] = (float)v.im;
  }
};

// out[i, k] = sum_t taps[t] in[site i shifted back by off[t] along dir, k]; thread per
// site, a chunk of `per` columns per blockIdx.y; with `partial`, the row sums of
// |out|^2 over the chunk go to partial[(b nch + chunk) L + i].
template <typename T, int LAYOUT>
__global__ void band_prop_kernel(const void* in, void* out, int L, int N, int Lx, int Ly, int dir, const z64* taps,
                                 const int* off, int ntap, int per, double* partial, int nch) {
  __shared__ cplx<T> tp[kBandMaxTaps];
  __shared__ int of[kBandMaxTaps];
  for (int t = threadIdx.x; t < ntap; t += blockDim.x) {
    tp[t] = cmk<T>((T)taps[t].re, (T)taps[t].im);
    of[t] = off[t];
  }
  __syncthreads();
  const int64_t b = blockIdx.z;
  const int c = blockIdx.y;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= L) return;
  const int x = i % Lx, y = i / Lx;
  int src[kBandMaxTaps];
#pragma unroll 4
  for (int t = 0; t < ntap; ++t) {
    if (dir == 0) {
      int xs = (x - of[t]) % Lx;
      if (xs < 0) xs += Lx;
      src[t] = xs + Lx * y;
    } else {
      int ys = (y - of[t]) % Ly;
      if (ys < 0) ys += Ly;
      src[t] = x + Lx * ys;
    }
  }
  const int k0 = c * per, k1 = min(N, k0 + per);
  double s = 0.0;
  for (int k = k0; k < k1; ++k) {
    cplx<T> acc = cmk<T>((T)0, (T)0);
    for (int t = 0; t < ntap; ++t) {
      const cplx<T> u = band_io<T, LAYOUT>::ld(in, b, L, N, src[t], k);
      acc.re += tp[t].re * u.re - tp[t].im * u.im;
      acc.im += tp[t].re * u.im + tp[t].im * u.re;
    }
    band_io<T, LAYOUT>::st(out, b, L, N, i, k, acc);
    s += (double)acc.re * acc.re + (double)acc.im * acc.im;
  }
  if (partial) partial[(b * nch + c) * L + i] = s;
}

int band_chunks(int L, int N, int B) {
  const int blocks = FM_CEIL_DIV(L, 256) * B;
  return std::max(1, std::min(std::min(N, 128), FM_CEIL_DIV(4 * 152, blocks)));
}

cudaError_t band_propagate(cudaStream_t st, int layout, const void* in, void* out, int L, int N, int B, int Lx,
                           int Ly, int dir, const z64* taps, const int* off, int ntap, double* partial, int nch) {
  if (ntap < 1 || ntap > kBandMaxTaps) return cudaErrorInvalidValue;
  const int per = FM_CEIL_DIV(N, nch);
  const dim3 grid(FM_CEIL_DIV(L, 256), nch, B);
  if (layout == 0)
    band_prop_kernel<double, 0><<<grid, 256, 0, st>>>(in, out, L, N, Lx, Ly, dir, taps, off, ntap, per, partial, nch);
  else
    band_prop_kernel<float, 1><<<grid, 256, 0, st>>>(in, out, L, N, Lx, Ly, dir, taps, off, ntap, per, partial, nch);
  return cudaGetLastError();
}

}  // namespace fm
