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
// |out|^2 over the chunk go to partial[(b nch + chunk) L + i].  The offsets are
// consecutive (off[t] = off[0] + t), so the source site steps back by one along
// dir (with wrap) from tap to tap: no per-tap index array.
template <typename T, int LAYOUT>
__global__ void __launch_bounds__(256) band_prop_kernel(const void* in, void* out, int L, int N, int Lx, int Ly,
                                                        int dir, const z64* taps, const int* off, int ntap, int per,
                                                        double* partial, int nch, int tap_stride) {
  __shared__ cplx<T> tp[kBandMaxTaps];
  const int64_t b = blockIdx.z;
  taps += b * tap_stride;                     // per-trajectory taps when tap_stride > 0
  for (int t = threadIdx.x; t < ntap; t += blockDim.x) tp[t] = cmk<T>((T)taps[t].re, (T)taps[t].im);
  __syncthreads();
  const int c = blockIdx.y;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= L) return;
  const int x = i % Lx, y = i / Lx;
  const int n = dir == 0 ? Lx : Ly;           // period along dir
  const int stride = dir == 0 ? 1 : Lx;       // site step along dir
  const int pos = dir == 0 ? x : y;
  int p0 = (pos - off[0]) % n;                // source position of tap 0
  if (p0 < 0) p0 += n;
  const int base = i - pos * stride;          // site with coordinate 0 along dir
  const int k0 = c * per, k1 = min(N, k0 + per);
  double s = 0.0;
  for (int k = k0; k < k1; ++k) {
    cplx<T> acc = cmk<T>((T)0, (T)0);
    int p = p0;
    for (int t = 0; t < ntap; ++t) {
      const cplx<T> u = band_io<T, LAYOUT>::ld(in, b, L, N, base + p * stride, k);
      acc.re += tp[t].re * u.re - tp[t].im * u.im;
      acc.im += tp[t].re * u.im + tp[t].im * u.re;
      p = p == 0 ? n - 1 : p - 1;
    }
    band_io<T, LAYOUT>::st(out, b, L, N, i, k, acc);
    if (partial) s += (double)(acc.re * acc.re + acc.im * acc.im);
  }
  if (partial) partial[(b * nch + c) * L + i] = s;
}

int band_chunks(int L, int N, int B) {
  const int blocks = FM_CEIL_DIV(L, 256) * B;
  return std::max(1, std::min(std::min(N, 128), FM_CEIL_DIV(4 * 152, blocks)));
}

cudaError_t band_propagate(cudaStream_t st, int layout, const void* in, void* out, int L, int N, int B, int Lx,
                           int Ly, int dir, const z64* taps, const int* off, int ntap, double* partial, int nch,
                           int tap_stride) {
  if (ntap < 1 || ntap > kBandMaxTaps) return cudaErrorInvalidValue;
  const int per = FM_CEIL_DIV(N, nch);
  const dim3 grid(FM_CEIL_DIV(L, 256), nch, B);
  if (layout == 0)
    band_prop_kernel<double, 0><<<grid, 256, 0, st>>>(in, out, L, N, Lx, Ly, dir, taps, off, ntap, per, partial, nch,
                                                      tap_stride);
  else
    band_prop_kernel<float, 1><<<grid, 256, 0, st>>>(in, out, L, N, Lx, Ly, dir, taps, off, ntap, per, partial, nch,
                                                     tap_stride);
  return cudaGetLastError();
}


// ------------------------------------------------------------------ Runge-Kutta step of Eq. (QSD_evo)
// One Horner stage of the fourth-order Taylor polynomial of X = A dt,
// A dt = -i dt H~ + diag(m), m_i = ln w_i (w = exp(m) from reduce_occupations):
//   out = U0 + c X Y,   (X Y)_i = -i dt J sum_{nearest neighbours j of i} Y_j + m_i Y_i.
// With c = 1/4, 1/3, 1/2, 1 in turn starting from Y = U0 the last stage gives
// U0 + X U0 + X^2 U0 / 2 + X^3 U0 / 6 + X^4 U0 / 24, the RK4 step of the linear
// constant-coefficient equation.  Neighbours x +- 1 (and y +- 1 on the torus),
// periodic; a direction of length 2 counts its one neighbour twice, as H~ does.
template <typename T, int LAYOUT>
__global__ void rk4_stage_kernel(const void* U0, const void* Y, void* out, int L, int N, int Lx, int Ly,
                                 const double* __restrict__ w, double dtJ, double c, int per) {
  const int64_t b = blockIdx.z;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= L) return;
  const int x = i % Lx, y = i / Lx;
  const int xp = (x + 1) % Lx + Lx * y, xm = (x + Lx - 1) % Lx + Lx * y;
  const int yp = Ly > 1 ? x + Lx * ((y + 1) % Ly) : -1, ym = Ly > 1 ? x + Lx * ((y + Ly - 1) % Ly) : -1;
  const T m = (T)log(w[b * L + i]);
  const T h = (T)dtJ, cc = (T)c;
  const int k0 = blockIdx.y * per, k1 = min(N, k0 + per);
  for (int k = k0; k < k1; ++k) {
    cplx<T> s = cadd(band_io<T, LAYOUT>::ld(Y, b, L, N, xp, k), band_io<T, LAYOUT>::ld(Y, b, L, N, xm, k));
    if (yp >= 0) s = cadd(s, cadd(band_io<T, LAYOUT>::ld(Y, b, L, N, yp, k), band_io<T, LAYOUT>::ld(Y, b, L, N, ym, k)));
    const cplx<T> yi = band_io<T, LAYOUT>::ld(Y, b, L, N, i, k);
    // X Y = -i h s + m y_i
    const cplx<T> xy = cmk<T>(h * s.im + m * yi.re, -h * s.re + m * yi.im);
    const cplx<T> u0 = band_io<T, LAYOUT>::ld(U0, b, L, N, i, k);
    band_io<T, LAYOUT>::st(out, b, L, N, i, k, cmk<T>(u0.re + cc * xy.re, u0.im + cc * xy.im));
  }
}

cudaError_t rk4_stage(cudaStream_t st, int layout, const void* U0, const void* Y, void* out, int L, int N, int B,
                      int Lx, int Ly, const double* w, double dtJ, double c) {
  const int nch = band_chunks(L, N, B);
  const int per = FM_CEIL_DIV(N, nch);
  const dim3 grid(FM_CEIL_DIV(L, 256), nch, B);
  if (layout == 0)
    rk4_stage_kernel<double, 0><<<grid, 256, 0, st>>>(U0, Y, out, L, N, Lx, Ly, w, dtJ, c, per);
  else
    rk4_stage_kernel<float, 1><<<grid, 256, 0, st>>>(U0, Y, out, L, N, Lx, Ly, w, dtJ, c, per);
  return cudaGetLastError();
}

}  // namespace fm
