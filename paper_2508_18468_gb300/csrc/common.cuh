// Common device / host definitions of the fm library (sm_103a).
#pragma once

#include <cuda_runtime.h>
#include <cuda_fp16.h>
#include <stdint.h>

#include "fm.h"

#define FM_DEVFN __device__ __forceinline__

// ------------------------------------------------------------------ complex
template <typename T> struct cplx { T re, im; };
typedef cplx<double> z64;
typedef cplx<float> c32;

template <typename T> FM_DEVFN cplx<T> cmk(T r, T i) { cplx<T> z; z.re = r; z.im = i; return z; }
template <typename T> FM_DEVFN cplx<T> cadd(cplx<T> a, cplx<T> b) { return cmk(a.re + b.re, a.im + b.im); }
template <typename T> FM_DEVFN cplx<T> csub(cplx<T> a, cplx<T> b) { return cmk(a.re - b.re, a.im - b.im); }
template <typename T> FM_DEVFN cplx<T> cmul(cplx<T> a, cplx<T> b) {
  return cmk(a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re);
}
template <typename T> FM_DEVFN cplx<T> cconj(cplx<T> a) { return cmk(a.re, -a.im); }
template <typename T> FM_DEVFN cplx<T> cscale(cplx<T> a, T s) { return cmk(a.re * s, a.im * s); }
template <typename T> FM_DEVFN T cabs2(cplx<T> a) { return a.re * a.re + a.im * a.im; }
// acc += a * b
template <typename T> FM_DEVFN void cfma(cplx<T>& acc, cplx<T> a, cplx<T> b) {
  acc.re = fma(a.re, b.re, acc.re);
  acc.re = fma(-a.im, b.im, acc.re);
  acc.im = fma(a.re, b.im, acc.im);
  acc.im = fma(a.im, b.re, acc.im);
}

// ------------------------------------------------------------------ Philox4x32-10
// Salmon, Moraes, Dror, Shaw, SC'11: ten rounds of (multiply words 0 and 2 by
// M0, M1 into 64-bit products; new counter = (hi1^c1^k0, lo1, hi0^c3^k1, lo0)),
// the key advanced by the Weyl increments W0, W1 between rounds.
struct philox_out { uint32_t w[4]; };

FM_DEVFN philox_out philox4x32_10(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                  uint32_t k0, uint32_t k1) {
  const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
  const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r > 0) { k0 += W0; k1 += W1; }
    uint32_t hi0 = __umulhi(M0, c0), lo0 = M0 * c0;
    uint32_t hi1 = __umulhi(M1, c2), lo1 = M1 * c2;
    uint32_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
    c0 = n0; c1 = lo1; c2 = n2; c3 = lo0;
  }
  philox_out o; o.w[0] = c0; o.w[1] = c1; o.w[2] = c2; o.w[3] = c3;
  return o;
}

enum { FM_TAG_MEASURE = 1, FM_TAG_NOISE = 2 };

// Draw for (site, step, trajectory, tag) under `seed`.
// Replay of projective outcomes (fm_force_outcomes): f holds n entries (step, trajectory,
// site, outcome) sorted by (step, trajectory, site).  Returns the forced outcome of the
// measurement of `site` by trajectory b at `step`, or -1 if it is not listed.
FM_DEVFN int fm_forced_outcome(const int4* f, int n, int64_t step, int b, int site) {
  if (n <= 0 || step > 0x7fffffff) return -1;
  const int st = (int)step;
  int lo = 0, hi = n;
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    const int4 e = f[mid];
    const bool less = e.x < st || (e.x == st && (e.y < b || (e.y == b && e.z < site)));
    if (less) lo = mid + 1; else hi = mid;
  }
  if (lo < n) {
    const int4 e = f[lo];
    if (e.x == st && e.y == b && e.z == site) return e.w;
  }
  return -1;
}
// The outcome draw that makes the rule "outcome 1 iff u < p" (p clamped to [0, 1]) give
// the forced outcome: -1 forces a click, 2 a no-click.
FM_DEVFN double fm_forced_u(int outcome) { return outcome ? -1.0 : 2.0; }

FM_DEVFN philox_out fm_draw(uint64_t seed, uint64_t traj, int64_t step, int site, uint32_t tag) {
  return philox4x32_10((uint32_t)site, (uint32_t)step, (uint32_t)(traj & 0xFFFFFFFFu),
                       tag | ((uint32_t)(traj >> 32) << 8),
                       (uint32_t)(seed & 0xFFFFFFFFu), (uint32_t)(seed >> 32));
}

// 53-bit uniform double in [0, 1): 27 bits of wa, 26 of wb (exact in double).
FM_DEVFN double fm_u53(uint32_t wa, uint32_t wb) {
  return ((double)(wa >> 5) * 67108864.0 + (double)(wb >> 6)) * (1.0 / 9007199254740992.0);
}

// Box-Muller standard normal from one draw.
FM_DEVFN double fm_normal(philox_out o) {
  double u1 = fm_u53(o.w[0], o.w[1]);
  double u2 = fm_u53(o.w[2], o.w[3]);
  return sqrt(-2.0 * log1p(-u1)) * cos(2.0 * 3.141592653589793 * u2);
}

// ------------------------------------------------------------------ device error flags
// Bit flags written by kernels into the state's status word; read by the host
// at synchronisation points.
enum { FM_DEVERR_PIVOT = 1, FM_DEVERR_NONFINITE = 2, FM_DEVERR_TIMEOUT = 4, FM_DEVERR_BOUNDS = 8,
       FM_DEVERR_REORTH = 16 };

// ------------------------------------------------------------------ host helpers
#define FM_CEIL_DIV(a, b) (((a) + (b) - 1) / (b))
