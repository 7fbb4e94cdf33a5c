// FP64 entanglement entropy of a Hermitian correlation block (Sec. II):
// S = -sum_i f(lambda_i), f(x) = x ln x + (1-x) ln(1-x), lambda the eigenvalues
// of the m x m Hermitian matrix M (C_A = U_A U_A^dag or U_A^dag U_A).
//
// Eigenvalues: Householder reduction to a real symmetric tridiagonal matrix
// (reflectors H = I - tau v v^dag with v_0 = 1 and real beta, so that
// H^dag x = beta e_1), then Sturm-sequence bisection, one eigenvalue per thread.
// Everything is float64 and deterministic (fixed-order reductions).
#include <float.h>
#include <math.h>

#include "kernels.h"

namespace fm {

// ------------------------------------------------------------------ helpers
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// fixed-order block sum for blockDim.x a multiple of 32, <= 1024 (red: 33 doubles of shared memory)
__device__ double bsum(double v, double* red) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  v = warp_sum(v);
  if (lane == 0) red[warp] = v;
  __syncthreads();
  if (warp == 0) {
    double s = (lane < (int)(blockDim.x >> 5)) ? red[lane] : 0.0;
    s = warp_sum(s);
    if (lane == 0) red[32] = s;
  }
  __syncthreads();
  const double s = red[32];
  __syncthreads();
  return s;
}

// Reflector for x = M[k+1 .. m-1, k] (length n): beta, tau, v (v_0 = 1), by
// the construction H^dag x = beta e_1, beta = -sign(Re x_0) |x|, tau = (beta - x_0)/beta,
// v_i = x_i / (x_0 - beta).  Returns tau; writes v and beta.
__device__ z64 reflector(const z64* x, int n, z64* v, double* beta_out, double* red, z64* sh) {
  double s = 0.0;
  for (int i = 1 + threadIdx.x; i < n; i += blockDim.x) s += cabs2(x[i]);
  const double xn2 = bsum(s, red);
  if (threadIdx.x == 0) {
    const z64 a = x[0];
    z64 tau, scale;
    double beta;
    if (xn2 == 0.0 && a.im == 0.0) {
      tau = cmk(0.0, 0.0);
      beta = a.re;
      scale = cmk(0.0, 0.0);
    } else {
      beta = -copysign(sqrt(cabs2(a) + xn2), a.re);
      tau = cmk((beta - a.re) / beta, -a.im / beta);
      // scale = 1 / (a - beta)
      const z64 d = cmk(a.re - beta, a.im);
      const double dd = cabs2(d);
      scale = cmk(d.re / dd, -d.im / dd);
    }
    sh[0] = tau;
    sh[1] = scale;
    *beta_out = beta;
  }
  __syncthreads();
  const z64 scale = sh[1];
  for (int i = threadIdx.x; i < n; i += blockDim.x) v[i] = (i == 0) ? cmk(1.0, 0.0) : cmul(x[i], scale);
  const z64 tau = sh[0];
  __syncthreads();
  return tau;
}

// ------------------------------------------------------------------ small m: one CTA
// The whole reduction in one CTA of 1024 threads; the matrix stays in global
// memory (L2 resident for the sizes this is used for).
__global__ void __launch_bounds__(1024) tridiag_small_kernel(z64* M, int m, z64* vb, z64* wb, double* d, double* e) {
  __shared__ double red[33];
  __shared__ z64 sh[4];
  __shared__ double sbeta;
  for (int k = 0; k + 1 < m; ++k) {
    const int n = m - k - 1;
    z64* col = M + (k + 1) + (int64_t)k * m;
    z64* M22 = M + (k + 1) + (int64_t)(k + 1) * m;
    const z64 tau = reflector(col, n, vb, &sbeta, red, sh);
    if (threadIdx.x == 0) { d[k] = M[k + (int64_t)k * m].re; e[k] = sbeta; }
    // p = M22 v, one warp per row i: p_i = sum_j conj(M22[j, i]) v_j (M22 Hermitian, so
    // the lanes read column i, contiguous); then s = v^dag p
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int i = warp; i < n; i += (int)(blockDim.x >> 5)) {
      const z64* ci = M22 + (int64_t)i * m;
      double ar = 0.0, ai = 0.0;
      for (int j = lane; j < n; j += 32) {
        const z64 a = ci[j], x = vb[j];
        ar += a.re * x.re + a.im * x.im;             // conj(a) x
        ai += a.re * x.im - a.im * x.re;
      }
      ar = warp_sum(ar);
      ai = warp_sum(ai);
      if (lane == 0) wb[i] = cmk(ar, ai);
    }
    __syncthreads();
    double sr = 0.0, si = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
      const z64 t = cmul(cconj(vb[i]), wb[i]);
      sr += t.re; si += t.im;
    }
    const double s_re = bsum(sr, red);
    const double s_im = bsum(si, red);
    // w = tau p - (1/2)|tau|^2 s v
    const double t2 = 0.5 * cabs2(tau);
    const z64 cs = cmk(t2 * s_re, t2 * s_im);
    for (int i = threadIdx.x; i < n; i += blockDim.x) wb[i] = csub(cmul(tau, wb[i]), cmul(cs, vb[i]));
    __syncthreads();
    // M22 -= v w^dag + w v^dag, every element by its own thread (coalesced along i)
    for (int idx = threadIdx.x; idx < n * n; idx += blockDim.x) {
      const int i = idx % n, j = idx / n;
      z64& a = M22[i + (int64_t)j * m];
      a = csub(a, cadd(cmul(vb[i], cconj(wb[j])), cmul(wb[i], cconj(vb[j]))));
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) d[m - 1] = M[(m - 1) + (int64_t)(m - 1) * m].re;
}

// ------------------------------------------------------------------ large m: per-column kernels
// Only the lower triangle (i >= j) of the trailing block is read and updated.
// Column k of the trailing matrix, after the rank-2 update still pending from
// column k - 1 (vp, wp: that column's reflector and w, indexed from row k), then
// its reflector.  One CTA.
__global__ void __launch_bounds__(256) hh_reflector_kernel(z64* M, int m, int k, const z64* __restrict__ vp,
                                                           const z64* __restrict__ wp, z64* vb, double* d,
                                                           double* e, z64* tau_out) {
  __shared__ double red[33];
  __shared__ z64 sh[4];
  __shared__ double sbeta;
  z64* col = M + k + (int64_t)k * m;          // rows k .. m-1 of column k
  if (vp) {
    const z64 w0c = cconj(wp[0]), v0c = cconj(vp[0]);
    for (int i = threadIdx.x; i < m - k; i += blockDim.x)
      col[i] = csub(col[i], cadd(cmul(vp[i], w0c), cmul(wp[i], v0c)));
    __syncthreads();
  }
  const int n = m - k - 1;
  const z64 tau = reflector(col + 1, n, vb, &sbeta, red, sh);
  if (threadIdx.x == 0) {
    d[k] = col[0].re;
    e[k] = sbeta;
    *tau_out = tau;
  }
}

constexpr int HT = EIG_TILE;  // tile of the Hermitian matrix-vector product (17 KB of shared memory)

// One pass over the lower triangle of the trailing block M22 (rows and columns
// k+1 .. m-1) per column: first the rank-2 update left pending by column k - 1,
// M22 -= v' w'^dag + w' v'^dag (vp, wp indexed from row k, so element (i, j) of
// M22 uses entries i + 1 and j + 1), written back; then p = M22 v from the
// updated tile: tile (I, J), J <= I, adds sum_j M_ij v_j to prow[J][i] and
// sum_{i > j} conj(M_ij) v_i to pcol[I][j].  The tile is staged in shared
// memory (column stride HT + 1) and read once with a row mapping and once with
// a column mapping; no shuffles.  Reading and writing each element once per
// column, instead of once for the product and again for the update.
__global__ void __launch_bounds__(256) hemv_lower_kernel(z64* M, int m, int k, const z64* __restrict__ vp,
                                                         const z64* __restrict__ wp, const z64* __restrict__ vb,
                                                         z64* prow, z64* pcol) {
  const int n = m - k - 1;
  z64* M22 = M + (k + 1) + (int64_t)(k + 1) * m;
  // decode lower tile t = I (I+1)/2 + J
  const int t = blockIdx.x;
  int I = (int)((sqrt(8.0 * t + 1.0) - 1.0) * 0.5);
  while ((I + 1) * (I + 2) / 2 <= t) ++I;
  while (I * (I + 1) / 2 > t) --I;
  const int J = t - I * (I + 1) / 2;
  extern __shared__ z64 tile[];             // HT columns of HT + 1
  constexpr int NQ = 256 / HT;               // phases
  __shared__ z64 vi_s[HT], vj_s[HT];
  __shared__ z64 red_s[NQ][HT + 1];
  __shared__ z64 pv_i[HT], pw_i[HT], pv_j[HT], pw_j[HT];
  const int lo = threadIdx.x % HT, q = threadIdx.x / HT;
  if (threadIdx.x < HT) {
    const int ii = I * HT + threadIdx.x, jj = J * HT + threadIdx.x;
    vi_s[threadIdx.x] = ii < n ? vb[ii] : cmk(0.0, 0.0);
    vj_s[threadIdx.x] = jj < n ? vb[jj] : cmk(0.0, 0.0);
    if (vp) {
      pv_i[threadIdx.x] = ii < n ? vp[ii + 1] : cmk(0.0, 0.0);
      pw_i[threadIdx.x] = ii < n ? wp[ii + 1] : cmk(0.0, 0.0);
      pv_j[threadIdx.x] = jj < n ? cconj(vp[jj + 1]) : cmk(0.0, 0.0);
      pw_j[threadIdx.x] = jj < n ? cconj(wp[jj + 1]) : cmk(0.0, 0.0);
    }
  }
  __syncthreads();
  for (int cc = q; cc < HT; cc += NQ) {
    const int i = I * HT + lo, j = J * HT + cc;
    z64 a = cmk(0.0, 0.0);
    if (i < n && j < n && j <= i) {
      z64* ap = &M22[i + (int64_t)j * m];
      a = *ap;
      if (vp) {
        a = csub(a, cadd(cmul(pv_i[lo], pw_j[cc]), cmul(pw_i[lo], pv_j[cc])));
        *ap = a;
      }
    }
    tile[cc * (HT + 1) + lo] = a;            // zero above the diagonal and outside
  }
  __syncthreads();
  // rows: sum_j M_ij v_j (diagonal included)
  z64 acc = cmk(0.0, 0.0);
  for (int cc = q; cc < HT; cc += NQ) cfma(acc, tile[cc * (HT + 1) + lo], vj_s[cc]);
  red_s[q][lo] = acc;
  __syncthreads();
  if (threadIdx.x < HT) {
    const int ii = I * HT + threadIdx.x;
    z64 s2 = cmk(0.0, 0.0);
    for (int qq = 0; qq < NQ; ++qq) s2 = cadd(s2, red_s[qq][threadIdx.x]);
    if (ii < n) prow[(int64_t)J * n + ii] = s2;
  }
  __syncthreads();
  // columns: sum_{i > j} conj(M_ij) v_i (strictly lower; on the diagonal tile skip i == j)
  acc = cmk(0.0, 0.0);
  const bool diag_tile = (I == J);
  for (int rr = q; rr < HT; rr += NQ) {
    if (diag_tile && rr <= lo) continue;
    cfma(acc, cconj(tile[lo * (HT + 1) + rr]), vi_s[rr]);
  }
  red_s[q][lo] = acc;
  __syncthreads();
  if (threadIdx.x < HT) {
    const int jj = J * HT + threadIdx.x;
    z64 s2 = cmk(0.0, 0.0);
    for (int qq = 0; qq < NQ; ++qq) s2 = cadd(s2, red_s[qq][threadIdx.x]);
    if (jj < n) pcol[(int64_t)I * n + jj] = s2;
  }
}

// p_i = sum_{J <= I(i)} prow[J][i] + sum_{I >= J(i)} pcol[I][i]; also partial v^dag p per block
__global__ void hemv_reduce_kernel(int m, int k, const z64* __restrict__ prow, const z64* __restrict__ pcol,
                                   const z64* __restrict__ vb, z64* p, z64* sdot) {
  const int n = m - k - 1;
  const int nb = FM_CEIL_DIV(n, HT);
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  double sr = 0.0, si = 0.0;
  if (i < n) {
    const int Ii = i / HT;
    z64 acc = cmk(0.0, 0.0);
    for (int J = 0; J <= Ii; ++J) acc = cadd(acc, prow[(int64_t)J * n + i]);
    for (int I = Ii; I < nb; ++I) acc = cadd(acc, pcol[(int64_t)I * n + i]);
    p[i] = acc;
    const z64 t = cmul(cconj(vb[i]), acc);
    sr = t.re; si = t.im;
  }
  __shared__ double red_r[8], red_i[8];
  for (int o = 16; o > 0; o >>= 1) {
    sr += __shfl_xor_sync(0xffffffffu, sr, o);
    si += __shfl_xor_sync(0xffffffffu, si, o);
  }
  if ((threadIdx.x & 31) == 0) { red_r[threadIdx.x >> 5] = sr; red_i[threadIdx.x >> 5] = si; }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0.0, b = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) { a += red_r[w]; b += red_i[w]; }
    sdot[blockIdx.x] = cmk(a, b);
  }
}

// w = tau p - (1/2)|tau|^2 (v^dag p) v, v^dag p from the per-block partials (fixed order)
__global__ void hh_w_kernel(int m, int k, const z64* __restrict__ p, const z64* __restrict__ sdot, int nsd,
                            const z64* __restrict__ vb, z64* wb, const z64* tau_in) {
  const int n = m - k - 1;
  __shared__ z64 s_sh;
  if (threadIdx.x == 0) {
    z64 s = cmk(0.0, 0.0);
    for (int b = 0; b < nsd; ++b) s = cadd(s, sdot[b]);
    s_sh = s;
  }
  __syncthreads();
  const z64 tau = *tau_in;
  const double t2 = 0.5 * cabs2(tau);
  const z64 cs = cmk(t2 * s_sh.re, t2 * s_sh.im);
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    wb[i] = csub(cmul(tau, p[i]), cmul(cs, vb[i]));
}

// the last diagonal entry after the update pending from column m - 2 (vp, wp of length 1)
__global__ void last_diag_kernel(const z64* M, int m, const z64* vp, const z64* wp, double* d) {
  double a = M[(m - 1) + (int64_t)(m - 1) * m].re;
  if (vp) a -= 2.0 * (vp[0].re * wp[0].re + vp[0].im * wp[0].im);
  d[m - 1] = a;
}

// ------------------------------------------------------------------ bisection
// count of eigenvalues of the symmetric tridiagonal (d, e) below x (Sturm / LDL^T inertia)
__device__ int sturm_count(const double* d, const double* e, int m, double x, double pivmin) {
  int c = 0;
  double q = d[0] - x;
  if (fabs(q) < pivmin) q = -pivmin;
  if (q < 0.0) ++c;
  for (int i = 1; i < m; ++i) {
    q = d[i] - x - e[i - 1] * e[i - 1] / q;
    if (fabs(q) < pivmin) q = -pivmin;
    if (q < 0.0) ++c;
  }
  return c;
}

// Eigenvalue q of the tridiagonal (d, e) by bisection, one thread per eigenvalue (large m:
// enough threads to fill the GPU, and the fewest Sturm sequences).
__global__ void bisect_thread_kernel(const double* __restrict__ d, const double* __restrict__ e, int m,
                                     double* lam) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= m) return;
  double lo = d[0], hi = d[0], emax2 = 0.0;
  for (int i = 0; i < m; ++i) {
    const double r = (i > 0 ? fabs(e[i - 1]) : 0.0) + (i + 1 < m ? fabs(e[i]) : 0.0);
    lo = fmin(lo, d[i] - r);
    hi = fmax(hi, d[i] + r);
    if (i + 1 < m) emax2 = fmax(emax2, e[i] * e[i]);
  }
  const double pivmin = DBL_MIN * fmax(1.0, emax2);
  const double span = fmax(fabs(lo), fabs(hi));
  lo -= 2.0 * DBL_EPSILON * span + pivmin;
  hi += 2.0 * DBL_EPSILON * span + pivmin;
  for (int it = 0; it < 200; ++it) {
    const double mid = 0.5 * (lo + hi);
    if (hi - lo <= 1e-18 + 2.0 * DBL_EPSILON * fabs(mid) || mid == lo || mid == hi) break;
    if (sturm_count(d, e, m, mid, pivmin) > q) hi = mid;
    else lo = mid;
  }
  lam[q] = 0.5 * (lo + hi);
}

// Eigenvalue q of the tridiagonal (d, e) by multisection, one warp per eigenvalue (small
// m, where one thread per eigenvalue leaves most of the GPU idle): each
// round the 32 lanes count the eigenvalues below 32 interior points of [lo, hi] that
// split it into 33 equal parts (one Sturm sequence per lane), and the part holding
// eigenvalue q becomes the new interval -- ~5 bits per round instead of bisection's 1.
// Gershgorin bounds and the stopping rule are bisection's: width <= 1e-18 + 2 eps |mid|.
__global__ void __launch_bounds__(128) bisect_kernel(const double* __restrict__ d, const double* __restrict__ e,
                                                     int m, double* lam) {
  const int lane = threadIdx.x & 31;
  const int q = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (q >= m) return;                              // warp-uniform
  double lo = INFINITY, hi = -INFINITY, emax2 = 0.0;
  for (int i = lane; i < m; i += 32) {
    const double r = (i > 0 ? fabs(e[i - 1]) : 0.0) + (i + 1 < m ? fabs(e[i]) : 0.0);
    lo = fmin(lo, d[i] - r);
    hi = fmax(hi, d[i] + r);
    if (i + 1 < m) emax2 = fmax(emax2, e[i] * e[i]);
  }
  for (int o = 16; o > 0; o >>= 1) {
    lo = fmin(lo, __shfl_xor_sync(0xffffffffu, lo, o));
    hi = fmax(hi, __shfl_xor_sync(0xffffffffu, hi, o));
    emax2 = fmax(emax2, __shfl_xor_sync(0xffffffffu, emax2, o));
  }
  const double pivmin = DBL_MIN * fmax(1.0, emax2);
  const double span = fmax(fabs(lo), fabs(hi));
  lo -= 2.0 * DBL_EPSILON * span + pivmin;
  hi += 2.0 * DBL_EPSILON * span + pivmin;
  for (int it = 0; it < 64; ++it) {
    const double mid = 0.5 * (lo + hi);
    if (hi - lo <= 1e-18 + 2.0 * DBL_EPSILON * fabs(mid)) break;
    const double x = lo + (hi - lo) * (double)(lane + 1) / 33.0;
    const bool above = (x > lo && x < hi) ? sturm_count(d, e, m, x, pivmin) > q : (x >= hi);
    const unsigned b = __ballot_sync(0xffffffffu, above);
    // points 0..k-1 have at most q eigenvalues below them, point k more (k = 32: none)
    const int k = b ? __ffs(b) - 1 : 32;
    const double nlo = k > 0 ? __shfl_sync(0xffffffffu, x, k - 1) : lo;
    const double nhi = k < 32 ? __shfl_sync(0xffffffffu, x, k) : hi;
    if (nlo == lo && nhi == hi) break;             // no representable progress
    lo = nlo;
    hi = nhi;
  }
  if (lane == 0) lam[q] = 0.5 * (lo + hi);
}

// S = -sum f(clamp(lambda, 0, 1)), one CTA, fixed order.  cross != 0: the inputs are
// sigma^2 = lambda (1 - lambda) in [0, 1/4], lambda = 2 sigma^2 / (1 + sqrt(1 - 4 sigma^2))
// (the root below 1/2; f is symmetric, so the other root gives the same term)
__global__ void __launch_bounds__(1024) entropy_sum_kernel(const double* lam, int m, double* S, int cross) {
  __shared__ double red[33];
  double s = 0.0;
  for (int q = threadIdx.x; q < m; q += blockDim.x) {
    double x;
    if (cross) {
      const double y = fmin(fmax(lam[q], 0.0), 0.25);
      x = 2.0 * y / (1.0 + sqrt(1.0 - 4.0 * y));
    } else {
      x = fmin(fmax(lam[q], 0.0), 1.0);
    }
    if (x > 0.0 && x < 1.0) s += x * log(x) + (1.0 - x) * log1p(-x);
  }
  const double tot = bsum(s, red);
  if (threadIdx.x == 0) *S = -tot;
}

__global__ void one_by_one_kernel(const z64* M, double* d) { d[0] = M[0].re; }



cudaError_t hermitian_entropy(cudaStream_t st, z64* M, int m, z64* vb, z64* wb, z64* pbuf, double* partial_unused,
                              double* d, double* e, double* lam, double* S, int* nlaunch, int cross) {
  (void)partial_unused;
  int launches = 0;
  if (m <= 0) return cudaSuccess;
  if (m == 1) {
    one_by_one_kernel<<<1, 1, 0, st>>>(M, d);
    ++launches;
  } else if (m <= 256) {
    tridiag_small_kernel<<<1, 1024, 0, st>>>(M, m, vb, wb, d, e);
    ++launches;
  } else {
    static_assert(HT * (HT + 1) * sizeof(z64) <= 48 * 1024, "hemv tile must not need a shared-memory opt-in");
    // pbuf layout: [tau][prow: nb*m][pcol: nb*m][p: m][sdot: m/256 + 1][v, w of the other parity: 2m]
    const int nbm = FM_CEIL_DIV(m, HT);
    z64* tau = pbuf;
    z64* prow = pbuf + 1;
    z64* pcol = prow + (int64_t)nbm * m;
    z64* p = pcol + (int64_t)nbm * m;
    z64* sdot = p + m;
    z64* vb2 = sdot + m / 256 + 1;
    z64* wb2 = vb2 + m;
    // column k uses (vb, wb) for even k, (vb2, wb2) for odd k; the other pair
    // holds the rank-2 update column k - 1 left pending
    for (int k = 0; k + 1 < m; ++k) {
      const int n = m - k - 1;
      const int nb = FM_CEIL_DIV(n, HT);
      z64* vc = (k & 1) ? vb2 : vb;
      z64* wc = (k & 1) ? wb2 : wb;
      const z64* vp = k == 0 ? nullptr : ((k & 1) ? vb : vb2);
      const z64* wp = k == 0 ? nullptr : ((k & 1) ? wb : wb2);
      hh_reflector_kernel<<<1, 256, 0, st>>>(M, m, k, vp, wp, vc, d, e, tau);
      hemv_lower_kernel<<<nb * (nb + 1) / 2, 256, HT * (HT + 1) * sizeof(z64), st>>>(M, m, k, vp, wp, vc, prow,
                                                                                    pcol);
      const int rb = FM_CEIL_DIV(n, 256);
      hemv_reduce_kernel<<<rb, 256, 0, st>>>(m, k, prow, pcol, vc, p, sdot);
      hh_w_kernel<<<FM_CEIL_DIV(n, 256), 256, 0, st>>>(m, k, p, sdot, rb, vc, wc, tau);
      launches += 4;
    }
    const int kl = m - 2;                      // the last column's pending update
    last_diag_kernel<<<1, 1, 0, st>>>(M, m, (kl & 1) ? vb2 : vb, (kl & 1) ? wb2 : wb, d);
    ++launches;
  }
  // measured: at m = 512 multisection brought the whole entropy from 34 ms to 21 ms; at
  // m = 8192 (GPU already full) its 32 Sturm sequences per round cost more than they save
  if (m <= 2048) bisect_kernel<<<FM_CEIL_DIV(m, 4), 128, 0, st>>>(d, e, m, lam);
  else bisect_thread_kernel<<<FM_CEIL_DIV(m, 64), 64, 0, st>>>(d, e, m, lam);
  entropy_sum_kernel<<<1, 1024, 0, st>>>(lam, m, S, cross);
  launches += 2;
  if (nlaunch) *nlaunch += launches;
  return cudaGetLastError();
}

}  // namespace fm
