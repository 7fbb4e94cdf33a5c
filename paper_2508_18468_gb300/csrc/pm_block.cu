// Projective measurements of one step as a block (Eqs. (A1), (A2)).
//
// The sites measured in a step are known before any outcome (the selection
// draws do not depend on the state), and every update is rank one,
// U <- U + a b^dag.  So instead of one pass over U per event, the sequence is
// run on the K selected sites alone and U is updated once:
//
//   W = U0[S, :] (K x N),   P = U0 W^dag = C0[:, S] (L x K),   C = P[S, :] (K x K).
//   With t_l the coefficient vectors of b_l = W^dag t_l, the state before event
//   i has rows U_i[S, :] = (1 + A_S T_B^dag) W, A_S = C T_A + T_E, and event i
//   (site j_i, draw u_i) is
//     rho   = e_i + T_B conj(A_S[i, :])              x_i = rho^dag W
//     y     = C rho,  p = Re rho^dag y               (p = C_jj of the current state)
//     outcome = u_i < p;  t_i = rho / sqrt(p),  ys = y / sqrt(p) = C t_i
//     g     = T_B^dag ys                             (g_l = b_l^dag b_i)
//     tau   = t_i + T_A g,   eps = T_E g,   C tau = ys + (C T_A) g
//     click:    T_A[:, i] = -tau,      T_E[:, i] = -eps + e_i
//     no click: T_A[:, i] = c tau,     T_E[:, i] = c eps - sqrt(p / (1 - p)) e_i,
//               c = 1 / sqrt(1 - p) - 1
//   and at the end  U = U0 + A B^dag  with  A = P T_A + E_S T_E,  B^dag = T_B^dag W.
// T_A, T_B, T_E are upper triangular.  C T_A and C T_B are kept as matrices of
// their own, so an event costs O(K i) instead of a pass over U.
//
// Here: the sequential part on K x K complex64 matrices, batched over the
// trajectories (one launch per phase of an event); the three large products
// (P, A, and the update) run on the tensor cores (mixed.cu).  Matrices are
// stored with leading dimension Kc (the capacity): row-major ones as
// X[r * Kc + l], column-major ones as X[r + l * Kc].
#include <algorithm>

#include "kernels.h"

namespace fm {

namespace {

FM_DEVFN c32 warp_csum(c32 v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    v.re += __shfl_xor_sync(0xffffffffu, v.re, o);
    v.im += __shfl_xor_sync(0xffffffffu, v.im, o);
  }
  return v;
}

FM_DEVFN void cfmaf(c32& acc, c32 a, c32 b) {
  acc.re = fmaf(a.re, b.re, acc.re);
  acc.re = fmaf(-a.im, b.im, acc.re);
  acc.im = fmaf(a.re, b.im, acc.im);
  acc.im = fmaf(a.im, b.re, acc.im);
}

}  // namespace

// ------------------------------------------------------------------ setup
// pos[b][i] = r if site i is the r-th selected site of trajectory b, else -1
__global__ void pmb_pos_kernel(const int* list, const int* count, int L, int* pos) {
  const int b = blockIdx.y;
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r < count[b]) pos[(int64_t)b * L + list[(int64_t)b * L + r]] = r;
}

// Rows of the B operand of P (2K x 2N fp16 planes, trajectory b): row l < K is
// row j_l of U~ (interleaved re, im), row K + l the same row with each pair
// (re, im) turned into (-im, re) (so that the product gives Im P); zero rows
// past the trajectory's count.
__global__ void pmb_gather_w_kernel(const __half* __restrict__ urm_h, const __half* __restrict__ urm_l, int L,
                                    int N, const int* list, const int* count, int K, __half* wt_h,
                                    __half* wt_l) {
  const int b = blockIdx.z;
  const int row = blockIdx.y;                 // 0 .. 2K-1 of trajectory b (planes rows b 2K + row)
  const int l = row < K ? row : row - K;
  const bool ok = l < count[b];
  const int64_t src = ok ? ((int64_t)b * L + list[(int64_t)b * L + l]) * 2 * N : 0;
  const __half zero = __float2half_rn(0.0f);
  for (int n = blockIdx.x * blockDim.x + threadIdx.x; n < N; n += gridDim.x * blockDim.x) {
    __half h0 = zero, h1 = zero, l0 = zero, l1 = zero;
    if (ok) {
      h0 = urm_h[src + 2 * n]; h1 = urm_h[src + 2 * n + 1];
      l0 = urm_l[src + 2 * n]; l1 = urm_l[src + 2 * n + 1];
      if (row >= K) {
        const __half th = h0, tl = l0;
        h0 = __hneg(h1); l0 = __hneg(l1);
        h1 = th; l1 = tl;
      }
    }
    const int64_t o = ((int64_t)b * 2 * K + row) * 2 * N + 2 * n;
    wt_h[o] = h0; wt_h[o + 1] = h1;
    wt_l[o] = l0; wt_l[o + 1] = l1;
  }
}

// C_b[r + c Kc] = P[j_r, c] from the row-major real form D'_b (L x 2K:
// [Re P | Im P]), made exactly Hermitian; zero outside count x count.
__global__ void pmb_gather_c_kernel(const float* Dp, int64_t sD, int L, int K, int Kc, const int* list,
                                    const int* count, c32* C, int64_t sC) {
  const int b = blockIdx.z;
  const int r = blockIdx.y, c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= K) return;
  const int n = count[b];
  c32 v = cmk(0.0f, 0.0f);
  if (r < n && c < n) {
    const float* D = Dp + b * sD;
    const int jr = list[(int64_t)b * L + r], jc = list[(int64_t)b * L + c];
    const c32 a = cmk(D[(int64_t)jr * 2 * K + c], D[(int64_t)jr * 2 * K + K + c]);
    const c32 t = cmk(D[(int64_t)jc * 2 * K + r], D[(int64_t)jc * 2 * K + K + r]);   // P[j_c, r]
    v = cmk(0.5f * (a.re + t.re), 0.5f * (a.im - t.im));
  }
  C[b * sC + r + (int64_t)c * Kc] = v;
}

// ------------------------------------------------------------------ one event (i), all trajectories
// E1: rho = e_i + T_B conj(a), y = C[:, i] + (C T_B) conj(a), a = row i of (C T_A + T_E);
// warp per row r.
__global__ void pmb_rho_kernel(int i, int Kc, const int* count, const c32* C, const c32* TBr, const c32* CTB,
                               const c32* CTA, const c32* TE, int64_t sM, c32* rho, c32* y) {
  const int b = blockIdx.z;
  const int n = count[b];
  if (i >= n) return;
  const int r = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5), lane = threadIdx.x & 31;
  if (r >= n) return;
  const int64_t o = b * sM;
  const c32* arow_a = CTA + o + (int64_t)i * Kc;
  const c32* arow_e = TE + o + (int64_t)i * Kc;
  c32 sr = cmk(0.0f, 0.0f), sy = cmk(0.0f, 0.0f);
  for (int l = lane; l < i; l += 32) {
    const c32 a = cconj(cadd(arow_a[l], arow_e[l]));
    if (l >= r) cfmaf(sr, TBr[o + (int64_t)r * Kc + l], a);
    cfmaf(sy, CTB[o + (int64_t)r * Kc + l], a);
  }
  sr = warp_csum(sr);
  sy = warp_csum(sy);
  if (lane == 0) {
    if (r == i) sr.re += 1.0f;
    rho[b * Kc + r] = r <= i ? sr : cmk(0.0f, 0.0f);
    y[b * Kc + r] = cadd(sy, C[o + r + (int64_t)i * Kc]);
  }
}

// E3: Born weight, outcome, t_i and C t_i; one CTA per trajectory.
__global__ void __launch_bounds__(256) pmb_decide_kernel(int i, int Kc, int L, const int* count, const int* list,
                                                         const double* ulist, const int64_t* step, const c32* rho,
                                                         const c32* y, c32* TBr, c32* TBc, c32* CTB, int64_t sM,
                                                         c32* ys, PmbEvent* ev, fm_event* log,
                                                         unsigned long long* log_count, int log_capacity) {
  const int b = blockIdx.x;
  const int n = count[b];
  __shared__ double red[33];
  __shared__ double sp_sh;
  __shared__ int act_sh;
  if (i >= n) {
    if (threadIdx.x == 0) ev[b].active = 0;
    return;
  }
  double part = 0.0;
  for (int r = threadIdx.x; r <= i; r += blockDim.x) {
    const c32 a = rho[b * Kc + r], c = y[b * Kc + r];
    part += (double)a.re * c.re + (double)a.im * c.im;
  }
  // fixed-order block sum
  for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = part;
  __syncthreads();
  if (threadIdx.x == 0) {
    double p = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) p += red[w];
    p = fmin(fmax(p, 0.0), 1.0);
    const int j = list[(int64_t)b * L + i];
    const double u = ulist[(int64_t)b * L + i];
    PmbEvent e;
    e.outcome = (u < p) ? 1 : 0;
    e.active = (p >= 1e-300) ? 1 : 0;
    e.sp = sqrt(p);
    e.c = e.outcome ? -1.0 : 1.0 / sqrt(1.0 - p) - 1.0;
    e.dsel = e.outcome ? 1.0 : -e.sp / sqrt(1.0 - p);
    ev[b] = e;
    sp_sh = e.sp;
    act_sh = e.active;
    if (log && log_capacity > 0) {
      const unsigned long long slot = atomicAdd(log_count, 1ull);
      if (slot < (unsigned long long)log_capacity) {
        fm_event le;
        le.step = step[b]; le.traj = b; le.site = j; le.u = u; le.p = p; le.outcome = e.outcome; le.pad = 0;
        log[slot] = le;
      }
    }
  }
  __syncthreads();
  if (!act_sh) return;
  const float inv = (float)(1.0 / sp_sh);
  const int64_t o = b * sM;
  for (int r = threadIdx.x; r < n; r += blockDim.x) {
    const c32 yr = cscale(y[b * Kc + r], inv);
    ys[b * Kc + r] = yr;
    CTB[o + (int64_t)r * Kc + i] = yr;
    if (r <= i) {
      const c32 t = cscale(rho[b * Kc + r], inv);
      TBr[o + (int64_t)r * Kc + i] = t;
      TBc[o + r + (int64_t)i * Kc] = t;
    }
  }
}

// E4: g_l = sum_{r <= l} conj(T_B[r, l]) ys_r for l < i; warp per column.
__global__ void pmb_g_kernel(int i, int Kc, const int* count, const PmbEvent* ev, const c32* TBc, int64_t sM,
                             const c32* ys, c32* g) {
  const int b = blockIdx.z;
  if (i >= count[b] || !ev[b].active) return;
  const int l = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5), lane = threadIdx.x & 31;
  if (l >= i) return;
  const c32* col = TBc + b * sM + (int64_t)l * Kc;
  c32 s = cmk(0.0f, 0.0f);
  for (int r = lane; r <= l; r += 32) cfmaf(s, cconj(col[r]), ys[b * Kc + r]);
  s = warp_csum(s);
  if (lane == 0) g[b * Kc + l] = s;
}

// E5: column i of T_A, C T_A and T_E; warp per row.
__global__ void pmb_update_kernel(int i, int Kc, const int* count, const PmbEvent* ev, c32* TA, c32* CTA, c32* TE,
                                  const c32* TBr, int64_t sM, const c32* ys, const c32* g) {
  const int b = blockIdx.z;
  const int n = count[b];
  if (i >= n || !ev[b].active) return;
  const int r = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5), lane = threadIdx.x & 31;
  if (r >= n) return;
  const int64_t o = b * sM + (int64_t)r * Kc;
  c32 tau = cmk(0.0f, 0.0f), ctau = cmk(0.0f, 0.0f), eps = cmk(0.0f, 0.0f);
  for (int l = lane; l < i; l += 32) {
    const c32 gl = g[b * Kc + l];
    if (l >= r) {
      cfmaf(tau, TA[o + l], gl);
      cfmaf(eps, TE[o + l], gl);
    }
    cfmaf(ctau, CTA[o + l], gl);
  }
  tau = warp_csum(tau);
  ctau = warp_csum(ctau);
  eps = warp_csum(eps);
  if (lane == 0) {
    const PmbEvent e = ev[b];
    const float c = (float)e.c;
    if (r <= i) {
      tau = cadd(tau, TBr[o + i]);
      TA[o + i] = cscale(tau, c);
      c32 te = cscale(eps, c);
      if (r == i) te.re += (float)e.dsel;
      TE[o + i] = te;
    }
    ctau = cadd(ctau, ys[b * Kc + r]);
    CTA[o + i] = cscale(ctau, c);
  }
}

// ------------------------------------------------------------------ all events of a step, one launch
// Every event i < count[b] of trajectory b in one CTA of 512 threads (trajectories are
// independent; the events of one are sequential), in phases separated by CTA barriers:
//   E1  rho = e_i + T_B conj(a), y = C[:, i] + (C T_B) conj(a), a = row i of (C T_A + T_E)
//       (a warp per row, lane-strided terms);
//   E3  the Born weight p = Re rho^dag y (the first 8 warps, fixed order), the outcome, the
//       event log, then t_i = rho / sqrt(p) into T_B and ys = y / sqrt(p) = C t_i into C T_B;
//   E4  g_l = sum_{r <= l} conj(T_B[r, l]) ys_r for l < i (a warp per column);
//   E5  column i of T_A, C T_A and T_E (a warp per row).
// One launch per step instead of four per event: the choice when many trajectories keep the
// SMs busy or the events are few (pmb_events_fit); the per-phase kernels above spread one
// event's rows over the whole GPU, which long event lists of a few trajectories need.
constexpr int kEvThreads = 512;          // two CTAs per SM (46 registers a thread)

__global__ void __launch_bounds__(kEvThreads) pmb_events_kernel(int Kc, int L, const int* count, const int* list,
                                                                 const double* ulist, const int64_t* step,
                                                                 PmbMats m, fm_event* log,
                                                                 unsigned long long* log_count, int log_capacity) {
  const int b = blockIdx.x;
  const int n = count[b];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarps = kEvThreads >> 5;
  const int64_t o = b * m.sM;
  c32* rho = m.rho + b * Kc;
  c32* y = m.y + b * Kc;
  c32* ys = m.ys + b * Kc;
  c32* g = m.g + b * Kc;
  __shared__ double red[33];
  __shared__ double sp_sh, c_sh, dsel_sh;
  __shared__ int act_sh;
  for (int i = 0; i < n; ++i) {
    // E1: rho, y (warp per row)
    const c32* arow_a = m.CTA + o + (int64_t)i * Kc;
    const c32* arow_e = m.TE + o + (int64_t)i * Kc;
    for (int r = warp; r < n; r += nwarps) {
      c32 sr = cmk(0.0f, 0.0f), sy = cmk(0.0f, 0.0f);
      for (int l = lane; l < i; l += 32) {
        const c32 a = cconj(cadd(arow_a[l], arow_e[l]));
        if (l >= r) cfmaf(sr, m.TBr[o + (int64_t)r * Kc + l], a);
        cfmaf(sy, m.CTB[o + (int64_t)r * Kc + l], a);
      }
      sr = warp_csum(sr);
      sy = warp_csum(sy);
      if (lane == 0) {
        if (r == i) sr.re += 1.0f;
        rho[r] = r <= i ? sr : cmk(0.0f, 0.0f);
        y[r] = cadd(sy, m.C[o + r + (int64_t)i * Kc]);
      }
    }
    __syncthreads();
    // E3: Born weight by the first 256 threads (the per-phase kernel's order), outcome
    if (tid < 256) {
      double part = 0.0;
      for (int r = tid; r <= i; r += 256) {
        const c32 a = rho[r], c = y[r];
        part += (double)a.re * c.re + (double)a.im * c.im;
      }
      for (int w = 16; w > 0; w >>= 1) part += __shfl_xor_sync(0xffffffffu, part, w);
      if (lane == 0) red[warp] = part;
    }
    __syncthreads();
    if (tid == 0) {
      double p = 0.0;
      for (int w = 0; w < 8; ++w) p += red[w];
      p = fmin(fmax(p, 0.0), 1.0);
      const int j = list[(int64_t)b * L + i];
      const double u = ulist[(int64_t)b * L + i];
      PmbEvent e;
      e.outcome = (u < p) ? 1 : 0;
      e.active = (p >= 1e-300) ? 1 : 0;
      e.sp = sqrt(p);
      e.c = e.outcome ? -1.0 : 1.0 / sqrt(1.0 - p) - 1.0;
      e.dsel = e.outcome ? 1.0 : -e.sp / sqrt(1.0 - p);
      m.ev[b] = e;
      sp_sh = e.sp;
      c_sh = e.c;
      dsel_sh = e.dsel;
      act_sh = e.active;
      if (log && log_capacity > 0) {
        const unsigned long long slot = atomicAdd(log_count, 1ull);
        if (slot < (unsigned long long)log_capacity) {
          fm_event le;
          le.step = step[b]; le.traj = b; le.site = j; le.u = u; le.p = p; le.outcome = e.outcome; le.pad = 0;
          log[slot] = le;
        }
      }
    }
    __syncthreads();
    if (!act_sh) continue;                         // no weight on the site: nothing changes
    const float inv = (float)(1.0 / sp_sh);
    for (int r = tid; r < n; r += kEvThreads) {
      const c32 yr = cscale(y[r], inv);
      ys[r] = yr;
      m.CTB[o + (int64_t)r * Kc + i] = yr;
      if (r <= i) {
        const c32 t = cscale(rho[r], inv);
        m.TBr[o + (int64_t)r * Kc + i] = t;
        m.TBc[o + r + (int64_t)i * Kc] = t;
      }
    }
    __syncthreads();
    // E4: g (warp per column l < i)
    for (int l = warp; l < i; l += nwarps) {
      const c32* col = m.TBc + o + (int64_t)l * Kc;
      c32 sg = cmk(0.0f, 0.0f);
      for (int r = lane; r <= l; r += 32) cfmaf(sg, cconj(col[r]), ys[r]);
      sg = warp_csum(sg);
      if (lane == 0) g[l] = sg;
    }
    __syncthreads();
    // E5: column i of T_A, C T_A, T_E (warp per row)
    const float c = (float)c_sh;
    for (int r = warp; r < n; r += nwarps) {
      const int64_t orow = o + (int64_t)r * Kc;
      c32 tau = cmk(0.0f, 0.0f), ctau = cmk(0.0f, 0.0f), eps = cmk(0.0f, 0.0f);
      for (int l = lane; l < i; l += 32) {
        const c32 gl = g[l];
        if (l >= r) {
          cfmaf(tau, m.TA[orow + l], gl);
          cfmaf(eps, m.TE[orow + l], gl);
        }
        cfmaf(ctau, m.CTA[orow + l], gl);
      }
      tau = warp_csum(tau);
      ctau = warp_csum(ctau);
      eps = warp_csum(eps);
      if (lane == 0) {
        if (r <= i) {
          tau = cadd(tau, m.TBr[orow + i]);
          m.TA[orow + i] = cscale(tau, c);
          c32 te = cscale(eps, c);
          if (r == i) te.re += (float)dsel_sh;
          m.TE[orow + i] = te;
        }
        ctau = cadd(ctau, ys[r]);
        m.CTA[orow + i] = cscale(ctau, c);
      }
    }
    __syncthreads();
  }
}

bool pmb_events_fit(int B, int kmax) { return B >= 64 || kmax <= 128; }

cudaError_t pmb_events(cudaStream_t st, int Kc, int L, int B, const int* count, const int* list, const double* ulist,
                       const int64_t* step, const PmbMats& m, fm_event* log, unsigned long long* log_count,
                       int log_capacity) {
  pmb_events_kernel<<<B, kEvThreads, 0, st>>>(Kc, L, count, list, ulist, step, m, log, log_count, log_capacity);
  return cudaGetLastError();
}

// ------------------------------------------------------------------ operands of the final products
// K-major planes of M^T, M = [[Re T_A, Im T_A], [-Im T_A, Re T_A]] (2K x 2K), trajectory b
__global__ void pmb_ttilde_kernel(const c32* TA, int64_t sM, int Kc, int K, __half* th, __half* tl) {
  const int b = blockIdx.z;
  const int cp = blockIdx.y;                            // row of the plane = column c' of M
  th += (int64_t)b * 4 * K * K;
  tl += (int64_t)b * 4 * K * K;
  for (int kp = blockIdx.x * blockDim.x + threadIdx.x; kp < 2 * K; kp += gridDim.x * blockDim.x) {
    const int c = cp < K ? cp : cp - K, k = kp < K ? kp : kp - K;
    const c32 t = TA[b * sM + (int64_t)k * Kc + c];
    float v;
    if (kp < K) v = cp < K ? t.re : t.im;
    else v = cp < K ? -t.im : t.re;
    const __half h = __float2half_rn(v);
    th[(int64_t)cp * 2 * K + kp] = h;
    tl[(int64_t)cp * 2 * K + kp] = __float2half_rn((v - __half2float(h)) * 2048.0f);
  }
}

// split-fp16 planes of a float array
__global__ void pmb_split_kernel(const float* x, int64_t n, __half* h, __half* l) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const float v = x[i];
    const __half hh = __float2half_rn(v);
    h[i] = hh;
    l[i] = __float2half_rn((v - __half2float(hh)) * 2048.0f);
  }
}

// K-major planes of the real embedding of A = P T_A + E_S T_E (2L x 2K): row i
// [Re A_i, -Im A_i], row L + i [Im A_i, Re A_i]; Ap = row-major [Re(P T_A) | Im(P T_A)].
__global__ void pmb_atilde_kernel(const float* Ap, int L, int K, int Kc, const int* pos, const c32* TE,
                                  int64_t sM, __half* ah, __half* al) {
  const int b = blockIdx.z;
  const int i = blockIdx.y;
  Ap += (int64_t)b * L * 2 * K;
  ah += (int64_t)b * 2 * L * 2 * K;
  al += (int64_t)b * 2 * L * 2 * K;
  const int r = pos[(int64_t)b * L + i];
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < K; c += gridDim.x * blockDim.x) {
    float re = Ap[(int64_t)i * 2 * K + c], im = Ap[(int64_t)i * 2 * K + K + c];
    if (r >= 0) {
      const c32 t = TE[b * sM + (int64_t)r * Kc + c];
      re += t.re;
      im += t.im;
    }
    const float vals[4] = {re, -im, im, re};
    const int64_t offs[4] = {(int64_t)i * 2 * K + c, (int64_t)i * 2 * K + K + c, (int64_t)(L + i) * 2 * K + c,
                             (int64_t)(L + i) * 2 * K + K + c};
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const __half h = __float2half_rn(vals[q]);
      ah[offs[q]] = h;
      al[offs[q]] = __float2half_rn((vals[q] - __half2float(h)) * 2048.0f);
    }
  }
}

// Wc_b[r + n Kc] = U0[j_r, n] (complex64) from the float state V_b; zero rows past the count
__global__ void pmb_gather_wc_kernel(const float* V, int L, int N, int K, int Kc, const int* list, const int* count,
                                     c32* Wc, int64_t sW) {
  const int b = blockIdx.z;
  const int r = blockIdx.y;
  const bool ok = r < count[b];
  const int j = ok ? list[(int64_t)b * L + r] : 0;
  const float* Vb = V + (int64_t)b * 2 * L * N;
  for (int n = blockIdx.x * blockDim.x + threadIdx.x; n < N; n += gridDim.x * blockDim.x)
    Wc[b * sW + r + (int64_t)n * Kc] =
        ok ? cmk(Vb[j + (int64_t)n * 2 * L], Vb[L + j + (int64_t)n * 2 * L]) : cmk(0.0f, 0.0f);
}

// K-major planes of X~ (N x 2K): row n = [Re X[:, n], Im X[:, n]], X = T_B^dag W (K x N, ld Kc)
__global__ void pmb_xtilde_kernel(const c32* X, int64_t sX, int K, int Kc, int N, __half* xh, __half* xl) {
  const int b = blockIdx.z;
  const int n = blockIdx.y;
  xh += (int64_t)b * N * 2 * K;
  xl += (int64_t)b * N * 2 * K;
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < K; k += gridDim.x * blockDim.x) {
    const c32 x = X[b * sX + k + (int64_t)n * Kc];
    const float vals[2] = {x.re, x.im};
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      const int64_t o = (int64_t)n * 2 * K + q * K + k;
      const __half h = __float2half_rn(vals[q]);
      xh[o] = h;
      xl[o] = __float2half_rn((vals[q] - __half2float(h)) * 2048.0f);
    }
  }
}

// ------------------------------------------------------------------ launchers
int pmb_capacity(int L) {
  const int c = ((L / 8 + 64 + 63) / 64) * 64;
  return std::min(c, ((L + 63) / 64) * 64);
}

cudaError_t pmb_setup(cudaStream_t st, const int* list, const int* count, int L, int B, int nmax, int* pos) {
  cudaError_t e = cudaMemsetAsync(pos, 0xff, sizeof(int) * (size_t)B * L, st);   // -1
  if (e) return e;
  if (nmax > 0) pmb_pos_kernel<<<dim3(FM_CEIL_DIV(nmax, 256), B), 256, 0, st>>>(list, count, L, pos);
  return cudaGetLastError();
}

cudaError_t pmb_gather_w(cudaStream_t st, const __half* urm_h, const __half* urm_l, int L, int N, const int* list,
                         const int* count, int B, int K, __half* wt_h, __half* wt_l) {
  pmb_gather_w_kernel<<<dim3(FM_CEIL_DIV(N, 256), 2 * K, B), 256, 0, st>>>(urm_h, urm_l, L, N, list, count, K, wt_h,
                                                                             wt_l);
  return cudaGetLastError();
}

cudaError_t pmb_gather_c(cudaStream_t st, const float* Dp, int64_t sD, int L, int K, int B, const int* list,
                         const int* count, const PmbMats& m) {
  pmb_gather_c_kernel<<<dim3(FM_CEIL_DIV(K, 256), K, B), 256, 0, st>>>(Dp, sD, L, K, m.Kc, list, count, m.C, m.sM);
  return cudaGetLastError();
}

cudaError_t pmb_ttilde(cudaStream_t st, const PmbMats& m, int K, int B, __half* th, __half* tl) {
  pmb_ttilde_kernel<<<dim3(FM_CEIL_DIV(2 * K, 256), 2 * K, B), 256, 0, st>>>(m.TA, m.sM, m.Kc, K, th, tl);
  return cudaGetLastError();
}

cudaError_t pmb_split(cudaStream_t st, const float* x, int64_t n, __half* h, __half* l) {
  const int64_t blocks = std::min<int64_t>(FM_CEIL_DIV(n, 256), 152 * 16);
  pmb_split_kernel<<<(unsigned)blocks, 256, 0, st>>>(x, n, h, l);
  return cudaGetLastError();
}

cudaError_t pmb_atilde(cudaStream_t st, const float* Ap, int L, int K, int B, const int* pos, const PmbMats& m,
                       __half* ah, __half* al) {
  pmb_atilde_kernel<<<dim3(FM_CEIL_DIV(K, 256), L, B), 256, 0, st>>>(Ap, L, K, m.Kc, pos, m.TE, m.sM, ah, al);
  return cudaGetLastError();
}

cudaError_t pmb_gather_wc(cudaStream_t st, const float* V, int L, int N, int K, int B, const int* list,
                          const int* count, const PmbMats& m) {
  pmb_gather_wc_kernel<<<dim3(FM_CEIL_DIV(N, 256), K, B), 256, 0, st>>>(V, L, N, K, m.Kc, list, count, m.Wc, m.sW);
  return cudaGetLastError();
}

cudaError_t pmb_xtilde(cudaStream_t st, const PmbMats& m, int K, int B, int N, __half* xh, __half* xl) {
  pmb_xtilde_kernel<<<dim3(FM_CEIL_DIV(K, 256), N, B), 256, 0, st>>>(m.X, m.sW, K, m.Kc, N, xh, xl);
  return cudaGetLastError();
}

cudaError_t pmb_event(cudaStream_t st, int i, int Kc, int L, int B, const int* count, const int* list,
                      const double* ulist, const int64_t* step, const PmbMats& m, fm_event* log,
                      unsigned long long* log_count, int log_capacity, int nmax) {
  const int warps = 8;
  const dim3 rows(FM_CEIL_DIV(nmax, warps), 1, B);
  pmb_rho_kernel<<<rows, 32 * warps, 0, st>>>(i, Kc, count, m.C, m.TBr, m.CTB, m.CTA, m.TE, m.sM, m.rho, m.y);
  pmb_decide_kernel<<<B, 256, 0, st>>>(i, Kc, L, count, list, ulist, step, m.rho, m.y, m.TBr, m.TBc, m.CTB, m.sM,
                                       m.ys, m.ev, log, log_count, log_capacity);
  if (i > 0) {
    const dim3 cols(FM_CEIL_DIV(i, warps), 1, B);
    pmb_g_kernel<<<cols, 32 * warps, 0, st>>>(i, Kc, count, m.ev, m.TBc, m.sM, m.ys, m.g);
  }
  pmb_update_kernel<<<rows, 32 * warps, 0, st>>>(i, Kc, count, m.ev, m.TA, m.CTA, m.TE, m.TBr, m.sM, m.ys, m.g);
  return cudaGetLastError();
}

}  // namespace fm
