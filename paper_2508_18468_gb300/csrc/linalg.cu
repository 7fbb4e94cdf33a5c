// CUDA-core kernels of the fm library: the FP64 (and float) complex GEMM used by
// the all-FP64 path, occupations and the homodyne weight, the projective
// measurement, Cholesky pieces, and layout conversions.
#include <float.h>

#include <algorithm>
#include <vector>
#include <math.h>

#include "kernels.h"

namespace fm {

// =================================================================== complex GEMM
// 64 x 64 output tile per CTA, K-step 16, 256 threads; thread (tx, ty) owns
// rows m0 + tx + 16 i and columns n0 + ty + 16 j (i, j < 4).
template <typename T>
__global__ void __launch_bounds__(256) zgemm_kernel(int M, int N, int K, int opA, int opB, cplx<T> alpha,
                                                    const cplx<T>* __restrict__ A, int64_t lda, int64_t sA,
                                                    const cplx<T>* __restrict__ B, int64_t ldb, int64_t sB,
                                                    cplx<T> beta, cplx<T>* __restrict__ C, int64_t ldc,
                                                    int64_t sC, int flags) {
  constexpr int BM = 64, BN = 64, BK = 16;
  __shared__ cplx<T> As[BK][BM];
  __shared__ cplx<T> Bs[BK][BN];
  const int64_t bz = blockIdx.z;
  A += bz * sA;
  B += bz * sB;
  C += bz * sC;
  const int m0 = blockIdx.x * BM, n0 = blockIdx.y * BN;
  if ((flags & GEMM_UPPER_ONLY) && m0 > n0 + BN - 1) return;
  if ((flags & GEMM_LOWER_ONLY) && n0 > m0 + BM - 1) return;
  int kbeg = 0, kend = K;
  if (flags & GEMM_TRI_A_UPPER) kbeg = (m0 / BK) * BK;
  if (flags & GEMM_TRI_B_UPPER) kend = min(K, n0 + BN);
  const int t = threadIdx.x, tx = t % 16, ty = t / 16;
  cplx<T> acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = cmk<T>(0, 0);

  for (int k0 = kbeg; k0 < kend; k0 += BK) {
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      int mm, kk;
      if (opA == OP_N) { mm = t % 64; kk = t / 64 + 4 * r; }
      else { kk = t % 16; mm = t / 16 + 16 * r; }
      const int m = m0 + mm, k = k0 + kk;
      cplx<T> v = cmk<T>(0, 0);
      if (m < M && k < K) {
        v = (opA == OP_N) ? A[m + (int64_t)k * lda] : A[k + (int64_t)m * lda];
        if (opA == OP_C) v.im = -v.im;
      }
      As[kk][mm] = v;
    }
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      int kk, nn;
      if (opB == OP_N) { kk = t % 16; nn = t / 16 + 16 * r; }
      else { nn = t % 64; kk = t / 64 + 4 * r; }
      const int n = n0 + nn, k = k0 + kk;
      cplx<T> v = cmk<T>(0, 0);
      if (n < N && k < K) {
        v = (opB == OP_N) ? B[k + (int64_t)n * ldb] : B[n + (int64_t)k * ldb];
        if (opB == OP_C) v.im = -v.im;
      }
      Bs[kk][nn] = v;
    }
    __syncthreads();
#pragma unroll 4
    for (int kk = 0; kk < BK; ++kk) {
      cplx<T> a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[kk][tx + 16 * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = Bs[kk][ty + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) cfma(acc[i][j], a[i], b[j]);
    }
    __syncthreads();
  }
  const bool use_beta = (beta.re != (T)0 || beta.im != (T)0);
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int m = m0 + tx + 16 * i, n = n0 + ty + 16 * j;
      if (m < M && n < N) {
        cplx<T> r = cmul(alpha, acc[i][j]);
        cplx<T>* c = C + m + (int64_t)n * ldc;
        if (use_beta) r = cadd(r, cmul(beta, *c));
        *c = r;
      }
    }
}

template <typename T>
cudaError_t zgemm(cudaStream_t st, int M, int N, int K, int opA, int opB, cplx<T> alpha, const cplx<T>* A,
                  int64_t lda, int64_t sA, const cplx<T>* B, int64_t ldb, int64_t sB, cplx<T> beta, cplx<T>* C,
                  int64_t ldc, int64_t sC, int batch, int flags) {
  if (M <= 0 || N <= 0 || batch <= 0) return cudaSuccess;
  dim3 grid(FM_CEIL_DIV(M, 64), FM_CEIL_DIV(N, 64), batch);
  if (grid.y > 65535 || grid.z > 65535) return cudaErrorInvalidConfiguration;
  zgemm_kernel<T><<<grid, 256, 0, st>>>(M, N, K, opA, opB, alpha, A, lda, sA, B, ldb, sB, beta, C, ldc, sC, flags);
  return cudaGetLastError();
}
template cudaError_t zgemm<double>(cudaStream_t, int, int, int, int, int, z64, const z64*, int64_t, int64_t,
                                   const z64*, int64_t, int64_t, z64, z64*, int64_t, int64_t, int, int);
template cudaError_t zgemm<float>(cudaStream_t, int, int, int, int, int, c32, const c32*, int64_t, int64_t,
                                  const c32*, int64_t, int64_t, c32, c32*, int64_t, int64_t, int, int);

// =================================================================== occupations
// grid (ceil(L/32), nchunks, batch), block (32, 8): warp y walks columns
// k = chunk_start + y, +8, ... of 32 consecutive rows; fixed-order reductions.
__global__ void rownorm_partials_z_kernel(const z64* __restrict__ U, int L, int N, double* partial, int nchunks) {
  const int64_t b = blockIdx.z;
  const z64* Ub = U + b * L * (int64_t)N;
  const int i = blockIdx.x * 32 + threadIdx.x;
  const int per = FM_CEIL_DIV(N, nchunks);
  const int k0 = blockIdx.y * per, k1 = min(N, k0 + per);
  double acc = 0.0;
  if (i < L)
    for (int k = k0 + threadIdx.y; k < k1; k += 8) acc += cabs2(Ub[i + (int64_t)k * L]);
  __shared__ double red[8][33];
  red[threadIdx.y][threadIdx.x] = acc;
  __syncthreads();
  if (threadIdx.y == 0 && i < L) {
    double s = 0.0;
    for (int w = 0; w < 8; ++w) s += red[w][threadIdx.x];
    partial[(b * nchunks + blockIdx.y) * L + i] = s;
  }
}

__global__ void rownorm_partials_v_kernel(const float* __restrict__ V, int L, int N, double* partial, int nchunks) {
  const int64_t b = blockIdx.z;
  const float* Vb = V + b * 2 * (int64_t)L * N;
  const int i = blockIdx.x * 32 + threadIdx.x;
  const int per = FM_CEIL_DIV(N, nchunks);
  const int k0 = blockIdx.y * per, k1 = min(N, k0 + per);
  double acc = 0.0;
  if (i < L)
    for (int k = k0 + threadIdx.y; k < k1; k += 8) {
      const float re = Vb[i + (int64_t)k * 2 * L], im = Vb[L + i + (int64_t)k * 2 * L];
      acc += (double)re * re + (double)im * im;
    }
  __shared__ double red[8][33];
  red[threadIdx.y][threadIdx.x] = acc;
  __syncthreads();
  if (threadIdx.y == 0 && i < L) {
    double s = 0.0;
    for (int w = 0; w < 8; ++w) s += red[w][threadIdx.x];
    partial[(b * nchunks + blockIdx.y) * L + i] = s;
  }
}

int occupation_chunks(int L, int N, int batch) {
  int rows_blocks = FM_CEIL_DIV(L, 32) * batch;
  int c = FM_CEIL_DIV(4 * 152, rows_blocks);
  int cmax = max(1, N / 16);
  return max(1, min(c, min(cmax, 64)));
}

cudaError_t rownorm_partials_z(cudaStream_t st, const z64* U, int L, int N, int batch, double* partial,
                               int nchunks) {
  dim3 grid(FM_CEIL_DIV(L, 32), nchunks, batch);
  rownorm_partials_z_kernel<<<grid, dim3(32, 8), 0, st>>>(U, L, N, partial, nchunks);
  return cudaGetLastError();
}
cudaError_t rownorm_partials_v(cudaStream_t st, const float* V, int L, int N, int batch, double* partial,
                               int nchunks) {
  dim3 grid(FM_CEIL_DIV(L, 32), nchunks, batch);
  rownorm_partials_v_kernel<<<grid, dim3(32, 8), 0, st>>>(V, L, N, partial, nchunks);
  return cudaGetLastError();
}

__global__ void reduce_occupations_kernel(const double* __restrict__ partial, int nchunks, int L, int batch,
                                          double* n, double* w, const double* gamma, double dt,
                                          const uint64_t* traj, const int64_t* step, uint64_t seed) {
  const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (idx >= (int64_t)L * batch) return;
  const int b = (int)(idx / L), i = (int)(idx % L);
  double s = 0.0;
  for (int c = 0; c < nchunks; ++c) s += partial[((int64_t)b * nchunks + c) * L + i];
  n[idx] = s;
  if (w) {
    const double g = gamma[b];
    const double xi = fm_normal(fm_draw(seed, traj[b], step[b], i, FM_TAG_NOISE));
    const double m = sqrt(g * dt) * xi + (2.0 * s - 1.0) * g * dt;
    w[idx] = exp(m);
  }
}

cudaError_t reduce_occupations(cudaStream_t st, const double* partial, int nchunks, int L, int batch, double* n,
                               double* w, const double* gamma, double dt, const uint64_t* traj,
                               const int64_t* step, uint64_t seed) {
  int64_t tot = (int64_t)L * batch;
  reduce_occupations_kernel<<<(unsigned)FM_CEIL_DIV(tot, 256), 256, 0, st>>>(partial, nchunks, L, batch, n, w,
                                                                            gamma, dt, traj, step, seed);
  return cudaGetLastError();
}

__global__ void scale_rows_z_kernel(z64* U, int L, int N, int batch, const double* __restrict__ w) {
  const int64_t tot = (int64_t)L * N * batch;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < tot;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = idx % L;
    const int64_t b = idx / ((int64_t)L * N);
    const double s = w[b * L + i];
    z64 u = U[idx];
    U[idx] = cmk(u.re * s, u.im * s);
  }
}

cudaError_t scale_rows_z(cudaStream_t st, z64* U, int L, int N, int batch, const double* w) {
  scale_rows_z_kernel<<<152 * 8, 256, 0, st>>>(U, L, N, batch, w);
  return cudaGetLastError();
}

// h = fp16(x), l = fp16((x - h) * 2^11): x = h + l 2^-11 to ~2^-22 relative.
FM_DEVFN void split16(float x, __half& h, __half& l) {
  h = __float2half_rn(x);
  l = __float2half_rn((x - __half2float(h)) * 2048.0f);
}

// One thread scales 4 consecutive rows (of the 2L) of a run of columns: 16-byte loads
// and stores of V, 8-byte stores of each fp16 plane, the 4 weights reloaded only when
// the run enters the next trajectory; 4 columns' loads are issued before their stores.
// Grid (2L / 1024 row blocks, column runs); 2L is a multiple of 4 (L even).
__global__ void __launch_bounds__(256) scale_rows_v_kernel(float* __restrict__ V, __half* __restrict__ Vh,
                                                           __half* __restrict__ Vl, int L, int N, int64_t ncols,
                                                           int64_t run, const double* __restrict__ w) {
  const int r0 = (blockIdx.x * blockDim.x + threadIdx.x) * 4;
  if (r0 >= 2 * L) return;
  const int64_t L2 = 2 * (int64_t)L;
  const int64_t c0 = blockIdx.y * run, c1 = min(ncols, c0 + run);
  int64_t bcur = -1;
  float s[4];
  for (int64_t c = c0; c < c1; c += 4) {
    const int nc = (int)(c1 - c < 4 ? c1 - c : 4);
    float4 x[4];
#pragma unroll
    for (int q = 0; q < 4; ++q)
      if (q < nc) x[q] = *(const float4*)(V + r0 + (c + q) * L2);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      if (q >= nc) break;
      const int64_t b = (c + q) / N;
      if (b != bcur) {
        bcur = b;
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const int r = r0 + e;
          s[e] = (float)w[b * L + (r < L ? r : r - L)];
        }
      }
      float4 y = x[q];
      y.x *= s[0]; y.y *= s[1]; y.z *= s[2]; y.w *= s[3];
      const int64_t idx = r0 + (c + q) * L2;
      *(float4*)(V + idx) = y;
      __align__(8) __half h[4], l[4];
      split16(y.x, h[0], l[0]);
      split16(y.y, h[1], l[1]);
      split16(y.z, h[2], l[2]);
      split16(y.w, h[3], l[3]);
      *(uint2*)(Vh + idx) = *(const uint2*)h;
      *(uint2*)(Vl + idx) = *(const uint2*)l;
    }
  }
}

cudaError_t scale_rows_v(cudaStream_t st, float* V, __half* Vh, __half* Vl, int L, int N, int batch,
                         const double* w) {
  if (L % 2) return cudaErrorInvalidValue;
  const int64_t ncols = (int64_t)batch * N;
  const unsigned rblocks = (unsigned)FM_CEIL_DIV(2 * (int64_t)L, 1024);
  // about 8 resident blocks per SM in total, each over a run of columns
  const int64_t want = std::max<int64_t>(1, (int64_t)152 * 8 / rblocks);
  const int64_t run = std::max<int64_t>(4, ((ncols + want - 1) / want + 3) / 4 * 4);
  const unsigned cruns = (unsigned)FM_CEIL_DIV(ncols, run);
  scale_rows_v_kernel<<<dim3(rblocks, cruns), 256, 0, st>>>(V, Vh, Vl, L, N, ncols, run, w);
  return cudaGetLastError();
}

__global__ void split_planes_kernel(const float* __restrict__ x, __half* h, __half* l, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    __half a, b;
    split16(x[i], a, b);
    h[i] = a;
    l[i] = b;
  }
}

cudaError_t split_planes(cudaStream_t st, const float* x, __half* h, __half* l, int64_t n) {
  split_planes_kernel<<<152 * 8, 256, 0, st>>>(x, h, l, n);
  return cudaGetLastError();
}

// =================================================================== projective measurement
// One CTA (1024 threads) per trajectory processes the selected sites of one
// step in ascending order.  Per event: x = U_{j,:}, p = |x|^2, outcome u < p,
// v = U x^dag / sqrt(p), then U <- U + (v_new - v) x / sqrt(p) with v_new = e_j
// (click) or (v - sqrt(p) e_j)/sqrt(1-p) (no click).  Fixed-order reductions.
template <typename T, int LAYOUT>
struct uacc;
template <typename T>
struct uacc<T, 0> {  // complex128 U, L x N
  z64* U; int L;
  FM_DEVFN void init(void* base, int64_t b, int L_, int N) { L = L_; U = (z64*)base + b * L_ * (int64_t)N; }
  FM_DEVFN cplx<T> ld(int i, int k) const { z64 z = U[i + (int64_t)k * L]; return cmk<T>((T)z.re, (T)z.im); }
  FM_DEVFN void add(int i, int k, cplx<T> d) {
    z64& z = U[i + (int64_t)k * L]; z.re += d.re; z.im += d.im;
  }
};
template <typename T>
struct uacc<T, 1> {  // float V, 2L x N
  float* V; int L;
  FM_DEVFN void init(void* base, int64_t b, int L_, int N) { L = L_; V = (float*)base + b * 2 * L_ * (int64_t)N; }
  FM_DEVFN cplx<T> ld(int i, int k) const {
    const int64_t o = (int64_t)k * 2 * L;
    return cmk<T>((T)V[i + o], (T)V[L + i + o]);
  }
  FM_DEVFN void add(int i, int k, cplx<T> d) {
    const int64_t o = (int64_t)k * 2 * L;
    V[i + o] += (float)d.re; V[L + i + o] += (float)d.im;
  }
};

__device__ double block_sum_1024(double v, double* red) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if (lane == 0) red[warp] = v;
  __syncthreads();
  double s = 0.0;
  if (warp == 0) {
    s = (lane < (int)(blockDim.x >> 5)) ? red[lane] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) red[32] = s;
  }
  __syncthreads();
  s = red[32];
  __syncthreads();
  return s;
}

template <typename T, int LAYOUT>
__global__ void __launch_bounds__(1024) pm_kernel(pm_args a) {
  const int b = blockIdx.x;
  const int L = a.L, N = a.N;
  uacc<T, LAYOUT> u;
  u.init(a.U, b, L, N);
  cplx<T>* xb = (cplx<T>*)a.xbuf + (int64_t)b * N;
  cplx<T>* vb = (cplx<T>*)a.vbuf + (int64_t)b * L;
  const double g = a.gamma[b];
  const double pmeas = 1.0 - exp(-g * a.dt);
  const int64_t step = a.step[b];
  const uint64_t traj = a.traj[b];
  __shared__ int sel_site[1024];
  __shared__ double sel_u[1024];
  __shared__ int warp_cnt[33];
  __shared__ double red[33];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;

  for (int base = 0; base < L; base += 1024) {
    const int j = base + tid;
    bool s = false;
    double uo = 0.0;
    if (j < L) {
      philox_out o = fm_draw(a.seed, traj, step, j, FM_TAG_MEASURE);
      s = fm_u53(o.w[0], o.w[1]) < pmeas;
      uo = fm_u53(o.w[2], o.w[3]);
      if (s && a.force_n > 0) {
        const int fo = fm_forced_outcome(a.force, a.force_n, step, b, j);
        if (fo >= 0) uo = fm_forced_u(fo);
      }
    }
    const unsigned bal = __ballot_sync(0xffffffffu, s);
    if (lane == 0) warp_cnt[warp] = __popc(bal);
    __syncthreads();
    if (tid == 0) {
      int acc = 0;
      for (int w = 0; w < 32; ++w) { int c = warp_cnt[w]; warp_cnt[w] = acc; acc += c; }
      warp_cnt[32] = acc;
    }
    __syncthreads();
    if (s) {
      const int pos = warp_cnt[warp] + __popc(bal & ((1u << lane) - 1u));
      sel_site[pos] = j;
      sel_u[pos] = uo;
    }
    __syncthreads();
    const int nsel = warp_cnt[32];
    for (int e = 0; e < nsel; ++e) {
      const int js = sel_site[e];
      const double uu = sel_u[e];
      double ps = 0.0;
      for (int k = tid; k < N; k += 1024) {
        cplx<T> x = u.ld(js, k);
        xb[k] = x;
        ps += (double)x.re * x.re + (double)x.im * x.im;
      }
      double p = block_sum_1024(ps, red);  // includes __syncthreads: xb visible to the block
      p = fmin(fmax(p, 0.0), 1.0);
      const int outcome = (uu < p) ? 1 : 0;
      if (tid == 0 && a.log && a.log_capacity > 0) {
        unsigned long long slot = atomicAdd((unsigned long long*)a.log_count, 1ull);
        if (slot < (unsigned long long)a.log_capacity) {
          fm_event ev;
          ev.step = step; ev.traj = b; ev.site = js; ev.u = uu; ev.p = p; ev.outcome = outcome; ev.pad = 0;
          a.log[slot] = ev;
        }
      }
      if (p < 1e-300) continue;  // block-uniform
      const double sp = sqrt(p);
      const T inv_sp = (T)(1.0 / sp);
      for (int i = tid; i < L; i += 1024) {
        cplx<T> acc = cmk<T>(0, 0);
        for (int k = 0; k < N; ++k) cfma(acc, u.ld(i, k), cconj(xb[k]));
        vb[i] = cscale(acc, inv_sp);
      }
      __syncthreads();
      const T inv_s1 = (T)(outcome ? 0.0 : 1.0 / sqrt(1.0 - p));
      for (int i = tid; i < L; i += 1024) {
        const cplx<T> v = vb[i];
        cplx<T> vn;
        if (outcome) vn = cmk<T>(i == js ? (T)1 : (T)0, (T)0);
        else vn = cscale(cmk<T>(v.re - (i == js ? (T)sp : (T)0), v.im), inv_s1);
        const cplx<T> d = cscale(csub(vn, v), inv_sp);
        for (int k = 0; k < N; ++k) u.add(i, k, cmul(d, xb[k]));
      }
      __syncthreads();
    }
    __syncthreads();
  }
}

cudaError_t pm_measure(cudaStream_t st, const pm_args& a) {
  if (a.layout == 0) pm_kernel<double, 0><<<a.batch, 1024, 0, st>>>(a);
  else pm_kernel<float, 1><<<a.batch, 1024, 0, st>>>(a);
  return cudaGetLastError();
}

// ------------------------------------------------------------------ projective update, GPU-wide per event
// For lattices whose per-event passes are too large for one CTA: the sites of a
// step are selected first (list per trajectory, ascending), then every event e
// runs as three grid-wide kernels over all trajectories at once: the row x_j and
// its Born weight with the outcome (one CTA per trajectory), v = U x^dag / sqrt(p),
// and the rank-1 update U <- U + (v_new - v) x / sqrt(p).
struct PmEvent {
  double p, sp, inv_s1;
  int site, outcome, active, pad;
};

__global__ void __launch_bounds__(1024) pm_select_kernel(const double* gamma, double dt, const uint64_t* traj,
                                                         const int64_t* step, uint64_t seed, int L, int* list,
                                                         double* ulist, int* count, const int4* force,
                                                         int force_n) {
  const int b = blockIdx.x;
  const double pmeas = 1.0 - exp(-gamma[b] * dt);
  __shared__ int warp_cnt[33];
  __shared__ int base_sh;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (tid == 0) base_sh = 0;
  __syncthreads();
  for (int base = 0; base < L; base += 1024) {
    const int j = base + tid;
    bool sel = false;
    double uo = 0.0;
    if (j < L) {
      philox_out o = fm_draw(seed, traj[b], step[b], j, FM_TAG_MEASURE);
      sel = fm_u53(o.w[0], o.w[1]) < pmeas;
      uo = fm_u53(o.w[2], o.w[3]);
      if (sel && force_n > 0) {
        const int fo = fm_forced_outcome(force, force_n, step[b], b, j);
        if (fo >= 0) uo = fm_forced_u(fo);
      }
    }
    const unsigned bal = __ballot_sync(0xffffffffu, sel);
    if (lane == 0) warp_cnt[warp] = __popc(bal);
    __syncthreads();
    if (tid == 0) {
      int acc = 0;
      for (int w = 0; w < 32; ++w) { int c = warp_cnt[w]; warp_cnt[w] = acc; acc += c; }
      warp_cnt[32] = acc;
    }
    __syncthreads();
    if (sel) {
      const int pos = base_sh + warp_cnt[warp] + __popc(bal & ((1u << lane) - 1u));
      list[(int64_t)b * L + pos] = j;
      ulist[(int64_t)b * L + pos] = uo;
    }
    __syncthreads();
    if (tid == 0) base_sh += warp_cnt[32];
    __syncthreads();
  }
  if (tid == 0) count[b] = base_sh;
}

template <typename T, int LAYOUT>
__global__ void __launch_bounds__(1024) pm_row_kernel(void* Ub, int L, int N, int e, const int* list,
                                                      const double* ulist, int ld_list, const int* count,
                                                      const int64_t* step,
                                                      void* xbuf, PmEvent* ev, fm_event* log,
                                                      unsigned long long* log_count, int log_capacity) {
  const int b = blockIdx.x;
  __shared__ double red[33];
  uacc<T, LAYOUT> u;
  u.init(Ub, b, L, N);
  cplx<T>* xb = (cplx<T>*)xbuf + (int64_t)b * N;
  const bool has = e < count[b];
  const int js = has ? list[(int64_t)b * ld_list + e] : 0;
  double ps = 0.0;
  if (has)
    for (int k = threadIdx.x; k < N; k += blockDim.x) {
      const cplx<T> x = u.ld(js, k);
      xb[k] = x;
      ps += (double)x.re * x.re + (double)x.im * x.im;
    }
  double p = block_sum_1024(ps, red);
  if (threadIdx.x == 0) {
    PmEvent r;
    r.site = js;
    r.active = 0;
    r.outcome = 0;
    r.p = r.sp = r.inv_s1 = 0.0;
    r.pad = 0;
    if (has) {
      p = fmin(fmax(p, 0.0), 1.0);
      const double uu = ulist[(int64_t)b * ld_list + e];
      r.outcome = (uu < p) ? 1 : 0;
      r.p = p;
      r.sp = sqrt(p);
      r.inv_s1 = r.outcome ? 0.0 : 1.0 / sqrt(1.0 - p);
      r.active = (p >= 1e-300) ? 1 : 0;
      if (log && log_capacity > 0) {
        const unsigned long long slot = atomicAdd(log_count, 1ull);
        if (slot < (unsigned long long)log_capacity) {
          fm_event le;
          le.step = step[b]; le.traj = b; le.site = js; le.u = uu; le.p = p; le.outcome = r.outcome; le.pad = 0;
          log[slot] = le;
        }
      }
    }
    ev[b] = r;
  }
}

// v_i = sum_k U_ik conj(x_k) / sqrt(p); block (32 rows, 8 column phases), grid (ceil(L/32), 1, B)
template <typename T, int LAYOUT>
__global__ void pm_gemv_kernel(void* Ub, int L, int N, const void* xbuf, const PmEvent* ev, void* vbuf) {
  const int b = blockIdx.z;
  const PmEvent r = ev[b];
  if (!r.active) return;
  uacc<T, LAYOUT> u;
  u.init(Ub, b, L, N);
  const cplx<T>* xb = (const cplx<T>*)xbuf + (int64_t)b * N;
  const int i = blockIdx.x * 32 + threadIdx.x;
  cplx<T> acc = cmk<T>(0, 0);
  if (i < L)
    for (int k = threadIdx.y; k < N; k += 8) cfma(acc, u.ld(i, k), cconj(xb[k]));
  __shared__ cplx<T> red[8][33];
  red[threadIdx.y][threadIdx.x] = acc;
  __syncthreads();
  if (threadIdx.y == 0 && i < L) {
    cplx<T> s = cmk<T>(0, 0);
    for (int w = 0; w < 8; ++w) s = cadd(s, red[w][threadIdx.x]);
    ((cplx<T>*)vbuf)[(int64_t)b * L + i] = cscale(s, (T)(1.0 / r.sp));
  }
}

// U_ik += (v_new_i - v_i) x_k / sqrt(p); grid (ceil(L/256), column chunks, B)
template <typename T, int LAYOUT>
__global__ void pm_update_kernel(void* Ub, int L, int N, int kchunk, const void* xbuf, const PmEvent* ev,
                                 const void* vbuf) {
  const int b = blockIdx.z;
  const PmEvent r = ev[b];
  if (!r.active) return;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= L) return;
  uacc<T, LAYOUT> u;
  u.init(Ub, b, L, N);
  const cplx<T>* xb = (const cplx<T>*)xbuf + (int64_t)b * N;
  const cplx<T> v = ((const cplx<T>*)vbuf)[(int64_t)b * L + i];
  cplx<T> vn;
  if (r.outcome) vn = cmk<T>(i == r.site ? (T)1 : (T)0, (T)0);
  else vn = cscale(cmk<T>(v.re - (i == r.site ? (T)r.sp : (T)0), v.im), (T)r.inv_s1);
  const cplx<T> d = cscale(csub(vn, v), (T)(1.0 / r.sp));
  const int k0 = blockIdx.y * kchunk, k1 = min(N, k0 + kchunk);
  for (int k = k0; k < k1; ++k) u.add(i, k, cmul(d, xb[k]));
}

cudaError_t pm_select(cudaStream_t st, const pm_args& a, int* list, double* ulist, int* count) {
  pm_select_kernel<<<a.batch, 1024, 0, st>>>(a.gamma, a.dt, a.traj, a.step, a.seed, a.L, list, ulist, count,
                                             a.force, a.force_n);
  return cudaGetLastError();
}

cudaError_t pm_measure_wide(cudaStream_t st, const pm_args& a, void* scratch, int64_t* launches) {
  // scratch: list (B*L int), ulist (B*L double), count (B int), events (B PmEvent)
  char* s = (char*)scratch;
  int* list = (int*)s;
  s += (((int64_t)a.batch * a.L * 4) + 255) & ~(int64_t)255;
  double* ulist = (double*)s;
  s += (((int64_t)a.batch * a.L * 8) + 255) & ~(int64_t)255;
  int* count = (int*)s;
  s += (((int64_t)a.batch * 4) + 255) & ~(int64_t)255;
  PmEvent* ev = (PmEvent*)s;
  pm_select_kernel<<<a.batch, 1024, 0, st>>>(a.gamma, a.dt, a.traj, a.step, a.seed, a.L, list, ulist, count,
                                             a.force, a.force_n);
  cudaError_t e = cudaGetLastError();
  if (e) return e;
  ++*launches;
  std::vector<int> hc(a.batch);
  if ((e = cudaMemcpyAsync(hc.data(), count, 4 * a.batch, cudaMemcpyDeviceToHost, st))) return e;
  if ((e = cudaStreamSynchronize(st))) return e;
  int emax = 0;
  for (int c : hc) emax = std::max(emax, c);
  const int kchunk = std::max(32, FM_CEIL_DIV(a.N, std::max(1, (4 * 152) / std::max(1, FM_CEIL_DIV(a.L, 256) * a.batch))));
  const dim3 g_gemv(FM_CEIL_DIV(a.L, 32), 1, a.batch), g_upd(FM_CEIL_DIV(a.L, 256), FM_CEIL_DIV(a.N, kchunk), a.batch);
  for (int ev_i = 0; ev_i < emax; ++ev_i) {
    if (a.layout == 0) {
      pm_row_kernel<double, 0><<<a.batch, 1024, 0, st>>>(a.U, a.L, a.N, ev_i, list, ulist, a.L, count, a.step, a.xbuf, ev,
                                                         a.log, (unsigned long long*)a.log_count, a.log_capacity);
      pm_gemv_kernel<double, 0><<<g_gemv, dim3(32, 8), 0, st>>>(a.U, a.L, a.N, a.xbuf, ev, a.vbuf);
      pm_update_kernel<double, 0><<<g_upd, 256, 0, st>>>(a.U, a.L, a.N, kchunk, a.xbuf, ev, a.vbuf);
    } else {
      pm_row_kernel<float, 1><<<a.batch, 1024, 0, st>>>(a.U, a.L, a.N, ev_i, list, ulist, a.L, count, a.step, a.xbuf, ev,
                                                        a.log, (unsigned long long*)a.log_count, a.log_capacity);
      pm_gemv_kernel<float, 1><<<g_gemv, dim3(32, 8), 0, st>>>(a.U, a.L, a.N, a.xbuf, ev, a.vbuf);
      pm_update_kernel<float, 1><<<g_upd, 256, 0, st>>>(a.U, a.L, a.N, kchunk, a.xbuf, ev, a.vbuf);
    }
    if ((e = cudaGetLastError())) return e;
    *launches += 3;
  }
  return cudaSuccess;
}

cudaError_t pm_wide_event(cudaStream_t st, const pm_args& a, int e, const int* list, const double* ulist,
                          int ld_list, const int* count, void* scratch) {
  // the PmEvent array sits where pm_measure_wide keeps it in the same scratch
  char* s = (char*)scratch;
  s += (((int64_t)a.batch * a.L * 4) + 255) & ~(int64_t)255;
  s += (((int64_t)a.batch * a.L * 8) + 255) & ~(int64_t)255;
  s += (((int64_t)a.batch * 4) + 255) & ~(int64_t)255;
  PmEvent* ev = (PmEvent*)s;
  const int kchunk = std::max(32, FM_CEIL_DIV(a.N, std::max(1, (4 * 152) / std::max(1, FM_CEIL_DIV(a.L, 256) * a.batch))));
  const dim3 g_gemv(FM_CEIL_DIV(a.L, 32), 1, a.batch), g_upd(FM_CEIL_DIV(a.L, 256), FM_CEIL_DIV(a.N, kchunk), a.batch);
  if (a.layout == 0) {
    pm_row_kernel<double, 0><<<a.batch, 1024, 0, st>>>(a.U, a.L, a.N, e, list, ulist, ld_list, count, a.step, a.xbuf, ev, a.log,
                                                       (unsigned long long*)a.log_count, a.log_capacity);
    pm_gemv_kernel<double, 0><<<g_gemv, dim3(32, 8), 0, st>>>(a.U, a.L, a.N, a.xbuf, ev, a.vbuf);
    pm_update_kernel<double, 0><<<g_upd, 256, 0, st>>>(a.U, a.L, a.N, kchunk, a.xbuf, ev, a.vbuf);
  } else {
    pm_row_kernel<float, 1><<<a.batch, 1024, 0, st>>>(a.U, a.L, a.N, e, list, ulist, ld_list, count, a.step, a.xbuf, ev, a.log,
                                                      (unsigned long long*)a.log_count, a.log_capacity);
    pm_gemv_kernel<float, 1><<<g_gemv, dim3(32, 8), 0, st>>>(a.U, a.L, a.N, a.xbuf, ev, a.vbuf);
    pm_update_kernel<float, 1><<<g_upd, 256, 0, st>>>(a.U, a.L, a.N, kchunk, a.xbuf, ev, a.vbuf);
  }
  return cudaGetLastError();
}

size_t pm_wide_scratch_bytes(int L, int B) {
  auto al = [](int64_t x) { return (x + 255) & ~(int64_t)255; };
  return al((int64_t)B * L * 4) + al((int64_t)B * L * 8) + al((int64_t)B * 4) + al((int64_t)B * sizeof(PmEvent));
}

bool pm_use_wide(int L, int N, int B) { return !(B >= 64 && L <= 2048); }

// =================================================================== Cholesky pieces
// One CTA (32 x 32 threads) per trajectory: upper Cholesky of the nbk x nbk
// diagonal block at (k,k) of G (right-looking), written into R, and its
// triangular inverse into Dinv (nb x nb, column-major, block index k/nb).
template <typename T>
__global__ void __launch_bounds__(1024) chol_diag_kernel(const cplx<T>* __restrict__ G, int64_t ldg, int64_t sG,
                                                         cplx<T>* R, int64_t ldr, int64_t sR, cplx<T>* Dinv,
                                                         int64_t sD, int k, int nb, int nbk, int* status) {
  const int64_t b = blockIdx.x;
  G += b * sG;
  R += b * sR;
  Dinv += b * sD + (int64_t)(k / nb) * nb * nb;
  __shared__ cplx<T> A[32][33];
  __shared__ cplx<T> X[32][33];
  const int r = threadIdx.x / 32, c = threadIdx.x % 32;
  if (r < nbk && c < nbk) A[r][c] = G[(k + r) + (int64_t)(k + c) * ldg];
  else A[r][c] = cmk<T>(r == c ? (T)1 : (T)0, (T)0);
  __syncthreads();
  for (int j = 0; j < nbk; ++j) {
    if (threadIdx.x == 0) {
      T d = A[j][j].re;
      if (!(d > (T)0) || !isfinite(d)) { atomicOr(status, FM_DEVERR_PIVOT); d = (T)1; }
      A[j][j] = cmk<T>(sqrt(d), (T)0);
    }
    __syncthreads();
    if (r == j && c > j) A[j][c] = cscale(A[j][c], (T)1 / A[j][j].re);
    __syncthreads();
    if (r > j && c >= r) A[r][c] = csub(A[r][c], cmul(cconj(A[j][r]), A[j][c]));
    __syncthreads();
  }
  if (r < nbk && c < nbk) R[(k + r) + (int64_t)(k + c) * ldr] = (r <= c) ? A[r][c] : cmk<T>((T)0, (T)0);
  // inverse of the upper-triangular block, one column per thread
  if (threadIdx.x < 32) {
    const int cc = threadIdx.x;
    for (int i = 31; i >= 0; --i) {
      if (i > cc) { X[i][cc] = cmk<T>((T)0, (T)0); continue; }
      cplx<T> s = cmk<T>(i == cc ? (T)1 : (T)0, (T)0);
      for (int l = i + 1; l <= cc; ++l) s = csub(s, cmul(A[i][l], X[l][cc]));
      X[i][cc] = cscale(s, (T)1 / A[i][i].re);
    }
  }
  __syncthreads();
  if (r < nb && c < nb) Dinv[r + (int64_t)c * nb] = (r < nbk && c < nbk) ? X[r][c] : cmk<T>((T)0, (T)0);
}

template <typename T>
cudaError_t chol_diag_block(cudaStream_t st, const cplx<T>* G, int64_t ldg, int64_t sG, cplx<T>* R, int64_t ldr,
                            int64_t sR, cplx<T>* Dinv, int64_t sD, int k, int nb, int nbk, int batch, int* status) {
  chol_diag_kernel<T><<<batch, 1024, 0, st>>>(G, ldg, sG, R, ldr, sR, Dinv, sD, k, nb, nbk, status);
  return cudaGetLastError();
}
template cudaError_t chol_diag_block<double>(cudaStream_t, const z64*, int64_t, int64_t, z64*, int64_t, int64_t, z64*,
                                             int64_t, int, int, int, int, int*);
template cudaError_t chol_diag_block<float>(cudaStream_t, const c32*, int64_t, int64_t, c32*, int64_t, int64_t, c32*,
                                            int64_t, int, int, int, int, int*);

template <typename T>
__global__ void place_diag_blocks_kernel(const cplx<T>* __restrict__ Dinv, int64_t sD, cplx<T>* Tm, int64_t ldt,
                                         int64_t sT, int N, int nb) {
  const int64_t b = blockIdx.y;
  const int64_t tot = (int64_t)N * N;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < tot;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(idx % N), j = (int)(idx / N);
    cplx<T> v = cmk<T>((T)0, (T)0);
    if (i / nb == j / nb) {
      const int blk = i / nb;
      v = Dinv[b * sD + (int64_t)blk * nb * nb + (i % nb) + (int64_t)(j % nb) * nb];
    }
    Tm[b * sT + i + (int64_t)j * ldt] = v;
  }
}

template <typename T>
cudaError_t place_diag_blocks(cudaStream_t st, const cplx<T>* Dinv, int64_t sD, cplx<T>* Tm, int64_t ldt, int64_t sT,
                              int N, int nb, int batch) {
  dim3 grid((unsigned)min(FM_CEIL_DIV((int64_t)N * N, 256), (int64_t)2048), batch);
  place_diag_blocks_kernel<T><<<grid, 256, 0, st>>>(Dinv, sD, Tm, ldt, sT, N, nb);
  return cudaGetLastError();
}
template cudaError_t place_diag_blocks<double>(cudaStream_t, const z64*, int64_t, z64*, int64_t, int64_t, int, int, int);
template cudaError_t place_diag_blocks<float>(cudaStream_t, const c32*, int64_t, c32*, int64_t, int64_t, int, int, int);

__global__ void zero_lower_kernel(z64* R, int64_t ldr, int64_t sR, int N) {
  const int64_t b = blockIdx.y;
  const int64_t tot = (int64_t)N * N;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < tot;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(idx % N), j = (int)(idx / N);
    if (i > j) R[b * sR + i + (int64_t)j * ldr] = cmk(0.0, 0.0);
  }
}

cudaError_t zero_lower(cudaStream_t st, z64* R, int64_t ldr, int64_t sR, int N, int batch) {
  dim3 grid(min(FM_CEIL_DIV((int64_t)N * N, 256), (int64_t)2048), batch);
  zero_lower_kernel<<<grid, 256, 0, st>>>(R, ldr, sR, N);
  return cudaGetLastError();
}

// =================================================================== layout / misc
__global__ void gather_rows_z_kernel(const z64* __restrict__ U, int L, int N, const int* rows, int nrows, z64* out) {
  const int64_t tot = (int64_t)nrows * N;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < tot;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int a = (int)(idx % nrows);
    const int64_t k = idx / nrows;
    out[idx] = U[rows[a] + k * L];
  }
}
cudaError_t gather_rows_z(cudaStream_t st, const z64* U, int L, int N, const int* rows, int nrows, z64* out) {
  gather_rows_z_kernel<<<152 * 4, 256, 0, st>>>(U, L, N, rows, nrows, out);
  return cudaGetLastError();
}

__global__ void gather_rows_v_kernel(const float* __restrict__ V, int L, int N, const int* rows, int nrows,
                                     z64* out) {
  const int64_t tot = (int64_t)nrows * N;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < tot;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int a = (int)(idx % nrows);
    const int64_t k = idx / nrows;
    const int64_t o = k * 2 * L + rows[a];
    out[idx] = cmk((double)V[o], (double)V[o + L]);
  }
}
cudaError_t gather_rows_v(cudaStream_t st, const float* V, int L, int N, const int* rows, int nrows, z64* out) {
  gather_rows_v_kernel<<<152 * 4, 256, 0, st>>>(V, L, N, rows, nrows, out);
  return cudaGetLastError();
}

__global__ void v_to_z_kernel(const float* __restrict__ V, int L, int N, z64* U) {
  const int64_t tot = (int64_t)L * N;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < tot;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = idx % L, k = idx / L;
    U[idx] = cmk((double)V[i + k * 2 * L], (double)V[L + i + k * 2 * L]);
  }
}
cudaError_t v_to_z(cudaStream_t st, const float* V, int L, int N, z64* U) {
  v_to_z_kernel<<<152 * 4, 256, 0, st>>>(V, L, N, U);
  return cudaGetLastError();
}

__global__ void z_to_v_kernel(const z64* __restrict__ U, int L, int N, float* V, __half* Vh, __half* Vl) {
  const int64_t tot = (int64_t)L * N;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < tot;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = idx % L, k = idx / L;
    const z64 z = U[idx];
    const int64_t o = i + k * 2 * L;
    const float re = (float)z.re, im = (float)z.im;
    V[o] = re;
    V[o + L] = im;
    __half h, l;
    split16(re, h, l); Vh[o] = h; Vl[o] = l;
    split16(im, h, l); Vh[o + L] = h; Vl[o + L] = l;
  }
}
cudaError_t z_to_v(cudaStream_t st, const z64* U, int L, int N, float* V, __half* Vh, __half* Vl) {
  z_to_v_kernel<<<152 * 4, 256, 0, st>>>(U, L, N, V, Vh, Vl);
  return cudaGetLastError();
}

// U_b = 0 except U_b(occ[k], k) = 1
__global__ void neel_z_kernel(z64* U, int L, int N, int batch, const int* occ) {
  const int64_t tot = (int64_t)L * N * batch;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < tot;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = idx % L, k = (idx / L) % N;
    U[idx] = cmk(occ[k] == i ? 1.0 : 0.0, 0.0);
  }
}
__global__ void neel_v_kernel(float* V, __half* Vh, __half* Vl, int L, int N, int batch, const int* occ) {
  const int64_t tot = (int64_t)2 * L * N * batch;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < tot;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = idx % (2 * L), k = (idx / (2 * L)) % N;
    const float x = (occ[k] == r) ? 1.0f : 0.0f;   // r < L: real part
    V[idx] = x;
    Vh[idx] = __float2half_rn(x);
    Vl[idx] = __float2half_rn(0.0f);
  }
}
cudaError_t neel_init_z(cudaStream_t st, z64* U, int L, int N, int batch, const int* occ) {
  neel_z_kernel<<<152 * 4, 256, 0, st>>>(U, L, N, batch, occ);
  return cudaGetLastError();
}
cudaError_t neel_init_v(cudaStream_t st, float* V, __half* Vh, __half* Vl, int L, int N, int batch,
                        const int* occ) {
  neel_v_kernel<<<152 * 4, 256, 0, st>>>(V, Vh, Vl, L, N, batch, occ);
  return cudaGetLastError();
}

// dense P (L x L, column-major) from the ring rows px (Lx), py (Ly):
// P[(x,y),(x',y')] = px[(x-x') mod Lx] py[(y-y') mod Ly]
__global__ void expand_p_z_kernel(const z64* __restrict__ px, const z64* __restrict__ py, int Lx, int Ly, z64* P) {
  const int L = Lx * Ly;
  const int64_t tot = (int64_t)L * L;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < tot;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int a = (int)(idx % L), c = (int)(idx / L);
    const int xa = a % Lx, ya = a / Lx, xc = c % Lx, yc = c / Lx;
    const z64 vx = px[((xa - xc) % Lx + Lx) % Lx];
    const z64 vy = py[((ya - yc) % Ly + Ly) % Ly];
    P[idx] = cmul(vx, vy);
  }
}
cudaError_t expand_propagator_z(cudaStream_t st, const z64* px, const z64* py, int Lx, int Ly, z64* P) {
  expand_p_z_kernel<<<152 * 8, 256, 0, st>>>(px, py, Lx, Ly, P);
  return cudaGetLastError();
}

// real 2L x 2L embedding [[Re P, -Im P], [Im P, Re P]], row-major (K contiguous),
// as split-fp16 planes.
__global__ void expand_p_planes_kernel(const z64* __restrict__ px, const z64* __restrict__ py, int Lx, int Ly,
                                       __half* Ah, __half* Al) {
  const int L = Lx * Ly;
  const int64_t L2 = 2 * (int64_t)L;
  const int64_t tot = L2 * L2;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < tot;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = idx / L2, s = idx % L2;
    const int a = (int)(r % L), c = (int)(s % L);
    const int xa = a % Lx, ya = a / Lx, xc = c % Lx, yc = c / Lx;
    const z64 z = cmul(px[((xa - xc) % Lx + Lx) % Lx], py[((ya - yc) % Ly + Ly) % Ly]);
    const bool rb = r >= L, sb = s >= L;
    const double v = (!rb && !sb) ? z.re : (!rb && sb) ? -z.im : (rb && !sb) ? z.im : z.re;
    __half h, l;
    split16((float)v, h, l);
    // refine the low plane against the FP64 value
    l = __float2half_rn((float)((v - (double)__half2float(h)) * 2048.0));
    Ah[idx] = h;
    Al[idx] = l;
  }
}
cudaError_t expand_propagator_planes(cudaStream_t st, const z64* px, const z64* py, int Lx, int Ly, __half* Ah,
                                     __half* Al) {
  expand_p_planes_kernel<<<152 * 8, 256, 0, st>>>(px, py, Lx, Ly, Ah, Al);
  return cudaGetLastError();
}

__global__ void bump_steps_kernel(int64_t* step, int batch) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b < batch) step[b] += 1;
}
cudaError_t bump_steps(cudaStream_t st, int64_t* step, int batch) {
  bump_steps_kernel<<<FM_CEIL_DIV(batch, 256), 256, 0, st>>>(step, batch);
  return cudaGetLastError();
}

// out must be zeroed; |x| >= 0 doubles order like their int64 bit patterns.
__global__ void max_abs_minus_identity_kernel(const z64* __restrict__ G, int ncols, int N, const int* cols,
                                              unsigned long long* out) {
  const int64_t tot = (int64_t)ncols * N;
  double m = 0.0;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < tot;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int a = (int)(idx % ncols);
    const int l = (int)(idx / ncols);
    z64 g = G[idx];
    if (cols[a] == l) g.re -= 1.0;
    m = fmax(m, sqrt(cabs2(g)));
  }
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) atomicMax(out, (unsigned long long)__double_as_longlong(m));
}
cudaError_t max_abs_minus_identity(cudaStream_t st, const z64* G, int ncols, int N, const int* cols, double* out) {
  max_abs_minus_identity_kernel<<<152, 256, 0, st>>>(G, ncols, N, cols, (unsigned long long*)out);
  return cudaGetLastError();
}

__global__ void check_finite_z_kernel(const z64* __restrict__ X, int64_t n, int* status) {
  bool bad = false;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const z64 z = X[i];
    bad |= !isfinite(z.re) || !isfinite(z.im);
  }
  if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(status, FM_DEVERR_NONFINITE);
}
cudaError_t check_finite_z(cudaStream_t st, const z64* X, int64_t n, int* status) {
  check_finite_z_kernel<<<152 * 2, 256, 0, st>>>(X, n, status);
  return cudaGetLastError();
}

}  // namespace fm
